// Diagonally preconditioned Davidson for the lowest roots of H on V
// (Sec. II.A; the cached diagonal of Sec. IV.B is the preconditioner).
//
// Everything runs on the device in FP64: the block sigma product, the
// projected matrix V^T H V, its eigen-decomposition (a parallel cyclic Jacobi
// solver in one CTA), Ritz vectors, residuals, the preconditioner and the
// Gram-Schmidt orthogonalisation.  The host only sequences launches and reads
// a few scalars (Ritz values, residual norms) once per iteration.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "context.cuh"


namespace shci {

constexpr int DV_THREADS = 256;
constexpr int DOT_ROWS = 16;  // partial-sum slots per block for A-rows

// rows of A handled per multi-dot launch for NB columns of B (NA * NB <= 16)
template <int NB>
struct DotShape {
    static constexpr int NA = NB >= 16 ? 1 : 16 / NB;
};

// partial[blk][a][b] = sum over this block's slice of A[a][i] * B[b][i]
// for a < na (<= NA), b < NB
template <int NB>
__global__ void __launch_bounds__(DV_THREADS) k_multidot(const double *__restrict__ A, int na,
                                                        const double *__restrict__ B, int64_t n,
                                                        double *__restrict__ partial) {
    constexpr int NA = DotShape<NB>::NA;
    double acc[NA][NB];
#pragma unroll
    for (int a = 0; a < NA; a++)
#pragma unroll
        for (int b = 0; b < NB; b++) acc[a][b] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)DV_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DV_THREADS) {
        double bv[NB];
#pragma unroll
        for (int b = 0; b < NB; b++) bv[b] = B[b * n + i];
#pragma unroll
        for (int a = 0; a < NA; a++) {
            if (a < na) {
                const double av = A[a * n + i];
#pragma unroll
                for (int b = 0; b < NB; b++) acc[a][b] = fma(av, bv[b], acc[a][b]);
            }
        }
    }
    __shared__ double red[NA * NB][DV_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < NA; a++) {
#pragma unroll
        for (int b = 0; b < NB; b++) {
            double v = acc[a][b];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[a * NB + b][w] = v;
        }
    }
    __syncthreads();
    const int e = threadIdx.x;
    if (e < na * NB) {
        double s = 0.0;
#pragma unroll
        for (int x = 0; x < DV_THREADS / 32; x++) s += red[e][x];
        partial[(int64_t)blockIdx.x * DOT_ROWS * SHCI_MAX_K + (e / NB) * SHCI_MAX_K + (e % NB)] = s;
    }
}

// out[(a0 + a) * ld + b0 + b] = sum_blk partial[blk][a][b]  (and the mirror when sym)
__global__ void k_multidot_final(const double *__restrict__ partial, int nblk, int na, int nb, double *out, int ld,
                                 int a0, int b0, int sym) {
    int e = threadIdx.x;
    if (e >= na * nb) return;
    int a = e / nb, b = e % nb;
    double s = 0.0;
    for (int k = 0; k < nblk; k++) s += partial[(int64_t)k * DOT_ROWS * SHCI_MAX_K + a * SHCI_MAX_K + b];
    out[(a0 + a) * ld + b0 + b] = s;
    if (sym) out[(b0 + b) * ld + a0 + a] = s;
}

// ---------------------------------------------------------------- vector kernels

// X[i*k + b] = V[b][i]
__global__ void k_pack(const double *__restrict__ V, int k, int64_t n, double *__restrict__ X) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int b = 0; b < k; b++) X[i * k + b] = V[b * n + i];
}

__global__ void k_unpack(const double *__restrict__ X, int k, int64_t n, double *__restrict__ V) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int b = 0; b < k; b++) V[b * n + i] = X[i * k + b];
}

// T[l] -= sum_a C[a * ldc + l] * V[a]   for a < m, l < kb
__global__ void k_project_out(const double *__restrict__ V, int m, const double *__restrict__ C, int ldc, int kb,
                              int64_t n, double *__restrict__ T) {
    __shared__ double cs[SHCI_MAX_SUB * SHCI_MAX_K];
    for (int e = threadIdx.x; e < m * kb; e += blockDim.x) cs[e] = C[(e / kb) * ldc + (e % kb)];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t[SHCI_MAX_K];
#pragma unroll
        for (int l = 0; l < SHCI_MAX_K; l++) t[l] = l < kb ? T[l * n + i] : 0.0;
        for (int a = 0; a < m; a++) {
            const double v = V[a * n + i];
#pragma unroll
            for (int l = 0; l < SHCI_MAX_K; l++)
                if (l < kb) t[l] = fma(-cs[a * kb + l], v, t[l]);
        }
#pragma unroll
        for (int l = 0; l < SHCI_MAX_K; l++)
            if (l < kb) T[l * n + i] = t[l];
    }
}

// dst = src * (1 / sqrt(nrm2[0])) or zero if the norm is below tiny
__global__ void k_normalize(const double *__restrict__ src, const double *__restrict__ nrm2, int64_t n,
                            double *__restrict__ dst) {
    double s2 = nrm2[0];
    double f = s2 > 1e-26 ? 1.0 / sqrt(s2) : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] * f;
}

// Ritz vectors and residuals for roots l < k of the subspace of size m:
//   x_l = sum_a Y[a][l] V[a],  h_l = sum_a Y[a][l] AV[a],  r_l = h_l - theta_l x_l
// mode 0: T[l] = r_l / (theta_l - H_ii) (clamped), partial |r_l|^2 per block
// mode 1: X[l] = x_l, H[l] = h_l (restart / output)
__global__ void __launch_bounds__(DV_THREADS) k_ritz(const double *__restrict__ V, const double *__restrict__ AV,
                                                     int m, const double *__restrict__ evec, int ld,
                                                     const double *__restrict__ eval, int k, int64_t n,
                                                     const double *__restrict__ diag, int mode,
                                                     double *__restrict__ T, double *__restrict__ Xo,
                                                     double *__restrict__ Ho, double *__restrict__ partial) {
    __shared__ double ys[SHCI_MAX_SUB * SHCI_MAX_K];
    __shared__ double th[SHCI_MAX_K];
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) ys[e] = evec[(e % k) * ld + (e / k)];   // ys[a*k+l]
    if (threadIdx.x < k) th[threadIdx.x] = eval[threadIdx.x];
    __syncthreads();
    double rn[SHCI_MAX_K];
#pragma unroll
    for (int l = 0; l < SHCI_MAX_K; l++) rn[l] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)DV_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DV_THREADS) {
        double x[SHCI_MAX_K], h[SHCI_MAX_K];
#pragma unroll
        for (int l = 0; l < SHCI_MAX_K; l++) { x[l] = 0.0; h[l] = 0.0; }
        for (int a = 0; a < m; a++) {
            const double v = V[a * n + i], av = AV[a * n + i];
#pragma unroll
            for (int l = 0; l < SHCI_MAX_K; l++) {
                if (l < k) {
                    x[l] = fma(ys[a * k + l], v, x[l]);
                    h[l] = fma(ys[a * k + l], av, h[l]);
                }
            }
        }
        if (mode == 0) {
            const double d = diag[i];
#pragma unroll
            for (int l = 0; l < SHCI_MAX_K; l++) {
                if (l < k) {
                    const double r = fma(-th[l], x[l], h[l]);
                    rn[l] = fma(r, r, rn[l]);
                    double den = th[l] - d;
                    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
                    T[l * n + i] = r / den;
                }
            }
        } else {
#pragma unroll
            for (int l = 0; l < SHCI_MAX_K; l++) {
                if (l < k) {
                    Xo[l * n + i] = x[l];
                    Ho[l * n + i] = h[l];
                }
            }
        }
    }
    if (mode == 0) {
        __shared__ double red[DV_THREADS / 32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int l = 0; l < k; l++) {
            double v = rn[l];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[w] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s = 0.0;
                for (int x = 0; x < DV_THREADS / 32; x++) s += red[x];
                partial[(int64_t)blockIdx.x * SHCI_MAX_K + l] = s;
            }
            __syncthreads();
        }
    }
}

__global__ void k_sum_partials(const double *__restrict__ partial, int nblk, int k, double *__restrict__ out) {
    int l = threadIdx.x;
    if (l >= k) return;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += partial[(int64_t)b * SHCI_MAX_K + l];
    out[l] = s;
}

// ---------------------------------------------------------------- subspace eigensolver

// Eigen-decomposition of the symmetric m x m matrix G (row-major, leading
// dimension ld) by cyclic Jacobi with Brent-Luk parallel ordering: each round
// applies m/2 disjoint rotations at once.  Outputs eigenvalues ascending and
// eigenvectors as columns: evec[l * ld + a] = component a of vector l.
__global__ void k_jacobi(const double *__restrict__ G, int ld, int m, double *__restrict__ eval,
                         double *__restrict__ evec) {
    extern __shared__ double jsm[];
    double (*A)[SHCI_MAX_SUB + 1] = reinterpret_cast<double (*)[SHCI_MAX_SUB + 1]>(jsm);
    double (*Q)[SHCI_MAX_SUB + 1] = reinterpret_cast<double (*)[SHCI_MAX_SUB + 1]>(jsm + SHCI_MAX_SUB * (SHCI_MAX_SUB + 1));
    __shared__ double cs[SHCI_MAX_SUB / 2], sn[SHCI_MAX_SUB / 2];
    __shared__ int pp[SHCI_MAX_SUB / 2], qq[SHCI_MAX_SUB / 2];
    __shared__ double red[32];
    __shared__ int done;
    const int mm = (m + 1) & ~1;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < mm * mm; e += nt) {
        int r = e / mm, c = e % mm;
        double v;
        if (r < m && c < m) v = 0.5 * (G[r * ld + c] + G[c * ld + r]);
        else v = 0.0;
        A[r][c] = v;
        Q[r][c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (mm != m) {
        // padding index: decoupled, with a diagonal value above every Gershgorin bound
        if (tid == 0) {
            double bound = 0.0;
            for (int r = 0; r < m; r++) {
                double s = 0.0;
                for (int c = 0; c < m; c++) s += fabs(A[r][c]);
                bound = fmax(bound, s);
            }
            A[m][m] = 2.0 * bound + 1.0;
        }
        __syncthreads();
    }
    for (int sweep = 0; sweep < 60; sweep++) {
        // convergence test on the off-diagonal Frobenius norm
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < mm * mm; e += nt) {
            int r = e / mm, c = e % mm;
            double v = A[r][c] * A[r][c];
            tot += v;
            if (r != c) off += v;
        }
        for (int o = 16; o >= 1; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((tid & 31) == 0) {
            red[tid >> 5] = off;
            red[16 + (tid >> 5)] = tot;
        }
        __syncthreads();
        if (tid == 0) {
            double so = 0.0, st = 0.0;
            for (int x = 0; x < nt / 32; x++) {
                so += red[x];
                st += red[16 + x];
            }
            done = (so <= 1e-30 * st) || (so < 1e-300);
        }
        __syncthreads();
        if (done) break;
        for (int round = 0; round < mm - 1; round++) {
            if (tid < mm / 2) {
                int x = tid, y = mm - 1 - tid;
                int p = x == 0 ? 0 : ((x - 1 + round) % (mm - 1)) + 1;
                int q = y == 0 ? 0 : ((y - 1 + round) % (mm - 1)) + 1;
                if (p > q) { int t = p; p = q; q = t; }
                double apq = A[p][q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
                    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[tid] = c;
                sn[tid] = s;
                pp[tid] = p;
                qq[tid] = q;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < (mm / 2) * mm; e += nt) {
                int t = e / mm, j = e % mm;
                int p = pp[t], q = qq[t];
                double c = cs[t], s = sn[t];
                double ap = A[p][j], aq = A[q][j];
                A[p][j] = c * ap - s * aq;
                A[q][j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, Q <- Q J
            for (int e = tid; e < (mm / 2) * mm; e += nt) {
                int t = e / mm, i = e % mm;
                int p = pp[t], q = qq[t];
                double c = cs[t], s = sn[t];
                double ap = A[i][p], aq = A[i][q];
                A[i][p] = c * ap - s * aq;
                A[i][q] = s * ap + c * aq;
                double qp = Q[i][p], qv = Q[i][q];
                Q[i][p] = c * qp - s * qv;
                Q[i][q] = s * qp + c * qv;
            }
            __syncthreads();
        }
    }
    // sort ascending (rank by value, ties by index) and write out the first m
    for (int a = tid; a < mm; a += nt) {
        double va = A[a][a];
        int rank = 0;
        for (int b = 0; b < mm; b++) {
            double vb = A[b][b];
            rank += (vb < va) || (vb == va && b < a);
        }
        if (rank < m) {
            eval[rank] = va;
            for (int r = 0; r < m; r++) evec[rank * ld + r] = Q[r][a];
        }
    }
}

constexpr size_t JACOBI_SMEM = sizeof(double) * 2 * SHCI_MAX_SUB * (SHCI_MAX_SUB + 1);

// ---------------------------------------------------------------- guesses

__global__ void k_argmin_partial(const double *__restrict__ d, int64_t n, const int64_t *__restrict__ excl,
                                 int n_excl, double *__restrict__ pv, int64_t *__restrict__ pi) {
    double best = INFINITY;
    int64_t bi = INT64_MAX;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        bool skip = false;
        for (int e = 0; e < n_excl; e++) skip |= excl[e] == i;
        if (skip) continue;
        double v = d[i];
        if (v < best || (v == best && i < bi)) { best = v; bi = i; }
    }
    for (int o = 16; o >= 1; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, best, o);
        int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov < best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    __shared__ double sv[32];
    __shared__ int64_t si[32];
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++)
            if (sv[w] < best || (sv[w] == best && si[w] < bi)) { best = sv[w]; bi = si[w]; }
        pv[blockIdx.x] = best;
        pi[blockIdx.x] = bi;
    }
}

__global__ void k_argmin_final(const double *__restrict__ pv, const int64_t *__restrict__ pi, int nb,
                               int64_t *__restrict__ excl, int slot) {
    if (threadIdx.x != 0) return;
    double best = INFINITY;
    int64_t bi = INT64_MAX;
    for (int b = 0; b < nb; b++)
        if (pv[b] < best || (pv[b] == best && pi[b] < bi)) { best = pv[b]; bi = pi[b]; }
    excl[slot] = bi;
}

__global__ void k_unit_vectors(const int64_t *__restrict__ idx, int k, int64_t n, double *__restrict__ V) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)k * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int l = (int)(e / n);
        int64_t i = e % n;
        V[e] = (i == idx[l]) ? 1.0 : 0.0;
    }
}

// ---------------------------------------------------------------- host driver

struct Dav {
    shci_ctx *c;
    int64_t n;
    int k, m_max, keep;
    int dot_blocks, vec_blocks;
    cudaStream_t st;

    double *Vr(int a) { return c->dw.V.p + (int64_t)a * n; }
    double *AVr(int a) { return c->dw.AV.p + (int64_t)a * n; }

    // out[a0 + a][b0 + b] (ld) = A[a] . B[b], a < na, b < nb; mirror if sym
    template <int NB>
    void dots_nb(const double *A, int na, const double *B, double *out, int ld, int a0, int b0, bool sym) {
        constexpr int NA = DotShape<NB>::NA;
        for (int base = 0; base < na; base += NA) {
            int cnt = std::min(NA, na - base);
            k_multidot<NB><<<dot_blocks, DV_THREADS, 0, st>>>(A + (int64_t)base * n, cnt, B, n, c->dw.partial.p);
            k_multidot_final<<<1, DOT_ROWS * SHCI_MAX_K, 0, st>>>(c->dw.partial.p, dot_blocks, cnt, NB, out, ld,
                                                                  a0 + base, b0, sym ? 1 : 0);
            KERNEL_CHECK();
            g_kernel_launches += 2;
        }
    }

    // out[a0 + a][b0 + b] (ld) = A[a] . B[b], a < na, b < nb; mirror if sym
    void dots(const double *A, int na, const double *B, int nb, double *out, int ld, int a0, int b0, bool sym) {
        int b = 0;
        while (b < nb) {
            int left = nb - b;
            const double *Bb = B + (int64_t)b * n;
            if (left >= 8) { dots_nb<8>(A, na, Bb, out, ld, a0, b0 + b, sym); b += 8; }
            else if (left >= 4) { dots_nb<4>(A, na, Bb, out, ld, a0, b0 + b, sym); b += 4; }
            else if (left >= 2) { dots_nb<2>(A, na, Bb, out, ld, a0, b0 + b, sym); b += 2; }
            else { dots_nb<1>(A, na, Bb, out, ld, a0, b0 + b, sym); b += 1; }
        }
    }

    // orthonormalise the kb vectors T[0..kb) against V[0..m) and each other,
    // appending the accepted ones to V; returns how many were accepted
    int orthonormalize_append(double *T, int kb, int m) {
        double *coef = c->dw.small.p;                 // [SHCI_MAX_SUB][SHCI_MAX_K]
        double *nrm = c->dw.small.p + SHCI_MAX_SUB * SHCI_MAX_K;
        int added = 0;
        for (int l = 0; l < kb; l++) {
            double *t = T + (int64_t)l * n;
            int mb = m + added;
            for (int pass = 0; pass < 2; pass++) {
                if (mb > 0) {
                    dots(c->dw.V.p, mb, t, 1, coef, 1, 0, 0, false);
                    k_project_out<<<vec_blocks, DV_THREADS, 0, st>>>(c->dw.V.p, mb, coef, 1, 1, n, t);
                    KERNEL_CHECK();
                    g_kernel_launches += 1;
                }
            }
            dots(t, 1, t, 1, nrm, 1, 0, 0, false);
            double h_n = 0.0;
            CUDA_TRY(cudaMemcpyAsync(&h_n, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (!(h_n > 1e-20)) continue;            // linearly dependent: drop
            k_normalize<<<vec_blocks, DV_THREADS, 0, st>>>(t, nrm, n, Vr(mb));
            KERNEL_CHECK();
            g_kernel_launches += 1;
            added++;
        }
        return added;
    }

    // AV[m0 .. m0 + kb) = H V[m0 .. m0 + kb); G columns updated
    void expand(int m0, int kb) {
        k_pack<<<vec_blocks, DV_THREADS, 0, st>>>(Vr(m0), kb, n, c->dw.X.p);
        KERNEL_CHECK();
        sigma(c, kb, c->dw.X.p, c->dw.Y.p, true);
        k_unpack<<<vec_blocks, DV_THREADS, 0, st>>>(c->dw.Y.p, kb, n, AVr(m0));
        KERNEL_CHECK();
        g_kernel_launches += 2;
        dots(c->dw.V.p, m0 + kb, AVr(m0), kb, c->dw.G.p, m_max, 0, m0, true);
    }
};

int davidson(shci_ctx *c, int k, double tol, int max_iter, const double *guess, double *energies, double *vecs,
             int mem, int *iters_out) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before Davidson"};
    if (k < 1 || k > SHCI_MAX_K) throw ShciError{SHCI_ERR_INVALID, "k_roots must be in [1, 8]"};
    if (k > c->n_det) throw ShciError{SHCI_ERR_INVALID, "k_roots exceeds the number of determinants"};
    if (!(tol > 0.0)) throw ShciError{SHCI_ERR_INVALID, "tol must be positive"};
    if (max_iter < 1) throw ShciError{SHCI_ERR_INVALID, "max_iter must be >= 1"};
    if (!energies) throw ShciError{SHCI_ERR_INVALID, "energies must not be NULL"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    static bool jacobi_attr = false;
    if (!jacobi_attr) {
        CUDA_TRY(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JACOBI_SMEM));
        jacobi_attr = true;
    }
    Dav d;
    d.c = c;
    d.n = c->n_det;
    d.k = k;
    d.st = c->st;
    d.m_max = (int)std::min<int64_t>(std::min(SHCI_MAX_SUB, 16 + 16 * k), c->n_det);
    if (d.m_max < k) d.m_max = k;
    d.keep = std::max(k, std::min(d.m_max - k, std::max(2 * k, d.m_max / 3)));
    d.dot_blocks = std::max(1, std::min<int>((int)ceil_div(d.n, DV_THREADS * 8), c->n_sm * 4));
    d.vec_blocks = std::max(1, std::min<int>((int)ceil_div(d.n, DV_THREADS), c->n_sm * 8));
    const int64_t n = d.n;
    const double res_tol = 0.1 * std::sqrt(tol);
    DavidsonWork &w = c->dw;
    w.V.alloc((size_t)d.m_max * n);
    w.AV.alloc((size_t)d.m_max * n);
    w.X.alloc((size_t)SHCI_MAX_K * n);
    w.Y.alloc((size_t)SHCI_MAX_K * n);
    w.T.alloc((size_t)2 * SHCI_MAX_K * n);
    w.RV.alloc((size_t)d.keep * n);
    w.RAV.alloc((size_t)d.keep * n);
    w.G.alloc((size_t)d.m_max * d.m_max);
    w.evec.alloc((size_t)d.m_max * d.m_max);
    w.eval.alloc((size_t)d.m_max);
    w.partial.alloc((size_t)std::max(d.dot_blocks, d.vec_blocks) * DOT_ROWS * SHCI_MAX_K);
    w.small.alloc((size_t)SHCI_MAX_SUB * SHCI_MAX_K + 64);
    DevBuf<int64_t> idx;
    idx.alloc(SHCI_MAX_K);
    cudaStream_t st = c->st;
    CUDA_TRY(cudaMemsetAsync(w.G.p, 0, sizeof(double) * d.m_max * d.m_max, st));

    // initial subspace
    int m = 0;
    double *T = w.T.p;
    if (guess) {
        CUDA_TRY(cudaMemcpyAsync(T, guess, sizeof(double) * k * n,
                                 mem == SHCI_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
        m = d.orthonormalize_append(T, k, 0);
        if (m < k) throw ShciError{SHCI_ERR_INVALID, "guess vectors are linearly dependent"};
    } else {
        int nb = d.vec_blocks;
        DevBuf<double> pv;
        DevBuf<int64_t> pi;
        pv.alloc(nb);
        pi.alloc(nb);
        for (int l = 0; l < k; l++) {
            k_argmin_partial<<<nb, DV_THREADS, 0, st>>>(c->diag.p, n, idx.p, l, pv.p, pi.p);
            k_argmin_final<<<1, 32, 0, st>>>(pv.p, pi.p, nb, idx.p, l);
            KERNEL_CHECK();
            g_kernel_launches += 2;
        }
        k_unit_vectors<<<d.vec_blocks, DV_THREADS, 0, st>>>(idx.p, k, n, w.V.p);
        KERNEL_CHECK();
        g_kernel_launches += 1;
        m = k;
    }
    d.expand(0, m);

    std::vector<double> theta_old(k, INFINITY), status(2 * SHCI_MAX_K);
    double *d_rn = w.small.p + SHCI_MAX_SUB * SHCI_MAX_K + 8;
    int it = 0;
    bool conv = false;
    std::vector<double> theta(k), rnorm(k);
    for (it = 1; it <= max_iter; it++) {
        k_jacobi<<<1, 256, JACOBI_SMEM, st>>>(w.G.p, d.m_max, m, w.eval.p, w.evec.p);
        k_ritz<<<d.vec_blocks, DV_THREADS, 0, st>>>(w.V.p, w.AV.p, m, w.evec.p, d.m_max, w.eval.p, k, n, c->diag.p,
                                                    0, T, nullptr, nullptr, w.partial.p);
        k_sum_partials<<<1, 32, 0, st>>>(w.partial.p, d.vec_blocks, k, d_rn);
        KERNEL_CHECK();
        g_kernel_launches += 3;
        CUDA_TRY(cudaMemcpyAsync(status.data(), w.eval.p, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(status.data() + SHCI_MAX_K, d_rn, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        conv = true;
        std::vector<int> todo;
        for (int l = 0; l < k; l++) {
            theta[l] = status[l];
            rnorm[l] = std::sqrt(std::max(0.0, status[SHCI_MAX_K + l]));
            bool cl = std::fabs(theta[l] - theta_old[l]) < tol && rnorm[l] < res_tol;
            conv = conv && cl;
            if (rnorm[l] >= res_tol * 1e-3) todo.push_back(l);
        }
        theta_old = theta;
        if (conv || it == max_iter) break;
        // thick restart: keep the `keep` lowest Ritz vectors of the current subspace
        if (m + (int)todo.size() > d.m_max) {
            const int keep = std::min(m, d.keep);
            for (int j0 = 0; j0 < keep; j0 += SHCI_MAX_K) {
                const int cnt = std::min(SHCI_MAX_K, keep - j0);
                k_ritz<<<d.vec_blocks, DV_THREADS, 0, st>>>(w.V.p, w.AV.p, m, w.evec.p + (int64_t)j0 * d.m_max,
                                                            d.m_max, w.eval.p + j0, cnt, n, c->diag.p, 1, nullptr,
                                                            w.RV.p + (int64_t)j0 * n, w.RAV.p + (int64_t)j0 * n,
                                                            nullptr);
                KERNEL_CHECK();
                g_kernel_launches += 1;
            }
            CUDA_TRY(cudaMemcpyAsync(w.V.p, w.RV.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(w.AV.p, w.RAV.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, st));
            // recompute the projected block exactly (V^T H V over the kept Ritz vectors)
            CUDA_TRY(cudaMemsetAsync(w.G.p, 0, sizeof(double) * d.m_max * d.m_max, st));
            d.dots(w.V.p, keep, w.AV.p, keep, w.G.p, d.m_max, 0, 0, true);
            m = keep;
            // the residual corrections in T[0..k) are still valid: they depend only on the Ritz pairs
        }
        // corrections for the roots that are not yet converged
        int kb = 0;
        for (int l : todo) {
            if (l != kb)
                CUDA_TRY(cudaMemcpyAsync(T + (int64_t)kb * n, T + (int64_t)l * n, sizeof(double) * n,
                                         cudaMemcpyDeviceToDevice, st));
            kb++;
        }
        kb = std::min(kb, d.m_max - m);              // never grow past the subspace buffers
        if (kb <= 0) break;
        int added = d.orthonormalize_append(T, kb, m);
        if (added == 0) break;
        d.expand(m, added);
        m += added;
    }
    if (iters_out) *iters_out = it > max_iter ? max_iter : it;
    c->stats.davidson_iters = it > max_iter ? max_iter : it;
    for (int l = 0; l < k; l++) energies[l] = theta[l];
    if (vecs) {
        double *Xr = w.T.p + (int64_t)SHCI_MAX_K * n;
        k_jacobi<<<1, 256, JACOBI_SMEM, st>>>(w.G.p, d.m_max, m, w.eval.p, w.evec.p);
        k_ritz<<<d.vec_blocks, DV_THREADS, 0, st>>>(w.V.p, w.AV.p, m, w.evec.p, d.m_max, w.eval.p, k, n, c->diag.p,
                                                    1, nullptr, Xr, w.X.p, nullptr);
        KERNEL_CHECK();
        g_kernel_launches += 2;
        CUDA_TRY(cudaMemcpyAsync(vecs, Xr, sizeof(double) * k * n,
                                 mem == SHCI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return conv ? SHCI_OK : SHCI_ERR_NOT_CONVERGED;
}

}  // namespace shci
