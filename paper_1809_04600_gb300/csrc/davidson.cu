// Diagonally preconditioned Davidson for the lowest roots of H on V
// (Sec. II.A; the cached diagonal of Sec. V.B is the preconditioner).
//
// Everything runs on the device in FP64: the block sigma product, the
// projected matrix V^T H V, its eigen-decomposition (warm-started threshold
// Jacobi in one CTA), Ritz vectors, residuals, the preconditioner and the
// block orthonormalisation (classical Gram-Schmidt against the basis, a second
// pass only when the first removed most of a vector, Cholesky-QR within the
// block).  Reductions finish in the last block of each launch (no separate
// reduction kernels).  The host only sequences launches and reads a few
// scalars twice per iteration (Ritz values and residual norms; the number of
// accepted new vectors).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>

#include "context.cuh"
#include "jacobi.cuh"

namespace shci {

constexpr int DV_THREADS = 256;
constexpr int N_CTR = 128;                 // reduction counters: Gram row groups, last group, Ritz
constexpr int RITZ_CTR = N_CTR - 1;

// ---------------------------------------------------------------- block Gram products

// rows of A handled per block for NB columns of B (NA * NB <= 16 accumulators)
template <int NB>
struct GramShape {
    static constexpr int NA = NB >= 16 ? 1 : 16 / NB;
};

// What the last block does with a finished Gram product R = A^T B (A: the
// rows V[0..mv) then T[0..mt), B: NB vectors).
enum { EP_STORE = 0, EP_ORTHO = 1, EP_CHOL = 2 };

struct GramOut {
    int mode;
    double *R;              // [mv + mt][NB]: the product, always written
    double *dst;            // EP_STORE: dst[(a0 + a) * ld + b0 + b] (and mirrored when sym)
    int ld, a0, b0, sym;
    // EP_ORTHO (A = [V; T], B = T, mt = NB) and EP_CHOL (A = T, B = T)
    int pass;               // EP_ORTHO: 1 (decides on a second pass) or 2
    double *pre;            // [NB] squared norms before projection (pass 1 writes them)
    double *M;              // [NB][NB] coefficients of the new block
    double *CM;             // [mv][NB] = C M (EP_ORTHO)
    int *count;             // accepted vectors
    int *skip2;             // EP_ORTHO pass 1: 1 when the second pass is not needed
};

// Parallel reduction over slices, in a fixed order: out[e] for this group's
// outputs, one warp per output.
__device__ __forceinline__ double slice_sum(const double *partial, int64_t base, int stride, int nslices, int lane) {
    double s = 0.0;
    for (int x = lane; x < nslices; x += 32) s += __ldcg(&partial[base + (int64_t)x * stride]);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// R = A^T B with A = [V[0..mv); T[0..mt)] (rows of n) and B = NB vectors.
// blockIdx.x = slice of the vectors, blockIdx.y = group of NA rows of A.  Each
// block writes its partial sums; the last block of a group (atomic counter
// ctr[y]) sums the group's partials in slice order; for EP_ORTHO / EP_CHOL the
// last group (ctr[gridDim.y]) then computes the small-matrix coefficients.
// Counters are reset by the blocks that finish with them.
template <int NB>
__global__ void __launch_bounds__(DV_THREADS) k_gram_f(const double *__restrict__ V, int mv,
                                                      const double *__restrict__ T, int mt,
                                                      const double *__restrict__ B, int64_t n,
                                                      double *__restrict__ partial, unsigned *__restrict__ ctr,
                                                      GramOut o, const int *__restrict__ skip) {
    if (skip && *skip) return;              // device-side decision: this product is not needed
    constexpr int NA = GramShape<NB>::NA;
    constexpr int NE = NA * NB;
    const int na = mv + mt;
    const int a0 = blockIdx.y * NA;
    const int cnt = min(NA, na - a0);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const double *rowp[NA];
#pragma unroll
    for (int a = 0; a < NA; a++) {
        const int r = min(a0 + a, na - 1);
        rowp[a] = r < mv ? V + (int64_t)r * n : T + (int64_t)(r - mv) * n;
    }
    double acc[NA][NB];
#pragma unroll
    for (int a = 0; a < NA; a++)
#pragma unroll
        for (int b = 0; b < NB; b++) acc[a][b] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * DV_THREADS;
    for (int64_t i = blockIdx.x * (int64_t)DV_THREADS + tid; i < n; i += stride) {
        double bv[NB];
#pragma unroll
        for (int b = 0; b < NB; b++) bv[b] = B[b * n + i];
#pragma unroll
        for (int a = 0; a < NA; a++) {
            if (a < cnt) {
                const double av = rowp[a][i];
#pragma unroll
                for (int b = 0; b < NB; b++) acc[a][b] = fma(av, bv[b], acc[a][b]);
            }
        }
    }
    __shared__ double red[NE][DV_THREADS / 32];
#pragma unroll
    for (int a = 0; a < NA; a++) {
#pragma unroll
        for (int b = 0; b < NB; b++) {
            double v = acc[a][b];
#pragma unroll
            for (int o2 = 16; o2 >= 1; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
            if (lane == 0) red[a * NB + b][w] = v;
        }
    }
    __syncthreads();
    const int64_t gbase = (int64_t)blockIdx.y * gridDim.x * NE;
    if (tid < cnt * NB) {
        double s = 0.0;
#pragma unroll
        for (int x = 0; x < DV_THREADS / 32; x++) s += red[tid][x];
        partial[gbase + (int64_t)blockIdx.x * NE + tid] = s;
    }
    // last block of this group: the group's outputs
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&ctr[blockIdx.y], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int e = w; e < cnt * NB; e += DV_THREADS / 32) {
        const double v = slice_sum(partial, gbase + e, NE, gridDim.x, lane);
        if (lane == 0) {
            const int a = a0 + e / NB, b = e % NB;
            o.R[a * NB + b] = v;
            if (o.mode == EP_STORE) {
                const int r = o.a0 + a, c = o.b0 + b;
                o.dst[r * o.ld + c] = v;
                // the mirror, unless it is a product of its own (then both orders
                // are kept as computed: one writer per entry, deterministic)
                const bool own = c >= o.a0 && c < o.a0 + na && r >= o.b0 && r < o.b0 + NB;
                if (o.sym && !own) o.dst[c * o.ld + r] = v;
            }
        }
    }
    if (tid == 0) ctr[blockIdx.y] = 0u;
    if (o.mode == EP_STORE) return;
    // last group: the small-matrix step
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&ctr[gridDim.y], 1u) == gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid == 0) ctr[gridDim.y] = 0u;
    __shared__ double Ss[NB * NB], Ms[NB * NB], pres[NB];
    __shared__ int cnt_s;
    if (o.mode == EP_CHOL) {
        if (tid == 0) {
            for (int e = 0; e < NB * NB; e++) Ss[e] = __ldcg(&o.R[e]);
            *o.count = cholqr_coef(Ss, NB, nullptr, 1e-12, o.M);
        }
        return;
    }
    // EP_ORTHO: C = R[0..mv), S = R[mv..mv + NB); projected Gram S' = S - C^T C
    // (V orthonormal), then Cholesky-QR coefficients M of (T - V C) and C M
    for (int e = tid; e < NB * NB; e += DV_THREADS) {
        const int j = e / NB, l = e % NB;
        double v = __ldcg(&o.R[(mv + j) * NB + l]);
        for (int a = 0; a < mv; a++) v -= __ldcg(&o.R[a * NB + j]) * __ldcg(&o.R[a * NB + l]);
        Ss[e] = v;
    }
    if (o.pass == 1 && tid < NB) {
        pres[tid] = __ldcg(&o.R[(mv + tid) * NB + tid]);
        o.pre[tid] = pres[tid];
    } else if (tid < NB) {
        pres[tid] = __ldcg(&o.pre[tid]);
    }
    __syncthreads();
    if (tid == 0) {
        // "twice is enough": a second projection is needed only when the first
        // removed more than half of some vector's norm (squared norm below a
        // quarter); S' is then too inexact to orthonormalise from
        int need2 = 0;
        if (o.pass == 1)
            for (int l = 0; l < NB; l++) need2 |= Ss[l * NB + l] < 0.25 * pres[l];
        if (need2) {
            for (int e = 0; e < NB * NB; e++) Ms[e] = (e / NB == e % NB) ? 1.0 : 0.0;
            cnt_s = NB;
        } else {
            cnt_s = cholqr_coef(Ss, NB, pres, 1e-20, Ms);
        }
        if (o.pass == 1) *o.skip2 = need2 ? 0 : 1;
        *o.count = cnt_s;
    }
    __syncthreads();
    for (int e = tid; e < NB * NB; e += DV_THREADS) o.M[e] = Ms[e];
    for (int e = tid; e < mv * NB; e += DV_THREADS) {
        const int a = e / NB, l = e % NB;
        double v = 0.0;
        for (int j = 0; j < NB; j++) v = fma(__ldcg(&o.R[a * NB + j]), Ms[j * NB + l], v);
        o.CM[e] = v;
    }
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

// In place: T[l] <- sum_j M[j][l] T[j] - sum_a CM[a][l] V[a] for l < *count,
// zero for l >= *count (the projection T - V C followed by the block's
// coefficients M, with CM = C M).
template <int KB>
__global__ void __launch_bounds__(DV_THREADS) k_combine(const double *__restrict__ V, int m,
                                                       const double *__restrict__ CM, const double *__restrict__ M,
                                                       const int *__restrict__ count, int64_t n,
                                                       double *__restrict__ T, const int *__restrict__ skip) {
    if (skip && *skip) return;
    __shared__ double cs[SHCI_MAX_SUB * KB];
    __shared__ double ms[KB * KB];
    for (int e = threadIdx.x; e < m * KB; e += blockDim.x) cs[e] = CM[e];
    for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) ms[e] = M[e];
    __syncthreads();
    const int na = *count;
    for (int64_t i = blockIdx.x * (int64_t)DV_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DV_THREADS) {
        double t[KB], o[KB];
#pragma unroll
        for (int l = 0; l < KB; l++) t[l] = T[l * n + i];
#pragma unroll
        for (int l = 0; l < KB; l++) {
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < KB; j++) v = fma(ms[j * KB + l], t[j], v);
            o[l] = v;
        }
        int a = 0;
        for (; a + 4 <= m; a += 4) {
            const double v0 = V[(int64_t)a * n + i], v1 = V[(int64_t)(a + 1) * n + i];
            const double v2 = V[(int64_t)(a + 2) * n + i], v3 = V[(int64_t)(a + 3) * n + i];
#pragma unroll
            for (int l = 0; l < KB; l++) {
                o[l] = fma(-cs[a * KB + l], v0, o[l]);
                o[l] = fma(-cs[(a + 1) * KB + l], v1, o[l]);
                o[l] = fma(-cs[(a + 2) * KB + l], v2, o[l]);
                o[l] = fma(-cs[(a + 3) * KB + l], v3, o[l]);
            }
        }
        for (; a < m; a++) {
            const double v = V[(int64_t)a * n + i];
#pragma unroll
            for (int l = 0; l < KB; l++) o[l] = fma(-cs[a * KB + l], v, o[l]);
        }
#pragma unroll
        for (int l = 0; l < KB; l++) T[l * n + i] = l < na ? o[l] : 0.0;
    }
}

// out[l'] = sum_j M[j * KB + l'] T[j] for l' < *count (the accepted vectors)
template <int KB>
__global__ void __launch_bounds__(DV_THREADS) k_apply_coef(const double *__restrict__ T,
                                                          const double *__restrict__ M,
                                                          const int *__restrict__ count, int64_t n,
                                                          double *__restrict__ out) {
    __shared__ double ms[KB * KB];
    for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) ms[e] = M[e];
    __syncthreads();
    const int na = *count;
    for (int64_t i = blockIdx.x * (int64_t)DV_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DV_THREADS) {
        double t[KB];
#pragma unroll
        for (int j = 0; j < KB; j++) t[j] = T[j * n + i];
#pragma unroll
        for (int l = 0; l < KB; l++) {
            if (l < na) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < KB; j++) s = fma(ms[j * KB + l], t[j], s);
                out[l * n + i] = s;
            }
        }
    }
}

// Ritz vectors and residuals for K roots of the subspace of size m:
//   x_l = sum_a Y[a][l] V[a],  h_l = sum_a Y[a][l] AV[a],  r_l = h_l - theta_l x_l
// MODE 0: T[l] = r_l / (theta_l - H_ii) (clamped), partial |r_l|^2 per block
// MODE 1: Xo[l] = x_l, Ho[l] = h_l (restart / output)
template <int K, int MODE>
__global__ void __launch_bounds__(DV_THREADS) k_ritz(const double *__restrict__ V, const double *__restrict__ AV,
                                                     int m, const double *__restrict__ evec, int ld,
                                                     const double *__restrict__ eval, int64_t n,
                                                     const double *__restrict__ diag, double *__restrict__ T,
                                                     double *__restrict__ Xo, double *__restrict__ Ho,
                                                     double *__restrict__ partial, unsigned *__restrict__ ctr,
                                                     double *__restrict__ rn_out) {
    __shared__ double ys[SHCI_MAX_SUB * K];
    __shared__ double th[K];
    for (int e = threadIdx.x; e < m * K; e += blockDim.x) ys[e] = evec[(e % K) * ld + (e / K)];   // ys[a*K+l]
    if (threadIdx.x < K) th[threadIdx.x] = eval[threadIdx.x];
    __syncthreads();
    double rn[K];
#pragma unroll
    for (int l = 0; l < K; l++) rn[l] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)DV_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DV_THREADS) {
        double x[K], h[K];
#pragma unroll
        for (int l = 0; l < K; l++) { x[l] = 0.0; h[l] = 0.0; }
        int a = 0;
        for (; a + 2 <= m; a += 2) {
            const double v0 = V[(int64_t)a * n + i], w0 = AV[(int64_t)a * n + i];
            const double v1 = V[(int64_t)(a + 1) * n + i], w1 = AV[(int64_t)(a + 1) * n + i];
#pragma unroll
            for (int l = 0; l < K; l++) {
                x[l] = fma(ys[a * K + l], v0, x[l]);
                h[l] = fma(ys[a * K + l], w0, h[l]);
                x[l] = fma(ys[(a + 1) * K + l], v1, x[l]);
                h[l] = fma(ys[(a + 1) * K + l], w1, h[l]);
            }
        }
        for (; a < m; a++) {
            const double v = V[(int64_t)a * n + i], w = AV[(int64_t)a * n + i];
#pragma unroll
            for (int l = 0; l < K; l++) {
                x[l] = fma(ys[a * K + l], v, x[l]);
                h[l] = fma(ys[a * K + l], w, h[l]);
            }
        }
        if (MODE == 0) {
            const double d = diag[i];
#pragma unroll
            for (int l = 0; l < K; l++) {
                const double r = fma(-th[l], x[l], h[l]);
                rn[l] = fma(r, r, rn[l]);
                double den = th[l] - d;
                if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
                T[l * n + i] = r / den;
            }
        } else {
#pragma unroll
            for (int l = 0; l < K; l++) {
                Xo[l * n + i] = x[l];
                Ho[l * n + i] = h[l];
            }
        }
    }
    if (MODE == 0) {
        __shared__ double red[K][DV_THREADS / 32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int l = 0; l < K; l++) {
            double v = rn[l];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[l][w] = v;
        }
        __syncthreads();
        if (threadIdx.x < K) {
            double s = 0.0;
#pragma unroll
            for (int x = 0; x < DV_THREADS / 32; x++) s += red[threadIdx.x][x];
            partial[(int64_t)blockIdx.x * K + threadIdx.x] = s;
        }
        // the last block sums the partial squared norms in block order
        __shared__ int last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(ctr, 1u) == gridDim.x - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
        if (w < K) {
            double s = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(&partial[(int64_t)b * K + w]);
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) rn_out[w] = s;
        }
        if (threadIdx.x == 0) *ctr = 0u;
    }
}

// ---------------------------------------------------------------- subspace eigensolver

// one CTA: the eigen-decomposition of one projected matrix (see jacobi.cuh)
__global__ void k_jacobi(const double *__restrict__ G, int ld, int m, int m_prev, double *__restrict__ eval,
                         double *__restrict__ evec) {
    extern __shared__ double jsm[];
    jacobi_solve(G, ld, m, m_prev, eval, evec, jsm);
}

// ---------------------------------------------------------------- start vectors

// Order-preserving 64-bit key of a double (ascending keys = ascending values)
// and the element's index, for a stable sort of the diagonal.
__global__ void k_diag_keys(const double *__restrict__ d, int64_t n, uint64_t *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = (uint64_t)__double_as_longlong(d[i]);
        keys[i] = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
        vals[i] = (uint32_t)i;
    }
}

// G[a * ld + b] = <D_sel[a]| H |D_sel[b]> for a, b < m (both triangles).
template <int W>
__global__ void k_guess_block(const uint64_t *__restrict__ dets, const double *__restrict__ diag,
                              const uint32_t *__restrict__ sel, int m, int ld, DevInts I, double *__restrict__ G) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
        const int a = e / m, b = e % m;
        if (a > b) continue;
        const int64_t i = sel[a], j = sel[b];
        double v;
        if (a == b) {
            v = diag[i];
        } else {
            const Str<W> ai = load_str<W>(dets, 2 * i), bi = load_str<W>(dets, 2 * i + 1);
            const Str<W> aj = load_str<W>(dets, 2 * j), bj = load_str<W>(dets, 2 * j + 1);
            const int d = xor_popc<W>(ai, aj) + xor_popc<W>(bi, bj);
            v = (d == 2 || d == 4) ? hij_offdiag<W>(I, ai, bi, aj, bj) : 0.0;
        }
        G[a * ld + b] = v;
        G[b * ld + a] = v;
    }
}

// T[l][sel[a]] = evec[l * ld + a] for l < k, a < m (T zeroed before)
__global__ void k_guess_scatter(const double *__restrict__ evec, int ld, const uint32_t *__restrict__ sel, int m,
                                int k, int64_t n, double *__restrict__ T) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * k; e += gridDim.x * blockDim.x) {
        const int l = e / m, a = e % m;
        T[(int64_t)l * n + sel[a]] = evec[l * ld + a];
    }
}

// The default start of the iteration: the k lowest eigenvectors of H
// restricted to the m = min(64, n) determinants of lowest H_ii (ties by
// index), written to T[0..k) as full vectors.
static void subspace_guess(shci_ctx *c, int k, double *T) {
    const int64_t n = c->n_det;
    const int m = (int)std::min<int64_t>(SHCI_MAX_SUB, n);
    cudaStream_t st = c->st;
    DavidsonWork &w = c->dw;
    c->sort_keys.alloc((size_t)std::max<int64_t>(n, 1) * c->W);
    c->sort_vals.alloc((size_t)std::max<int64_t>(n, 1));
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n, 256), (int64_t)c->n_sm * 16);
    k_diag_keys<<<g, 256, 0, st>>>(c->diag.p, n, c->sort_keys.p, c->sort_vals.p);
    KERNEL_CHECK();
    g_kernel_launches += 1;
    radix_sort<1>(c->sort_keys.p, c->sort_vals.p, n, c->sw, st);
    w.guess_G.alloc((size_t)SHCI_MAX_SUB * SHCI_MAX_SUB);
    w.guess_vec.alloc((size_t)SHCI_MAX_SUB * SHCI_MAX_SUB);
    w.guess_val.alloc((size_t)SHCI_MAX_SUB);
    const DevInts I = dev_ints(c);
    if (c->W == 1)
        k_guess_block<1><<<16, 256, 0, st>>>(c->dets.p, c->diag.p, c->sort_vals.p, m, SHCI_MAX_SUB, I, w.guess_G.p);
    else
        k_guess_block<2><<<16, 256, 0, st>>>(c->dets.p, c->diag.p, c->sort_vals.p, m, SHCI_MAX_SUB, I, w.guess_G.p);
    KERNEL_CHECK();
    k_jacobi<<<1, 256, JACOBI_SMEM, st>>>(w.guess_G.p, SHCI_MAX_SUB, m, 0, w.guess_val.p, w.guess_vec.p);
    KERNEL_CHECK();
    CUDA_TRY(cudaMemsetAsync(T, 0, sizeof(double) * k * n, st));
    k_guess_scatter<<<4, 256, 0, st>>>(w.guess_vec.p, SHCI_MAX_SUB, c->sort_vals.p, m, k, n, T);
    KERNEL_CHECK();
    g_kernel_launches += 3;
}

// ---------------------------------------------------------------- host driver

#define DISPATCH_K(kval, F)                         \
    switch (kval) {                                 \
        case 1: F(1); break;                        \
        case 2: F(2); break;                        \
        case 3: F(3); break;                        \
        case 4: F(4); break;                        \
        case 5: F(5); break;                        \
        case 6: F(6); break;                        \
        case 7: F(7); break;                        \
        case 8: F(8); break;                        \
        default: throw ShciError{SHCI_ERR_INVALID, "block size out of range"}; \
    }

// Per-part device timeline of one Davidson run: an event after each part;
// the time between consecutive events goes to the part that ended.
struct PartTimer {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> ev;
    std::vector<int> part;
    void mark(int p) {
        if (!on) return;
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        CUDA_TRY(cudaEventRecord(e, st));
        ev.push_back(e);
        part.push_back(p);
    }
    void finish(double *out, int n_parts) {
        if (!on || ev.empty()) return;
        for (int p = 0; p < n_parts; p++) out[p] = 0.0;
        CUDA_TRY(cudaEventSynchronize(ev.back()));
        for (size_t x = 1; x < ev.size(); x++) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, ev[x - 1], ev[x]));
            if (part[x] >= 0 && part[x] < n_parts) out[part[x]] += ms;
        }
        for (auto e : ev) cudaEventDestroy(e);
        ev.clear();
        part.clear();
    }
    ~PartTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

enum { DP_START = 0, DP_EIG = 1, DP_RITZ = 2, DP_RESTART = 3, DP_ORTHO = 4, DP_SIGMA = 5, DP_GRAM = 6 };

struct Dav {
    shci_ctx *c;
    PartTimer *pt = nullptr;
    int64_t n;
    int k, m_max, keep;
    int vec_blocks, n_slots;
    cudaStream_t st;
    double *R, *CM, *M, *pre;   // device small buffers: Gram result, coefficients, norms
    unsigned *ctr;              // reduction counters (zero between launches)
    int *d_count;
    int *d_skip;                // device flag: 1 = second Gram-Schmidt pass not needed

    double *Vr(int a) { return c->dw.V.p + (int64_t)a * n; }
    double *AVr(int a) { return c->dw.AV.p + (int64_t)a * n; }

    template <int NB>
    void gram_nb(const double *V, int mv, const double *T, int mt, const double *B, const GramOut &o,
                 const int *skip) {
        constexpr int NA = GramShape<NB>::NA;
        const int na = mv + mt;
        const int groups = (na + NA - 1) / NA;
        const int slices = std::max(1, std::min<int>((int)ceil_div(n, DV_THREADS * 4), n_slots / groups));
        dim3 grid(slices, groups);
        k_gram_f<NB><<<grid, DV_THREADS, 0, st>>>(V, mv, T, mt, B, n, c->dw.partial.p, ctr, o, skip);
        KERNEL_CHECK();
        g_kernel_launches += 1;
    }

    void gram_dispatch(int nb, const double *V, int mv, const double *T, int mt, const double *B, const GramOut &o,
                       const int *skip) {
#define F(NB) gram_nb<NB>(V, mv, T, mt, B, o, skip)
        DISPATCH_K(nb, F)
#undef F
    }

    // out[a0 + a][b0 + b] (leading dimension ld) = A[a] . B[b], a < na, b < nb; mirrored if sym.
    void gram(const double *A, int na, const double *B, int nb, double *out, int ld, int a0, int b0, bool sym) {
        if (na <= 0 || nb <= 0) return;
        for (int b = 0; b < nb; b += SHCI_MAX_K) {
            const int cnt = std::min(SHCI_MAX_K, nb - b);
            GramOut o{};
            o.mode = EP_STORE;
            o.R = R;
            o.dst = out;
            o.ld = ld;
            o.a0 = a0;
            o.b0 = b0 + b;
            o.sym = sym ? 1 : 0;
            gram_dispatch(cnt, A, na, nullptr, 0, B + (int64_t)b * n, o, nullptr);
        }
    }

    void combine(double *T, int kb, int m, const int *skip) {
#define F(KB) k_combine<KB><<<vec_blocks, DV_THREADS, 0, st>>>(c->dw.V.p, m, CM, M, d_count, n, T, skip)
        DISPATCH_K(kb, F)
#undef F
        KERNEL_CHECK();
        g_kernel_launches += 1;
    }

    void apply_coef(const double *T, int kb, double *out) {
#define F(KB) k_apply_coef<KB><<<vec_blocks, DV_THREADS, 0, st>>>(T, M, d_count, n, out)
        DISPATCH_K(kb, F)
#undef F
        KERNEL_CHECK();
        g_kernel_launches += 1;
    }

    // Orthonormalise the kb vectors T[0..kb) against V[0..m) and among
    // themselves, writing the accepted ones to V[m ..); returns how many were
    // accepted.  Pass 1 forms C = V^T T and S = T^T T in one sweep, and the last
    // block derives the coefficients of (T - V C) M from S - C^T C; when the
    // projection removed more than half of some vector's norm the device asks
    // for a second projection pass ("twice is enough"), otherwise that pass's
    // kernels return at once.  A last Cholesky-QR pass within the block follows.
    int orthonormalize_append(double *T, int kb, int m) {
        GramOut o{};
        o.mode = EP_ORTHO;
        o.R = R;
        o.pre = pre;
        o.M = M;
        o.CM = CM;
        o.count = d_count;
        o.skip2 = d_skip;
        o.pass = 1;
        gram_dispatch(kb, c->dw.V.p, m, T, kb, T, o, nullptr);
        combine(T, kb, m, nullptr);
        o.pass = 2;
        gram_dispatch(kb, c->dw.V.p, m, T, kb, T, o, d_skip);
        combine(T, kb, m, d_skip);
        GramOut q{};
        q.mode = EP_CHOL;
        q.R = R;
        q.M = M;
        q.count = d_count;
        gram_dispatch(kb, nullptr, 0, T, kb, T, q, nullptr);
        apply_coef(T, kb, Vr(m));
        int added = 0;
        CUDA_TRY(cudaMemcpyAsync(&added, d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return added;
    }

    // AV[m0 .. m0 + kb) = H V[m0 .. m0 + kb); G's new columns (and rows)
    void expand(int m0, int kb) {
        k_pack<<<vec_blocks, DV_THREADS, 0, st>>>(Vr(m0), kb, n, c->dw.X.p);
        KERNEL_CHECK();
        sigma(c, kb, c->dw.X.p, c->dw.Y.p, true);
        k_unpack<<<vec_blocks, DV_THREADS, 0, st>>>(c->dw.Y.p, kb, n, AVr(m0));
        KERNEL_CHECK();
        g_kernel_launches += 2;
        if (pt) pt->mark(m0 == 0 ? DP_START : DP_SIGMA);
        gram(c->dw.V.p, m0 + kb, AVr(m0), kb, c->dw.G.p, m_max, 0, m0, true);
        if (pt) pt->mark(m0 == 0 ? DP_START : DP_GRAM);
    }

    void ritz_residuals(int m, double *T, double *d_rn) {
#define F(K)                                                                                                 \
    k_ritz<K, 0><<<vec_blocks, DV_THREADS, 0, st>>>(c->dw.V.p, c->dw.AV.p, m, c->dw.evec.p, m_max,          \
                                                    c->dw.eval.p, n, c->diag.p, T, nullptr, nullptr,         \
                                                    c->dw.partial.p, ctr + RITZ_CTR, d_rn)
        DISPATCH_K(k, F)
#undef F
        KERNEL_CHECK();
        g_kernel_launches += 1;
    }

    // x_l = V y_l and h_l = AV y_l for l in [j0, j0 + cnt)
    void ritz_vectors(int m, int j0, int cnt, double *Xo, double *Ho) {
#define F(K)                                                                                                 \
    k_ritz<K, 1><<<vec_blocks, DV_THREADS, 0, st>>>(c->dw.V.p, c->dw.AV.p, m, c->dw.evec.p + (int64_t)j0 * m_max, \
                                                    m_max, c->dw.eval.p + j0, n, c->diag.p, nullptr, Xo, Ho, \
                                                    nullptr, nullptr, nullptr)
        DISPATCH_K(cnt, F)
#undef F
        KERNEL_CHECK();
        g_kernel_launches += 1;
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
    const auto t_entry = std::chrono::steady_clock::now();
    static bool jacobi_attr = false;
    if (!jacobi_attr) {
        CUDA_TRY(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JACOBI_SMEM));
        jacobi_attr = true;
    }
    Dav d;
    PartTimer timer;
    timer.on = c->timing_dav;
    timer.st = c->st;
    timer.mark(-1);
    d.pt = &timer;
    d.c = c;
    d.n = c->n_det;
    d.k = k;
    d.st = c->st;
    // subspace: larger when a product is expensive (on the fly), where fewer
    // iterations pay; smaller with a stored H, where the per-iteration vector
    // work and the eigensolver (both growing with the subspace) are a larger share
    const int per_root = c->mode == SHCI_ON_THE_FLY ? 16 : 8;
    d.m_max = (int)std::min<int64_t>(std::min(SHCI_MAX_SUB, 16 + per_root * k), c->n_det);
    if (d.m_max < k) d.m_max = k;
    d.keep = std::max(k, std::min(d.m_max - k, std::max(2 * k, d.m_max / 3)));
    d.vec_blocks = std::max(1, std::min<int>((int)ceil_div(d.n, DV_THREADS), c->n_sm * 8));
    d.n_slots = c->n_sm * 8;
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
    w.partial.alloc((size_t)std::max(d.n_slots, d.vec_blocks) * SHCI_MAX_SUB * SHCI_MAX_K);
    w.small.alloc((size_t)4 * SHCI_MAX_SUB * SHCI_MAX_K + 64);
    d.R = w.small.p;                                                    // [m_max + 8][kb]
    d.CM = w.small.p + (SHCI_MAX_SUB + SHCI_MAX_K) * SHCI_MAX_K;        // [m_max][kb]
    d.M = d.CM + SHCI_MAX_SUB * SHCI_MAX_K;                             // [kb][kb]
    d.pre = d.M + SHCI_MAX_K * SHCI_MAX_K;                              // [kb]
    double *d_rn = d.pre + SHCI_MAX_K;                                  // [k]
    w.ctr.alloc(N_CTR);
    CUDA_TRY(cudaMemsetAsync(w.ctr.p, 0, sizeof(unsigned) * N_CTR, c->st));
    d.ctr = w.ctr.p;
    c->counter.alloc(4);
    d.d_count = c->counter.p + 3;
    d.d_skip = c->counter.p + 2;
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
        subspace_guess(c, k, T);
        m = d.orthonormalize_append(T, k, 0);
        if (m < k) throw ShciError{SHCI_ERR_INVALID, "start vectors are linearly dependent"};
    }
    d.expand(0, m);

    std::vector<double> theta_old(k, INFINITY), status(2 * SHCI_MAX_K);
    c->hist_theta.clear();
    c->hist_rn.clear();
    c->hist_t.clear();
    c->hist_k = k;
    int it = 0;
    int m_eig = 0;          // size of the leading block whose eigenvectors are in evec
    bool conv = false;
    std::vector<double> theta(k), rnorm(k);
    for (it = 1; it <= max_iter; it++) {
        k_jacobi<<<1, 256, JACOBI_SMEM, st>>>(w.G.p, d.m_max, m, m_eig, w.eval.p, w.evec.p);
        KERNEL_CHECK();
        g_kernel_launches += 1;
        timer.mark(DP_EIG);
        m_eig = m;
        d.ritz_residuals(m, T, d_rn);
        CUDA_TRY(cudaMemcpyAsync(status.data(), w.eval.p, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(status.data() + SHCI_MAX_K, d_rn, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        timer.mark(DP_RITZ);
        c->hist_t.push_back(std::chrono::duration<double>(std::chrono::steady_clock::now() - t_entry).count());
        conv = true;
        std::vector<int> todo;
        for (int l = 0; l < k; l++) {
            theta[l] = status[l];
            rnorm[l] = std::sqrt(std::max(0.0, status[SHCI_MAX_K + l]));
            c->hist_theta.push_back(theta[l]);
            c->hist_rn.push_back(rnorm[l]);
            // converged: settled and small residual, or a residual so small that the
            // Ritz value is exact to rounding (e.g. a start that is already an eigenvector)
            const bool cl = (std::fabs(theta[l] - theta_old[l]) < tol && rnorm[l] < res_tol) ||
                            rnorm[l] < res_tol * 1e-3;
            conv = conv && cl;
            // a converged root is locked: no new direction for it
            if (!cl) todo.push_back(l);
        }
        theta_old = theta;
        if (conv || it == max_iter) break;
        // thick restart: keep the `keep` lowest Ritz vectors of the current subspace
        if (m + (int)todo.size() > d.m_max) {
            const int keep = std::min(m, d.keep);
            for (int j0 = 0; j0 < keep; j0 += SHCI_MAX_K) {
                const int cnt = std::min(SHCI_MAX_K, keep - j0);
                d.ritz_vectors(m, j0, cnt, w.RV.p + (int64_t)j0 * n, w.RAV.p + (int64_t)j0 * n);
            }
            CUDA_TRY(cudaMemcpyAsync(w.V.p, w.RV.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(w.AV.p, w.RAV.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, st));
            // recompute the projected block exactly (V^T H V over the kept Ritz vectors)
            CUDA_TRY(cudaMemsetAsync(w.G.p, 0, sizeof(double) * d.m_max * d.m_max, st));
            d.gram(w.V.p, keep, w.AV.p, keep, w.G.p, d.m_max, 0, 0, true);
            m = keep;
            m_eig = 0;
            // the residual corrections in T[0..k) are still valid: they depend only on the Ritz pairs
            timer.mark(DP_RESTART);
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
        timer.mark(DP_ORTHO);
        if (added == 0) break;
        d.expand(m, added);
        m += added;
    }
    if (iters_out) *iters_out = it > max_iter ? max_iter : it;
    c->stats.davidson_iters = it > max_iter ? max_iter : it;
    for (int l = 0; l < k; l++) energies[l] = theta[l];
    if (vecs) {
        // evec/eval still describe the current G (nothing changed since the last solve)
        double *Xr = w.T.p + (int64_t)SHCI_MAX_K * n;
        d.ritz_vectors(m, 0, k, Xr, w.X.p);
        CUDA_TRY(cudaMemcpyAsync(vecs, Xr, sizeof(double) * k * n,
                                 mem == SHCI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    timer.finish(c->stats.davidson_phase_ms, 8);
    return conv ? SHCI_OK : SHCI_ERR_NOT_CONVERGED;
}

}  // namespace shci
