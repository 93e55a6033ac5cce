// Batched Davidson: many independent systems (each with its own integrals and
// variational space) and up to four roots each, solved in ONE persistent,
// cooperative kernel launch that is captured in a CUDA graph.
//
// The systems form one block-diagonal problem.  Every phase of a Davidson
// iteration runs for all active systems at once and is separated from the
// next by a grid-wide barrier:
//   sigma      rows of stored Hamiltonians (CSR row chunks) and work items of
//              the on-the-fly enumeration (alpha-grouped, then beta-grouped);
//              an upper-triangle matrix sets Y = diag X in the first sigma
//              phase and adds its rows and their transposes in the second
//   vectors    slices of every system's vectors (Gram columns, Ritz vectors
//              and preconditioned residuals, projections, Cholesky-QR)
//   systems    one CTA per system (reductions of partial sums, the subspace
//              eigensolver, convergence, restart and block bookkeeping)
// Small systems no longer pay a launch and a host round trip per step, and
// the one-CTA eigensolvers of all systems run side by side.  Each system
// follows the algorithm of shci_davidson (thick restart, block Gram-Schmidt
// twice, Cholesky-QR twice, warm-started Jacobi).
//
// The barrier spins with a bound: if a block never arrives (a grid that is
// not co-resident) the waiters give up, set an error flag and return, and the
// host reports SHCI_ERR_TIMEOUT instead of hanging.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "enum_launch.cuh"
#include "jacobi.cuh"
#include "plan.h"

namespace shci {

constexpr int BK = 4;                      // roots per system in a batch (max)
constexpr int BT = 256;                    // threads per CTA
constexpr int VSLICE = 8192;               // vector elements per vector work item (default; tuned)
constexpr int GA = 8;                      // basis rows per register block in slice Gram products
constexpr int PSTRIDE = SHCI_MAX_SUB * BK + BK * BK + BK + 12;   // partial sums per vector item
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 27;             // default: x ~100 ns naps >= ~13 s
constexpr int OFF_S0 = SHCI_MAX_SUB * BK;                        // partial layout offsets
constexpr int OFF_RN = SHCI_MAX_SUB * BK + BK * BK;

// immutable description of one system
struct BSys {
    int64_t n;
    int mode, k, m_max, keep;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val, *diag;
    EnumArgs ea, eb;                       // on-the-fly enumeration: alpha items, beta items
                                           // (complete, read in place: no per-item copy)
    DevInts I;
    int64_t v_item_off, v_item_cnt;        // this system's vector items
    int64_t vslice;                        // and their length (the batch's)
    double *Vb[2], *AVb[2];                // current / rotation target (swapped by index)
    double *T, *T2, *X, *Y;
    double *G, *evec, *erot, *eval;
    double *jq;                            // the eigensolver's rotation accumulator (global scratch)
    double *coefC, *coefS0, *coefS, *coefM, *coefM2;
    double tol, res_tol;
};

// mutable per-system state, written by the system's CTA between barriers and
// read by everyone through L2 (ld.global.cg)
struct BState {
    int m, nb, m_eig, active, restart, m_old, it, ntodo, cnt1, cnt2, conv, cur;
    int todo[BK];
    double theta[BK], theta_old[BK], rn[BK];
};

constexpr int N_PHASES = 16;

struct BarrierState {
    unsigned count;
    unsigned gen;
    int err;
    int work;
    unsigned long long t_last;             // block 0: global time at the last barrier exit
    unsigned long long phase_ns[N_PHASES]; // block 0: time between barriers, per phase
};

struct BatchArgs {
    int S;
    const BSys *sys;
    BState *st;
    int max_iter;
    const int32_t *a1_sys, *a1_kind;       // sigma phase 1: kind 0 stored rows, 1 alpha items,
                                           // 2 Y = diag X rows of an upper-triangle matrix
    const int64_t *a1_local;
    int64_t n_a1;
    const int32_t *a2_sys, *a2_kind;       // sigma phase 2: kind 0 beta items, 1 upper-triangle rows
    const int64_t *a2_local;
    int64_t n_a2;
    int srows;                             // rows per stored-sigma item
    int lpr;                               // lanes per stored row: 32 or 8
    const int32_t *v_sys;                  // vector items
    const int64_t *v_start;
    int64_t n_v;
    double *partial;                       // [n_v][PSTRIDE]
    BarrierState *bar;
    long long spin_limit;                  // naps a waiting block takes before it gives up
};

// ---------------------------------------------------------------- barrier and helpers

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier; `phase` names the phase that ends here (block 0 adds
// the time since the previous barrier to that phase's total).  A block that
// has waited `limit` naps of ~100 ns gives up and raises the error flag.
__device__ bool grid_sync(BarrierState *b, int phase, long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = *(volatile int *)&b->err == 0;
        if (good) {
            volatile unsigned *vgen = &b->gen;
            const unsigned g = *vgen;
            __threadfence();
            const unsigned arrived = atomicAdd(&b->count, 1u) + 1u;
            if (arrived == gridDim.x) {
                atomicExch(&b->count, 0u);
                atomicExch(&b->work, 0);
                __threadfence();
                atomicAdd(&b->gen, 1u);
            } else {
                long long spins = 0;
                while (*vgen == g) {
                    if (*(volatile int *)&b->err) { good = 0; break; }
                    if (++spins > limit) {
                        atomicExch(&b->err, 1);
                        good = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
        }
        if (blockIdx.x == 0) {
            const unsigned long long now = global_ns();
            b->phase_ns[phase] += now - b->t_last;
            b->t_last = now;
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int next_item(BarrierState *b) {
    __shared__ int item;
    if (threadIdx.x == 0) item = atomicAdd(&b->work, 1);
    __syncthreads();
    const int v = item;
    __syncthreads();
    return v;
}

__device__ __forceinline__ int ldi(const int *p) { return __ldcg(p); }

// block reduction of NV per-thread values; part[e] = block sum of v[e] for e < cnt
template <int NV>
__device__ __forceinline__ void item_reduce(double *part, const double (&v)[NV], int cnt, double *red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < NV; e++) {
        double x = v[e];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w * NV + e] = x;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double s = 0.0;
#pragma unroll
        for (int x = 0; x < BT / 32; x++) s += red[x * NV + threadIdx.x];
        part[threadIdx.x] = s;
    }
    __syncthreads();
}

// part[a * BK + l] (a < na) = sum over [i0, i1) of A_a(i) * b_l(i); b(i) supplies BK values
template <class LoadB>
__device__ __forceinline__ void slice_gram(double *part, const double *A, int64_t n, int na, int64_t i0, int64_t i1,
                                           LoadB loadB, double *red) {
    for (int g0 = 0; g0 < na; g0 += GA) {
        double acc[GA * BK];
#pragma unroll
        for (int e = 0; e < GA * BK; e++) acc[e] = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
            double b[BK];
            loadB(i, b);
#pragma unroll
            for (int a = 0; a < GA; a++) {
                if (g0 + a < na) {
                    const double v = __ldcg(&A[(int64_t)(g0 + a) * n + i]);
#pragma unroll
                    for (int l = 0; l < BK; l++) acc[a * BK + l] = fma(v, b[l], acc[a * BK + l]);
                }
            }
        }
        item_reduce<GA * BK>(part + g0 * BK, acc, min(GA, na - g0) * BK, red);
    }
}

// sum of a system's vector-item partials at offset `off`
__device__ __forceinline__ double sum_items(const BatchArgs &B, const BSys &S, int off) {
    double v = 0.0;
    for (int64_t x = 0; x < S.v_item_cnt; x++) v += __ldcg(&B.partial[(S.v_item_off + x) * PSTRIDE + off]);
    return v;
}

// stored rows [r0, r0 + cnt): Y[i][q] = diag_i X[i][q] + sum_j H_ij X[j][q], q < NB.
// LPR lanes per row: 32 is a warp per determinant; fewer lanes work on
// 32 / LPR rows of a warp at once (short rows leave fewer lanes idle).  One
// instance per count of vectors in use, out of line (its registers apart from
// the persistent kernel's); SR nonzeros per lane per step with all loads
// issued before the FMAs, 8 in the variants with the registers for it.
template <int LPR, int NB, int MINB>
__device__ __noinline__ void sigma_rows_nb(const BSys &S, int64_t r0, int cnt) {
    constexpr int RPW = 32 / LPR;
    constexpr int SR = MINB <= 2 ? 8 : 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / LPR, sl = lane % LPR;
    const int64_t *__restrict__ rowptr = S.rowptr;      // the system's arrays in registers
    const int32_t *__restrict__ col = S.col;
    const double *__restrict__ val = S.val;
    const double *X = S.X;
    double *Y = S.Y;
    const int64_t r1 = min(r0 + cnt, S.n);
    auto load_x = [&](int64_t j, double (&o)[NB]) {
        if (NB == 1) {
            o[0] = __ldcg(&X[j * BK]);
        } else {
            const double2 a = __ldcg(reinterpret_cast<const double2 *>(X) + 2 * j);
            o[0] = a.x;
            o[NB > 1 ? 1 : 0] = a.y;
            if (NB > 2) {
                const double2 b = __ldcg(reinterpret_cast<const double2 *>(X) + 2 * j + 1);
                o[NB > 2 ? 2 : 0] = b.x;
                if (NB > 3) o[NB > 3 ? 3 : 0] = b.y;
            }
        }
    };
    for (int64_t i0 = r0 + (int64_t)warp * RPW; i0 < r1; i0 += (BT / 32) * RPW) {
        const int64_t i = i0 + sub;
        const bool ok = i < r1;
        double acc[NB];
#pragma unroll
        for (int q = 0; q < NB; q++) acc[q] = 0.0;
        const int64_t beg = ok ? rowptr[i] : 0, end = ok ? rowptr[i + 1] : 0;
        for (int64_t p0 = beg + sl; p0 < end; p0 += LPR * SR) {
            int32_t j[SR];
            double v[SR], xv[SR][NB];
#pragma unroll
            for (int u = 0; u < SR; u++) {
                const int64_t p = p0 + LPR * u;
                j[u] = p < end ? __ldg(&col[p]) : -1;
                v[u] = p < end ? __ldg(&val[p]) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < SR; u++) {
                if (j[u] >= 0) load_x(j[u], xv[u]);
                else
#pragma unroll
                    for (int q = 0; q < NB; q++) xv[u][q] = 0.0;
            }
#pragma unroll
            for (int u = 0; u < SR; u++)
#pragma unroll
                for (int q = 0; q < NB; q++) acc[q] = fma(v[u], xv[u][q], acc[q]);
        }
        // reduce over the row's LPR lanes (the whole warp takes part)
#pragma unroll
        for (int q = 0; q < NB; q++) {
#pragma unroll
            for (int o = LPR / 2; o >= 1; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        }
        if (ok && sl == 0) {
            const double d = S.diag[i];
#pragma unroll
            for (int q = 0; q < NB; q++) Y[i * BK + q] = fma(d, __ldcg(&X[i * BK + q]), acc[q]);
        }
    }
}

template <int LPR, int MINB>
__device__ __forceinline__ void sigma_rows(const BSys &S, int nb, int64_t r0, int cnt) {
    switch (nb) {
        case 1: sigma_rows_nb<LPR, 1, MINB>(S, r0, cnt); break;
        case 2: sigma_rows_nb<LPR, 2, MINB>(S, r0, cnt); break;
        case 3: sigma_rows_nb<LPR, 3, MINB>(S, r0, cnt); break;
        default: sigma_rows_nb<LPR, 4, MINB>(S, r0, cnt); break;
    }
}

// rows [r0, r0 + cnt) of an upper-triangle matrix, after Y = diag X
// (diag_rows, the phase before): each stored H_ij (j > i) adds H_ij X[j] to
// row i's sum and H_ij X[i] to Y[j] with an atomic add; the row sums are then
// added to Y[i] atomically (other rows scatter into it in the same phase).
// One instance per count of vectors in use, out of line: it gets its registers
// apart from the rest of the persistent kernel.  The scatter keeps a warp
// waiting on gathers and atomics, and the persistent grid has few warps per
// SM, so a variant with the registers for it (MINB <= 2) takes 8 nonzeros
// per lane per step.
template <int LPR, int NB, int MINB>
__device__ __noinline__ void sigma_rows_upper_nb(const BSys &S, int64_t r0, int cnt) {
    constexpr int RPW = 32 / LPR;
    constexpr int SR = MINB <= 2 ? 8 : 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / LPR, sl = lane % LPR;
    // the system's arrays in registers: the atomic adds below could alias the
    // descriptor in global memory, which would reload every pointer after each
    const int64_t *__restrict__ rowptr = S.rowptr;
    const int32_t *__restrict__ col = S.col;
    const double *__restrict__ val = S.val;
    const double *X = S.X;
    double *Y = S.Y;
    const int64_t r1 = min(r0 + cnt, S.n);
    auto load_x = [&](int64_t j, double (&o)[NB]) {
        if (NB == 1) {
            o[0] = __ldcg(&X[j * BK]);
        } else {
            const double2 a = __ldcg(reinterpret_cast<const double2 *>(X) + 2 * j);
            o[0] = a.x;
            o[NB > 1 ? 1 : 0] = a.y;
            if (NB > 2) {
                const double2 b = __ldcg(reinterpret_cast<const double2 *>(X) + 2 * j + 1);
                o[NB > 2 ? 2 : 0] = b.x;
                if (NB > 3) o[NB > 3 ? 3 : 0] = b.y;
            }
        }
    };
    for (int64_t i0 = r0 + (int64_t)warp * RPW; i0 < r1; i0 += (BT / 32) * RPW) {
        const int64_t i = i0 + sub;
        const bool ok = i < r1;
        double acc[NB], xi[NB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            acc[q] = 0.0;
            xi[q] = 0.0;
        }
        const int64_t beg = ok ? rowptr[i] : 0, end = ok ? rowptr[i + 1] : 0;
        if (ok) load_x(i, xi);
        for (int64_t p0 = beg + sl; p0 < end; p0 += LPR * SR) {
            int32_t j[SR];
            double v[SR], xv[SR][NB];
#pragma unroll
            for (int u = 0; u < SR; u++) {
                const int64_t p = p0 + LPR * u;
                j[u] = p < end ? __ldg(&col[p]) : -1;
                v[u] = p < end ? __ldg(&val[p]) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < SR; u++) {
                if (j[u] >= 0) load_x(j[u], xv[u]);
                else
#pragma unroll
                    for (int q = 0; q < NB; q++) xv[u][q] = 0.0;
            }
#pragma unroll
            for (int u = 0; u < SR; u++) {
                if (j[u] < 0) continue;
                double *yj = Y + (int64_t)j[u] * BK;
#pragma unroll
                for (int q = 0; q < NB; q++) {
                    acc[q] = fma(v[u], xv[u][q], acc[q]);
                    red_add(yj + q, v[u] * xi[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NB; q++) {
#pragma unroll
            for (int o = LPR / 2; o >= 1; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        }
        if (ok && sl == 0) {
#pragma unroll
            for (int q = 0; q < NB; q++)
                if (acc[q] != 0.0) red_add(&Y[i * BK + q], acc[q]);
        }
    }
}

template <int LPR, int MINB>
__device__ __forceinline__ void sigma_rows_upper(const BSys &S, int nb, int64_t r0, int cnt) {
    switch (nb) {
        case 1: sigma_rows_upper_nb<LPR, 1, MINB>(S, r0, cnt); break;
        case 2: sigma_rows_upper_nb<LPR, 2, MINB>(S, r0, cnt); break;
        case 3: sigma_rows_upper_nb<LPR, 3, MINB>(S, r0, cnt); break;
        default: sigma_rows_upper_nb<LPR, 4, MINB>(S, r0, cnt); break;
    }
}

// Y[i][q] = diag_i X[i][q], q < nb, for rows [r0, r0 + cnt): the start of an
// upper-triangle product
__device__ void diag_rows(const BSys &S, int nb, int64_t r0, int cnt) {
    const int64_t r1 = min(r0 + cnt, S.n);
    for (int64_t e = r0 * BK + threadIdx.x; e < r1 * BK; e += BT) {
        const int q = (int)(e % BK);
        if (q < nb) S.Y[e] = S.diag[e / BK] * __ldcg(&S.X[e]);
    }
}

// The enumeration items of the sigma phases, kept out of line: they are the
// hot code of an on-the-fly system, and as separate functions they get their
// registers allocated apart from the rest of the persistent kernel.
__device__ __noinline__ void batch_alpha_item(const BSys &S, int64_t local, EnumSmem<1> &es, int nb) {
    unsigned long long cand = 0;
    enum_alpha_item<1, ENUM_SIGMA, BK>(S.ea, S.I, local, es.T, es.Q[threadIdx.x >> 5], cand, nb);
}

__device__ __noinline__ void batch_beta_item(const BSys &S, int64_t local, EnumSmem<1> &es, int nb) {
    unsigned long long cand = 0;
    enum_beta_item<1, ENUM_SIGMA, BK>(S.eb, S.I, local, es.T, es.Q[threadIdx.x >> 5], cand, nb);
}

// ---------------------------------------------------------------- the persistent kernel

// MINB: CTAs per SM the kernel is compiled for (its register budget); the
// autotuner picks among the compiled variants.
template <int MINB>
__global__ void __launch_bounds__(BT, MINB) k_batch_davidson(BatchArgs B) {
    extern __shared__ double smem[];
    EnumSmem<1> &es = *reinterpret_cast<EnumSmem<1> *>(smem);
    double *sh = smem;                       // small-matrix scratch (phases never overlap)
    __shared__ double red[(BT / 32) * GA * BK];
    __shared__ int flag_sh;
    __shared__ int64_t pick[BK];
    __shared__ double bv[BT / 32];
    __shared__ int64_t bi[BT / 32];
    const int tid = threadIdx.x;

    if (blockIdx.x == 0 && tid == 0) B.bar->t_last = global_ns();
    // ---- init: unit vectors on the k lowest diagonal entries of each system
    for (int s = blockIdx.x; s < B.S; s += gridDim.x) {
        const BSys &S = B.sys[s];
        BState &st = B.st[s];
        for (int l = 0; l < S.k; l++) {
            double best = INFINITY;
            int64_t besti = INT64_MAX;
            for (int64_t i = tid; i < S.n; i += BT) {
                bool taken = false;
                for (int x = 0; x < l; x++) taken |= pick[x] == i;
                const double v = S.diag[i];
                if (!taken && (v < best || (v == best && i < besti))) { best = v; besti = i; }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int64_t oi = __shfl_xor_sync(0xffffffffu, besti, o);
                if (ov < best || (ov == best && oi < besti)) { best = ov; besti = oi; }
            }
            if ((tid & 31) == 0) { bv[tid >> 5] = best; bi[tid >> 5] = besti; }
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < BT / 32; w++)
                    if (bv[w] < best || (bv[w] == best && bi[w] < besti)) { best = bv[w]; besti = bi[w]; }
                pick[l] = besti;
            }
            __syncthreads();
        }
        double *V = S.Vb[0];
        for (int64_t e = tid; e < (int64_t)S.k * S.n; e += BT) {
            const int l = (int)(e / S.n);
            V[e] = (e % S.n == pick[l]) ? 1.0 : 0.0;
        }
        for (int64_t e = tid; e < (int64_t)BK * S.n; e += BT) {
            const int q = (int)(e % BK);
            S.X[e] = (q < S.k && e / BK == pick[q]) ? 1.0 : 0.0;
        }
        for (int e = tid; e < S.m_max * S.m_max; e += BT) S.G[e] = 0.0;
        if (tid == 0) {
            st.m = 0;
            st.nb = S.k;
            st.m_eig = 0;
            st.active = 1;
            st.restart = 0;
            st.it = 0;
            st.conv = 0;
            st.cur = 0;
            for (int l = 0; l < BK; l++) { st.theta_old[l] = INFINITY; st.theta[l] = 0.0; st.rn[l] = 0.0; }
        }
        __syncthreads();
    }
    if (!grid_sync(B.bar, 0, B.spin_limit)) return;

    for (int it = 0; it < B.max_iter; it++) {
        // ---- A1: sigma for stored rows and alpha-grouped on-the-fly items
        while (true) {
            const int item = next_item(B.bar);
            if (item >= B.n_a1) break;
            const int s = B.a1_sys[item];
            const BSys &S = B.sys[s];
            const int active = ldi(&B.st[s].active), nb = ldi(&B.st[s].nb);
            if (!active || nb == 0) continue;
            const int kind = B.a1_kind[item];
            if (kind == 0) {
                if (B.lpr == 32) sigma_rows<32, MINB>(S, nb, B.a1_local[item], B.srows);
                else sigma_rows<8, MINB>(S, nb, B.a1_local[item], B.srows);
            } else if (kind == 2) {
                diag_rows(S, nb, B.a1_local[item], B.srows);
            } else {
                batch_alpha_item(S, B.a1_local[item], es, nb);
            }
        }
        if (!grid_sync(B.bar, 1, B.spin_limit)) return;
        // ---- A2: beta-grouped on-the-fly items (adds the same-spin-alpha part)
        //         and the rows of upper-triangle matrices
        while (true) {
            const int item = next_item(B.bar);
            if (item >= B.n_a2) break;
            const int s = B.a2_sys[item];
            const BSys &S = B.sys[s];
            const int active = ldi(&B.st[s].active), nb = ldi(&B.st[s].nb);
            if (!active || nb == 0) continue;
            if (B.a2_kind[item] == 1) {
                if (B.lpr == 32) sigma_rows_upper<32, MINB>(S, nb, B.a2_local[item], B.srows);
                else sigma_rows_upper<8, MINB>(S, nb, B.a2_local[item], B.srows);
            } else {
                batch_beta_item(S, B.a2_local[item], es, nb);
            }
        }
        if (!grid_sync(B.bar, 2, B.spin_limit)) return;

        // ---- B: AV[m + q] = Y[:, q]; partial Gram columns V[a] . Y[:, q], a < m + nb
        for (int64_t item = blockIdx.x; item < B.n_v; item += gridDim.x) {
            const int s = B.v_sys[item];
            const BSys &S = B.sys[s];
            const BState &st = B.st[s];
            const int nb = ldi(&st.nb);
            if (!ldi(&st.active) || nb == 0) continue;
            const int m = ldi(&st.m), cur = ldi(&st.cur);
            const double *V = S.Vb[cur];
            double *AV = S.AVb[cur];
            const int64_t i0 = B.v_start[item], i1 = min(S.n, i0 + S.vslice);
            for (int64_t i = i0 + tid; i < i1; i += BT)
                for (int q = 0; q < nb; q++) AV[(int64_t)(m + q) * S.n + i] = __ldcg(&S.Y[i * BK + q]);
            auto loadY = [&](int64_t i, double (&b)[BK]) {
#pragma unroll
                for (int q = 0; q < BK; q++) b[q] = q < nb ? __ldcg(&S.Y[i * BK + q]) : 0.0;
            };
            slice_gram(B.partial + item * PSTRIDE, V, S.n, m + nb, i0, i1, loadY, red);
        }
        if (!grid_sync(B.bar, 3, B.spin_limit)) return;

        // ---- C: per system: new G columns, subspace eigen-decomposition
        for (int s = blockIdx.x; s < B.S; s += gridDim.x) {
            const BSys &S = B.sys[s];
            BState &st = B.st[s];
            if (!st.active || st.nb == 0) continue;
            const int m = st.m, nb = st.nb, mt = m + nb;
            for (int e = tid; e < mt * nb; e += BT) {
                const int a = e / nb, q = e % nb;
                const double v = sum_items(B, S, a * BK + q);
                S.G[a * S.m_max + m + q] = v;
                if (a < m) S.G[(m + q) * S.m_max + a] = v;   // the new corner: one writer per entry
            }
            __syncthreads();
            jacobi_solve<false>(S.G, S.m_max, mt, st.m_eig, S.eval, S.evec, sh, S.jq);
            __syncthreads();
            if (tid == 0) {
                st.m = mt;
                st.m_eig = mt;
                st.nb = 0;
            }
            __syncthreads();
        }
        if (!grid_sync(B.bar, 4, B.spin_limit)) return;

        // ---- D: Ritz vectors, residuals and corrections T[l] = r_l / (theta_l - H_ii);
        //         partials |r_l|^2, S0 = T^T T, C = V^T T
        for (int64_t item = blockIdx.x; item < B.n_v; item += gridDim.x) {
            const int s = B.v_sys[item];
            const BSys &S = B.sys[s];
            const BState &st = B.st[s];
            if (!ldi(&st.active)) continue;
            const int m = ldi(&st.m), k = S.k, cur = ldi(&st.cur);
            const double *V = S.Vb[cur], *AV = S.AVb[cur];
            double *ys = sh;                               // [m][BK]
            double *th = sh + SHCI_MAX_SUB * BK;
            for (int e = tid; e < m * BK; e += BT) {
                const int a = e / BK, l = e % BK;
                ys[e] = l < k ? __ldcg(&S.evec[l * S.m_max + a]) : 0.0;
            }
            if (tid < BK) th[tid] = tid < k ? __ldcg(&S.eval[tid]) : 0.0;
            __syncthreads();
            const int64_t i0 = B.v_start[item], i1 = min(S.n, i0 + S.vslice);
            double rs[BK * BK + BK];
#pragma unroll
            for (int e = 0; e < BK * BK + BK; e++) rs[e] = 0.0;
            for (int64_t i = i0 + tid; i < i1; i += BT) {
                double x[BK] = {0, 0, 0, 0}, h[BK] = {0, 0, 0, 0};
                for (int a = 0; a < m; a++) {
                    const double v = __ldcg(&V[(int64_t)a * S.n + i]), w = __ldcg(&AV[(int64_t)a * S.n + i]);
#pragma unroll
                    for (int l = 0; l < BK; l++) {
                        x[l] = fma(ys[a * BK + l], v, x[l]);
                        h[l] = fma(ys[a * BK + l], w, h[l]);
                    }
                }
                const double d = S.diag[i];
                double t[BK];
#pragma unroll
                for (int l = 0; l < BK; l++) {
                    const double r = fma(-th[l], x[l], h[l]);
                    double den = th[l] - d;
                    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
                    t[l] = l < k ? r / den : 0.0;
                    if (l < k) {
                        S.T[(int64_t)l * S.n + i] = t[l];
                        rs[BK * BK + l] = fma(r, r, rs[BK * BK + l]);
                    }
                }
#pragma unroll
                for (int l = 0; l < BK; l++)
#pragma unroll
                    for (int l2 = 0; l2 < BK; l2++) rs[l * BK + l2] = fma(t[l], t[l2], rs[l * BK + l2]);
            }
            double *part = B.partial + item * PSTRIDE;
            item_reduce<BK * BK + BK>(part + OFF_S0, rs, BK * BK + BK, red);
            auto loadT = [&](int64_t i, double (&b)[BK]) {
#pragma unroll
                for (int l = 0; l < BK; l++) b[l] = l < k ? __ldcg(&S.T[(int64_t)l * S.n + i]) : 0.0;
            };
            slice_gram(part, V, S.n, m, i0, i1, loadT, red);
        }
        if (!grid_sync(B.bar, 5, B.spin_limit)) return;

        // ---- E: per system: convergence, restart decision, coefficients of the kept corrections
        for (int s = blockIdx.x; s < B.S; s += gridDim.x) {
            const BSys &S = B.sys[s];
            BState &st = B.st[s];
            if (!st.active) continue;
            const int m = st.m, k = S.k;
            double *C = sh;                                  // [m][BK]
            double *S0 = sh + OFF_S0;                        // [BK][BK], then |r|^2 [BK]
            double *rn2 = sh + OFF_RN;
            for (int e = tid; e < m * BK; e += BT) C[e] = sum_items(B, S, e);
            for (int e = tid; e < BK * BK + BK; e += BT) S0[e] = sum_items(B, S, OFF_S0 + e);
            __syncthreads();
            if (tid == 0) {
                bool conv = true;
                int ntodo = 0;
                for (int l = 0; l < k; l++) {
                    st.theta[l] = S.eval[l];
                    st.rn[l] = sqrt(fmax(0.0, rn2[l]));
                    const bool cl = (fabs(st.theta[l] - st.theta_old[l]) < S.tol && st.rn[l] < S.res_tol) ||
                                    st.rn[l] < S.res_tol * 1e-3;
                    conv = conv && cl;
                    // a converged root is locked: no new direction for it
                    if (!cl) st.todo[ntodo++] = l;
                }
                for (int l = 0; l < k; l++) st.theta_old[l] = st.theta[l];
                st.it = st.it + 1;
                st.conv = conv ? 1 : 0;
                if (conv || st.it >= B.max_iter || ntodo == 0) st.active = 0;
                st.restart = (st.active && m + ntodo > S.m_max) ? 1 : 0;
                st.m_old = m;
                st.ntodo = ntodo;
                flag_sh = st.active ? (st.restart ? 2 : 1) : 0;
            }
            __syncthreads();
            if (flag_sh == 0) continue;
            const int ntodo = st.ntodo;
            if (flag_sh == 2) {
                // keep the `keep` lowest Ritz vectors: erot = evec[:, :keep];
                // C <- erot^T C, G <- diag(theta), evec <- I
                const int keep = min(m, S.keep);
                for (int e = tid; e < keep * m; e += BT) {
                    const int j = e / m, a = e % m;
                    S.erot[j * S.m_max + a] = S.evec[j * S.m_max + a];
                }
                __syncthreads();
                double *Cn = sh + OFF_RN + BK + 4;               // [keep][BK]
                for (int e = tid; e < keep * BK; e += BT) {
                    const int j = e / BK, l = e % BK;
                    double v = 0.0;
                    for (int a = 0; a < m; a++) v = fma(S.erot[j * S.m_max + a], C[a * BK + l], v);
                    Cn[e] = v;
                }
                __syncthreads();
                for (int e = tid; e < keep * BK; e += BT) C[e] = Cn[e];
                for (int e = tid; e < S.m_max * S.m_max; e += BT) {
                    const int r = e / S.m_max, c = e % S.m_max;
                    S.G[e] = (r == c && r < keep) ? S.eval[r] : 0.0;
                    S.evec[e] = (r == c) ? 1.0 : 0.0;
                }
                __syncthreads();
                if (tid == 0) {
                    st.m = keep;
                    st.m_eig = keep;
                }
                __syncthreads();
            }
            const int mm = st.m;
            for (int e = tid; e < mm * BK; e += BT) {
                const int a = e / BK, l = e % BK;
                S.coefC[e] = l < ntodo ? C[a * BK + st.todo[l]] : 0.0;
            }
            if (tid < BK) S.coefS0[tid] = tid < ntodo ? S0[st.todo[tid] * BK + st.todo[tid]] : 1.0;
            __syncthreads();
        }
        if (!grid_sync(B.bar, 6, B.spin_limit)) return;
        {
            int any = 0;
            for (int s = 0; s < B.S; s++) any |= ldi(&B.st[s].active);
            if (!any) break;
        }

        // ---- F: rotate the basis when restarting (V' = V erot, AV' = AV erot);
        //         first projection of the kept corrections into T2; partial V'^T T2
        for (int64_t item = blockIdx.x; item < B.n_v; item += gridDim.x) {
            const int s = B.v_sys[item];
            const BSys &S = B.sys[s];
            const BState &st = B.st[s];
            if (!ldi(&st.active)) continue;
            const int restart = ldi(&st.restart), m_old = ldi(&st.m_old), m = ldi(&st.m);
            const int ntodo = ldi(&st.ntodo), cur = ldi(&st.cur);
            int todo[BK];
#pragma unroll
            for (int l = 0; l < BK; l++) todo[l] = ldi(&st.todo[l]);
            double *cs = sh;                                 // [m][BK]
            double *er = sh + SHCI_MAX_SUB * BK;             // [keep][m_max]
            for (int e = tid; e < m * BK; e += BT) cs[e] = __ldcg(&S.coefC[e]);
            if (restart)
                for (int e = tid; e < m * S.m_max; e += BT) er[e] = __ldcg(&S.erot[e]);
            __syncthreads();
            const double *V = S.Vb[cur], *AV = S.AVb[cur];
            double *Vn = S.Vb[cur ^ 1], *AVn = S.AVb[cur ^ 1];
            const double *Vp = restart ? Vn : V;
            const int64_t i0 = B.v_start[item], i1 = min(S.n, i0 + S.vslice);
            for (int64_t i = i0 + tid; i < i1; i += BT) {
                double t[BK];
#pragma unroll
                for (int l = 0; l < BK; l++) t[l] = l < ntodo ? __ldcg(&S.T[(int64_t)todo[l] * S.n + i]) : 0.0;
                if (restart) {
                    for (int j = 0; j < m; j++) {
                        double v = 0.0, w = 0.0;
                        for (int a = 0; a < m_old; a++) {
                            const double e = er[j * S.m_max + a];
                            v = fma(e, __ldcg(&V[(int64_t)a * S.n + i]), v);
                            w = fma(e, __ldcg(&AV[(int64_t)a * S.n + i]), w);
                        }
                        Vn[(int64_t)j * S.n + i] = v;
                        AVn[(int64_t)j * S.n + i] = w;
#pragma unroll
                        for (int l = 0; l < BK; l++) t[l] = fma(-cs[j * BK + l], v, t[l]);
                    }
                } else {
                    for (int a = 0; a < m; a++) {
                        const double v = __ldcg(&V[(int64_t)a * S.n + i]);
#pragma unroll
                        for (int l = 0; l < BK; l++) t[l] = fma(-cs[a * BK + l], v, t[l]);
                    }
                }
#pragma unroll
                for (int l = 0; l < BK; l++)
                    if (l < ntodo) S.T2[(int64_t)l * S.n + i] = t[l];
            }
            __syncthreads();
            auto loadT2 = [&](int64_t i, double (&b)[BK]) {
#pragma unroll
                for (int l = 0; l < BK; l++) b[l] = l < ntodo ? __ldcg(&S.T2[(int64_t)l * S.n + i]) : 0.0;
            };
            slice_gram(B.partial + item * PSTRIDE, Vp, S.n, m, i0, i1, loadT2, red);
        }
        if (!grid_sync(B.bar, 7, B.spin_limit)) return;

        // ---- G: per system: switch to the rotated buffers; second-pass coefficients
        for (int s = blockIdx.x; s < B.S; s += gridDim.x) {
            const BSys &S = B.sys[s];
            BState &st = B.st[s];
            if (!st.active) continue;
            const int m = st.m, ntodo = st.ntodo;
            for (int e = tid; e < m * BK; e += BT) S.coefC[e] = (e % BK) < ntodo ? sum_items(B, S, e) : 0.0;
            __syncthreads();
            if (tid == 0 && st.restart) {
                st.cur ^= 1;
                st.restart = 0;
            }
            __syncthreads();
        }
        if (!grid_sync(B.bar, 8, B.spin_limit)) return;

        // ---- H: second projection T2 -= V C2; partial S = T2^T T2
        for (int64_t item = blockIdx.x; item < B.n_v; item += gridDim.x) {
            const int s = B.v_sys[item];
            const BSys &S = B.sys[s];
            const BState &st = B.st[s];
            if (!ldi(&st.active)) continue;
            const int m = ldi(&st.m), ntodo = ldi(&st.ntodo), cur = ldi(&st.cur);
            const double *V = S.Vb[cur];
            double *cs = sh;
            for (int e = tid; e < m * BK; e += BT) cs[e] = __ldcg(&S.coefC[e]);
            __syncthreads();
            const int64_t i0 = B.v_start[item], i1 = min(S.n, i0 + S.vslice);
            double s2[BK * BK];
#pragma unroll
            for (int e = 0; e < BK * BK; e++) s2[e] = 0.0;
            for (int64_t i = i0 + tid; i < i1; i += BT) {
                double t[BK];
#pragma unroll
                for (int l = 0; l < BK; l++) t[l] = l < ntodo ? __ldcg(&S.T2[(int64_t)l * S.n + i]) : 0.0;
                for (int a = 0; a < m; a++) {
                    const double v = __ldcg(&V[(int64_t)a * S.n + i]);
#pragma unroll
                    for (int l = 0; l < BK; l++) t[l] = fma(-cs[a * BK + l], v, t[l]);
                }
#pragma unroll
                for (int l = 0; l < BK; l++) {
                    if (l < ntodo) S.T2[(int64_t)l * S.n + i] = t[l];
#pragma unroll
                    for (int l2 = 0; l2 < BK; l2++) s2[l * BK + l2] = fma(t[l], t[l2], s2[l * BK + l2]);
                }
            }
            item_reduce<BK * BK>(B.partial + item * PSTRIDE, s2, BK * BK, red);
        }
        if (!grid_sync(B.bar, 9, B.spin_limit)) return;

        // ---- I: per system: Cholesky-QR coefficients, pass 1 (dependence test
        //         against the norms before projection)
        for (int s = blockIdx.x; s < B.S; s += gridDim.x) {
            const BSys &S = B.sys[s];
            BState &st = B.st[s];
            if (!st.active) continue;
            const int nt = st.ntodo;
            for (int e = tid; e < nt * nt; e += BT) S.coefS[e] = sum_items(B, S, (e / nt) * BK + e % nt);
            __syncthreads();
            if (tid == 0) st.cnt1 = cholqr_coef(S.coefS, nt, S.coefS0, 1e-20, S.coefM);
            __syncthreads();
        }
        if (!grid_sync(B.bar, 10, B.spin_limit)) return;

        // ---- J: T = T2 M (zero past cnt1); partial S = T^T T
        for (int64_t item = blockIdx.x; item < B.n_v; item += gridDim.x) {
            const int s = B.v_sys[item];
            const BSys &S = B.sys[s];
            const BState &st = B.st[s];
            if (!ldi(&st.active)) continue;
            const int nt = ldi(&st.ntodo), c1 = ldi(&st.cnt1);
            double *ms = sh;
            for (int e = tid; e < nt * nt; e += BT) ms[e] = __ldcg(&S.coefM[e]);
            __syncthreads();
            const int64_t i0 = B.v_start[item], i1 = min(S.n, i0 + S.vslice);
            double s2[BK * BK];
#pragma unroll
            for (int e = 0; e < BK * BK; e++) s2[e] = 0.0;
            for (int64_t i = i0 + tid; i < i1; i += BT) {
                double t[BK], u[BK];
#pragma unroll
                for (int l = 0; l < BK; l++) t[l] = l < nt ? __ldcg(&S.T2[(int64_t)l * S.n + i]) : 0.0;
#pragma unroll
                for (int l = 0; l < BK; l++) {
                    double v = 0.0;
                    if (l < c1)
                        for (int j = 0; j < nt; j++) v = fma(ms[j * nt + l], t[j], v);
                    u[l] = v;
                    if (l < nt) S.T[(int64_t)l * S.n + i] = v;
                }
#pragma unroll
                for (int l = 0; l < BK; l++)
#pragma unroll
                    for (int l2 = 0; l2 < BK; l2++) s2[l * BK + l2] = fma(u[l], u[l2], s2[l * BK + l2]);
            }
            item_reduce<BK * BK>(B.partial + item * PSTRIDE, s2, BK * BK, red);
        }
        if (!grid_sync(B.bar, 11, B.spin_limit)) return;

        // ---- K: per system: Cholesky-QR coefficients, pass 2
        for (int s = blockIdx.x; s < B.S; s += gridDim.x) {
            const BSys &S = B.sys[s];
            BState &st = B.st[s];
            if (!st.active) continue;
            const int nt = st.ntodo;
            for (int e = tid; e < nt * nt; e += BT) S.coefS[e] = sum_items(B, S, (e / nt) * BK + e % nt);
            __syncthreads();
            if (tid == 0) {
                int c2 = cholqr_coef(S.coefS, nt, nullptr, 1e-12, S.coefM2);
                st.cnt2 = min(c2, S.m_max - st.m);      // never grow past the subspace buffers
            }
            __syncthreads();
        }
        if (!grid_sync(B.bar, 12, B.spin_limit)) return;

        // ---- L: new basis vectors V[m + l] = T M2 (l < cnt2) and the next sigma input X
        for (int64_t item = blockIdx.x; item < B.n_v; item += gridDim.x) {
            const int s = B.v_sys[item];
            const BSys &S = B.sys[s];
            const BState &st = B.st[s];
            if (!ldi(&st.active)) continue;
            const int nt = ldi(&st.ntodo), c2 = ldi(&st.cnt2), m = ldi(&st.m), cur = ldi(&st.cur);
            double *V = S.Vb[cur];
            double *ms = sh;
            for (int e = tid; e < nt * nt; e += BT) ms[e] = __ldcg(&S.coefM2[e]);
            __syncthreads();
            const int64_t i0 = B.v_start[item], i1 = min(S.n, i0 + S.vslice);
            for (int64_t i = i0 + tid; i < i1; i += BT) {
                double t[BK], o[BK];
#pragma unroll
                for (int l = 0; l < BK; l++) t[l] = l < nt ? __ldcg(&S.T[(int64_t)l * S.n + i]) : 0.0;
#pragma unroll
                for (int l = 0; l < BK; l++) {
                    double v = 0.0;
                    if (l < c2) {
                        for (int j = 0; j < nt; j++) v = fma(ms[j * nt + l], t[j], v);
                        V[(int64_t)(m + l) * S.n + i] = v;
                    }
                    o[l] = v;
                }
                reinterpret_cast<double4 *>(S.X)[i] = make_double4(o[0], o[1], o[2], o[3]);
            }
            __syncthreads();
        }
        if (!grid_sync(B.bar, 13, B.spin_limit)) return;

        // ---- M: per system: the new block is ready for the next sigma
        if (tid == 0)
            for (int s = blockIdx.x; s < B.S; s += gridDim.x) {
                BState &st = B.st[s];
                if (!st.active) continue;
                st.nb = st.cnt2;
                if (st.cnt2 == 0) st.active = 0;     // no new direction: this system stops here
            }
        if (!grid_sync(B.bar, 14, B.spin_limit)) return;
    }
}

// dynamic shared memory: the eigensolver's working matrix (its rotations are
// accumulated in global scratch), the enumeration's tiles and queues, or the
// small-matrix scratch of the vector phases, whichever is largest
constexpr size_t BATCH_SCRATCH = sizeof(double) * (SHCI_MAX_SUB * BK + 24 * SHCI_MAX_SUB);
constexpr size_t BATCH_SMEM = JACOBI_SMEM_A > sizeof(EnumSmem<1>)
                                  ? (JACOBI_SMEM_A > BATCH_SCRATCH ? JACOBI_SMEM_A : BATCH_SCRATCH)
                                  : (sizeof(EnumSmem<1>) > BATCH_SCRATCH ? sizeof(EnumSmem<1>) : BATCH_SCRATCH);

// the compiled variants of the persistent kernel (CTAs per SM)
constexpr int BATCH_MINB_LO = 2, BATCH_MINB_HI = 5;

inline void (*batch_kernel(int minb))(BatchArgs) {
    switch (minb) {
        case 2: return k_batch_davidson<2>;
        case 3: return k_batch_davidson<3>;
        case 4: return k_batch_davidson<4>;
        default: return k_batch_davidson<5>;
    }
}

}  // namespace shci

// ======================================================================== host side

struct shci_batch {
    shci_ctx *parent = nullptr;
    std::vector<shci_ctx *> subs;
    int S = 0;
    int k = 0;                      // roots the Davidson buffers were sized for
    std::vector<shci::BSys> h_sys;
    std::vector<DevBuf<double> *> owned;
    DevBuf<shci::BSys> d_sys;
    DevBuf<shci::BState> d_st;
    DevBuf<shci::BarrierState> d_bar;
    DevBuf<int32_t> a1_sys, a1_kind, a2_sys, a2_kind, v_sys;
    DevBuf<int64_t> a1_local, a2_local, v_start;
    DevBuf<double> partial;
    int64_t n_a1 = 0, n_a2 = 0, n_v = 0;
    int vslice = shci::VSLICE;      // vector elements per vector work item
    int srows = 256, blocks_per_sm = 3, lpr = 32, grid = 0;
    std::vector<int> modes;         // storage mode of each system
    bool tuned = false;
    cudaGraphExec_t gexec = nullptr;
    int graph_max_iter = -1;
    long long spin_limit = shci::BARRIER_SPIN_LIMIT;
    long long graph_spin_limit = -1;
    double graph_tol = -1.0;
    bool graph_ok = false;
    shci_batch_stats_t stats{};
    ~shci_batch() {
        if (gexec) cudaGraphExecDestroy(gexec);
        for (auto *b : owned) delete b;
        for (auto *c : subs) delete c;
    }
    double *alloc(size_t n) {
        auto *b = new DevBuf<double>();
        owned.push_back(b);
        b->alloc(n);
        return b->p;
    }
};

namespace {

template <typename T>
void upload(DevBuf<T> &d, const std::vector<T> &h, cudaStream_t st) {
    d.alloc(std::max<size_t>(h.size(), 1));
    if (!h.empty()) CUDA_TRY(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
}

void launch_batch(shci_batch *b, int max_iter, bool capture_ok) {
    using namespace shci;
    cudaStream_t st = b->parent->st;
    BatchArgs A{};
    A.S = b->S;
    A.sys = b->d_sys.p;
    A.st = b->d_st.p;
    A.max_iter = max_iter;
    A.a1_sys = b->a1_sys.p;
    A.a1_kind = b->a1_kind.p;
    A.a1_local = b->a1_local.p;
    A.n_a1 = b->n_a1;
    A.a2_sys = b->a2_sys.p;
    A.a2_kind = b->a2_kind.p;
    A.a2_local = b->a2_local.p;
    A.n_a2 = b->n_a2;
    A.srows = b->srows;
    A.lpr = b->lpr;
    A.v_sys = b->v_sys.p;
    A.v_start = b->v_start.p;
    A.n_v = b->n_v;
    A.partial = b->partial.p;
    A.bar = b->d_bar.p;
    A.spin_limit = b->spin_limit;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = BATCH_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(b->d_bar.p, 0, sizeof(BarrierState), st);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, batch_kernel(b->blocks_per_sm), A);
    };
    if (capture_ok) {
        // one persistent launch captured in a CUDA graph, re-instantiated when its parameters change
        if (!b->gexec || b->graph_max_iter != max_iter || b->graph_spin_limit != b->spin_limit) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                cudaError_t e1 = enqueue();
                cudaError_t e2 = cudaStreamEndCapture(st, &g);
                ok = e1 == cudaSuccess && e2 == cudaSuccess && g != nullptr &&
                     cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess;
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();     // a failed capture leaves a recoverable error; clear it
            if (!ok) {
                if (b->gexec) cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            b->graph_max_iter = max_iter;
            b->graph_spin_limit = b->spin_limit;
        }
        if (b->gexec) {
            CUDA_TRY(cudaGraphLaunch(b->gexec, st));
            b->graph_ok = true;
            return;
        }
    }
    b->graph_ok = false;
    CUDA_TRY(enqueue());
}

double time_batch(shci_batch *b, int max_iter) {
    cudaStream_t st = b->parent->st;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e0, st));
    launch_batch(b, max_iter, false);
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// work lists for the current stored-row chunk size
void build_worklists(shci_batch *b) {
    std::vector<int32_t> a1s, a1k, a2s, a2k;
    std::vector<int64_t> a1l, a2l;
    for (int s = 0; s < b->S; s++) {
        shci_ctx *c = b->subs[s];
        if (c->mode == SHCI_STORED) {
            for (int64_t r = 0; r < c->n_det; r += b->srows) {
                a1s.push_back(s);
                a1k.push_back(0);
                a1l.push_back(r);
            }
        } else if (c->mode == SHCI_STORED_UPPER) {
            for (int64_t r = 0; r < c->n_det; r += b->srows) {
                a1s.push_back(s);
                a1k.push_back(2);
                a1l.push_back(r);
                a2s.push_back(s);
                a2k.push_back(1);
                a2l.push_back(r);
            }
        } else {
            for (int64_t t = 0; t < c->n_items_a; t++) {
                a1s.push_back(s);
                a1k.push_back(1);
                a1l.push_back(t);
            }
            for (int64_t t = 0; t < c->n_items_b; t++) {
                a2s.push_back(s);
                a2k.push_back(0);
                a2l.push_back(t);
            }
        }
    }
    cudaStream_t st = b->parent->st;
    upload(b->a1_sys, a1s, st);
    upload(b->a1_kind, a1k, st);
    upload(b->a1_local, a1l, st);
    upload(b->a2_sys, a2s, st);
    upload(b->a2_kind, a2k, st);
    upload(b->a2_local, a2l, st);
    b->n_a1 = (int64_t)a1s.size();
    b->n_a2 = (int64_t)a2s.size();
    CUDA_TRY(cudaStreamSynchronize(st));
}

void set_grid(shci_batch *b) {
    CUDA_TRY(cudaFuncSetAttribute(shci::batch_kernel(b->blocks_per_sm), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shci::BATCH_SMEM));
    int occ = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, shci::batch_kernel(b->blocks_per_sm), shci::BT,
                                                           shci::BATCH_SMEM));
    if (occ < 1) throw ShciError{SHCI_ERR_CUDA, "the batched solver does not fit on one SM"};
    b->grid = b->parent->n_sm * std::min(occ, b->blocks_per_sm);
}

// vector work items: slices of b->vslice elements of every system's vectors
void build_vitems(shci_batch *b) {
    using namespace shci;
    std::vector<int32_t> vs;
    std::vector<int64_t> vst;
    for (int s = 0; s < b->S; s++) {
        BSys &S = b->h_sys[s];
        S.vslice = b->vslice;
        S.v_item_off = (int64_t)vs.size();
        for (int64_t i0 = 0; i0 < S.n; i0 += S.vslice) {
            vs.push_back(s);
            vst.push_back(i0);
        }
        S.v_item_cnt = (int64_t)vs.size() - S.v_item_off;
    }
    cudaStream_t st = b->parent->st;
    upload(b->v_sys, vs, st);
    upload(b->v_start, vst, st);
    b->n_v = (int64_t)vs.size();
    b->partial.alloc((size_t)b->n_v * PSTRIDE);
    upload(b->d_sys, b->h_sys, st);
    CUDA_TRY(cudaStreamSynchronize(st));
}

void prepare_davidson(shci_batch *b, int k, double tol) {
    using namespace shci;
    cudaStream_t st = b->parent->st;
    if (b->k != k) {
        for (auto *x : b->owned) delete x;
        b->owned.clear();
        for (int s = 0; s < b->S; s++) {
            shci_ctx *c = b->subs[s];
            BSys &S = b->h_sys[s];
            const int64_t n = c->n_det;
            if (k > n) throw ShciError{SHCI_ERR_INVALID, "k_roots exceeds the size of a system"};
            S.k = k;
            // the subspace rule of shci_davidson: 16 + 8k vectors with a stored H,
            // 16 + 16k on the fly (at most 64)
            const int per_root = c->mode == SHCI_ON_THE_FLY ? 16 : 8;
            S.m_max = (int)std::min<int64_t>(std::min(SHCI_MAX_SUB, 16 + per_root * k), n);
            if (S.m_max < k) S.m_max = k;
            S.keep = std::max(k, std::min(S.m_max - k, std::max(2 * k, S.m_max / 3)));
            if (S.keep > 24) throw ShciError{SHCI_ERR_INVALID, "restart block exceeds the batch scratch"};
            for (int x = 0; x < 2; x++) {
                S.Vb[x] = b->alloc((size_t)S.m_max * n);
                S.AVb[x] = b->alloc((size_t)S.m_max * n);
            }
            S.T = b->alloc((size_t)BK * n);
            S.T2 = b->alloc((size_t)BK * n);
            S.X = b->alloc((size_t)BK * n);
            S.Y = b->alloc((size_t)BK * n);
            for (EnumArgs *e : {&S.ea, &S.eb}) {
                e->x = S.X;
                e->y = S.Y;
                e->diag = S.diag;
                e->k_active = 0;
            }
            S.G = b->alloc((size_t)S.m_max * S.m_max);
            S.evec = b->alloc((size_t)S.m_max * S.m_max);
            S.erot = b->alloc((size_t)S.m_max * S.m_max);
            S.jq = b->alloc((size_t)JACOBI_Q_DOUBLES);
            S.eval = b->alloc((size_t)S.m_max);
            S.coefC = b->alloc((size_t)SHCI_MAX_SUB * BK);
            S.coefS0 = b->alloc(BK);
            S.coefS = b->alloc(BK * BK);
            S.coefM = b->alloc(BK * BK);
            S.coefM2 = b->alloc(BK * BK);
        }
        build_vitems(b);
        b->d_st.alloc((size_t)b->S);
        b->d_bar.alloc(1);
        b->k = k;
    }
    for (auto &S : b->h_sys) {
        S.tol = tol;
        S.res_tol = 0.1 * std::sqrt(tol);
    }
    upload(b->d_sys, b->h_sys, st);
    CUDA_TRY(cudaStreamSynchronize(st));
}

// project autotuner: rows per stored-sigma work item and CTAs per SM, chosen by
// timing a few iterations of the real kernel for each candidate
void autotune(shci_batch *b) {
    // rows per stored-sigma item with the middle variant, then the variant
    // (register budget / CTAs per SM) with the best rows
    const int rows_c[3] = {64, 256, 1024};
    double best = INFINITY;
    int best_rows = b->srows, best_bps = 3;
    auto trial = [&](int r, int p) {
        b->srows = r;
        b->blocks_per_sm = p;
        build_worklists(b);
        set_grid(b);
        const double ms = time_batch(b, 3);
        shci::BarrierState bar{};
        CUDA_TRY(cudaMemcpy(&bar, b->d_bar.p, sizeof(bar), cudaMemcpyDeviceToHost));
        if (bar.err) throw ShciError{SHCI_ERR_TIMEOUT, "batched solver: grid barrier timed out while tuning"};
        if (ms < best) {
            best = ms;
            best_rows = r;
            best_bps = p;
        }
    };
    for (int r : rows_c) trial(r, 3);
    const int rows_best = best_rows;
    for (int p = shci::BATCH_MINB_LO; p <= shci::BATCH_MINB_HI; p++)
        if (p != 3) trial(rows_best, p);
    // lanes per stored row: a warp per determinant, or 8 lanes (4 rows per warp)
    int best_lpr = 32;
    if (b->stats.n_stored + b->stats.n_stored_upper > 0) {
        const double before = best;
        b->lpr = 8;
        trial(best_rows, best_bps);
        if (best < before) best_lpr = 8;
    }
    b->lpr = best_lpr;
    // elements per vector item: shorter slices give the phases over vectors
    // more items when one or a few large systems hold most of the elements
    // (more partial sums to add up otherwise: the full 64-system batch keeps
    // 8192, a lone 1e6-determinant system takes 2048)
    int best_vs = b->vslice;
    {
        const double before = best;
        b->vslice = 2048;
        build_vitems(b);
        trial(best_rows, best_bps);
        if (best < before) best_vs = 2048;
    }
    b->vslice = best_vs;
    build_vitems(b);
    b->srows = best_rows;
    b->blocks_per_sm = best_bps;
    build_worklists(b);
    set_grid(b);
    b->stats.tuned_rows_per_item = best_rows;
    b->stats.tuned_ctas_per_sm = best_bps;
    b->stats.tuned_lanes_per_row = best_lpr;
    b->stats.tuned_vslice = best_vs;
    b->stats.tune_ms = best;
    b->tuned = true;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

}  // namespace

extern "C" {

int shci_batch_create(shci_ctx *ctx, int n_sys, const shci_system_desc *systems, int mem_space,
                      double stored_budget_bytes, shci_batch **out) {
    if (!ctx || !out) return SHCI_ERR_INVALID;
    *out = nullptr;
    shci_batch *b = nullptr;
    try {
        CUDA_TRY(cudaSetDevice(ctx->device));
        ctx->err.clear();
        if (n_sys < 1 || !systems) throw ShciError{SHCI_ERR_INVALID, "need at least one system"};
        b = new shci_batch();
        b->parent = ctx;
        b->S = n_sys;
        // pass 1: helper lists, diagonal and pair count of every system
        for (int s = 0; s < n_sys; s++) {
            const shci_system_desc &d = systems[s];
            if (d.n_orb < 1 || d.n_orb > 64) throw ShciError{SHCI_ERR_INVALID, "batched systems need n_orb <= 64"};
            shci_ctx *c = new shci_ctx();
            b->subs.push_back(c);
            c->device = ctx->device;
            c->st = ctx->st;
            c->own_stream = false;
            c->n_sm = ctx->n_sm;
            CUDA_TRY(cudaEventCreate(&c->ev0));
            CUDA_TRY(cudaEventCreate(&c->ev1));
            shci::load_integrals(c, d.n_orb, d.e_core, d.h, d.eri_packed, mem_space);
            shci::build(c, d.n_alpha, d.n_beta, d.n_det, d.dets, mem_space, SHCI_ON_THE_FLY);
            b->stats.total_det += c->n_det;
            b->stats.total_nnz_upper += c->nnz_upper;
        }
        // the storage plan (plan.h) within the budget and 80 % of the free memory
        size_t free_b = 0, total_b = 0;
        CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        double left = 0.8 * (double)free_b;
        if (stored_budget_bytes >= 0.0) left = std::min(left, stored_budget_bytes);
        std::vector<int64_t> pairs;
        for (auto *c : b->subs) pairs.push_back(c->nnz_upper);
        b->modes = shci::storage_plan(pairs, left);
        // pass 2: store, and describe each system to the kernel
        for (int s = 0; s < n_sys; s++) {
            shci_ctx *c = b->subs[s];
            if (b->modes[s] != SHCI_ON_THE_FLY) shci::store(c, b->modes[s]);
            if (c->mode == SHCI_STORED) b->stats.n_stored++;
            else if (c->mode == SHCI_STORED_UPPER) b->stats.n_stored_upper++;
            else b->stats.n_on_the_fly++;
            shci::BSys S{};
            S.n = c->n_det;
            S.mode = c->mode;
            S.rowptr = c->rowptr.p;
            S.col = c->col.p;
            S.val = c->val.p;
            S.diag = c->diag.p;
            S.ea = shci::enum_args(c);
            S.ea.item_group = c->item_a_group.p;
            S.ea.item_first = c->item_a_first.p;
            S.ea.n_items = c->n_items_a;
            S.ea.accumulate = 0;
            S.eb = shci::enum_args(c);
            S.eb.item_group = c->item_b_group.p;
            S.eb.item_first = c->item_b_first.p;
            S.eb.n_items = c->n_items_b;
            S.eb.accumulate = 1;
            S.I = shci::dev_ints(c);
            b->h_sys.push_back(S);
        }
        b->stats.n_sys = n_sys;
        build_worklists(b);
        set_grid(b);
        *out = b;
        return SHCI_OK;
    } catch (const ShciError &e) {
        ctx->err = e.msg;
        delete b;
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        delete b;
        return SHCI_ERR_INVALID;
    }
}

int shci_batch_davidson(shci_batch *b, int k_roots, double tol, int max_iter, double *energies, int *iters,
                        int *converged) {
    if (!b) return SHCI_ERR_INVALID;
    shci_ctx *ctx = b->parent;
    try {
        CUDA_TRY(cudaSetDevice(ctx->device));
        ctx->err.clear();
        if (k_roots < 1 || k_roots > shci::BK) throw ShciError{SHCI_ERR_INVALID, "batched k_roots must be in [1, 4]"};
        if (!(tol > 0.0) || max_iter < 1) throw ShciError{SHCI_ERR_INVALID, "bad tol or max_iter"};
        if (!energies) throw ShciError{SHCI_ERR_INVALID, "energies must not be NULL"};
        prepare_davidson(b, k_roots, tol);
        if (!b->tuned) autotune(b);
        cudaStream_t st = ctx->st;
        cudaEvent_t e0, e1;
        CUDA_TRY(cudaEventCreate(&e0));
        CUDA_TRY(cudaEventCreate(&e1));
        CUDA_TRY(cudaEventRecord(e0, st));
        launch_batch(b, max_iter, true);
        CUDA_TRY(cudaEventRecord(e1, st));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        g_kernel_launches += 1;
        shci::BarrierState bar{};
        CUDA_TRY(cudaMemcpy(&bar, b->d_bar.p, sizeof(bar), cudaMemcpyDeviceToHost));
        if (bar.err) throw ShciError{SHCI_ERR_TIMEOUT, "batched solver: grid barrier timed out"};
        std::vector<shci::BState> hs(b->S);
        CUDA_TRY(cudaMemcpy(hs.data(), b->d_st.p, sizeof(shci::BState) * b->S, cudaMemcpyDeviceToHost));
        bool all = true;
        int max_it = 0;
        for (int s = 0; s < b->S; s++) {
            for (int l = 0; l < k_roots; l++) energies[s * k_roots + l] = hs[s].theta[l];
            if (iters) iters[s] = hs[s].it;
            if (converged) converged[s] = hs[s].conv;
            all = all && hs[s].conv;
            max_it = std::max(max_it, hs[s].it);
        }
        b->stats.solve_ms = ms;
        for (int ph = 0; ph < 16; ph++) b->stats.phase_ms[ph] = ph < shci::N_PHASES ? bar.phase_ns[ph] * 1e-6 : 0.0;
        b->stats.max_iters = max_it;
        b->stats.graph = b->graph_ok ? 1 : 0;
        b->stats.grid_ctas = b->grid;
        if (!all) {
            ctx->err = "some systems did not converge within max_iter";
            return SHCI_ERR_NOT_CONVERGED;
        }
        return SHCI_OK;
    } catch (const ShciError &e) {
        ctx->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        return SHCI_ERR_INVALID;
    }
}

int shci_batch_get_modes(const shci_batch *b, int cap, int *modes) {
    if (!b || !modes || cap < b->S) return SHCI_ERR_INVALID;
    for (int s = 0; s < b->S; s++) modes[s] = b->modes[s];
    return SHCI_OK;
}

int shci_batch_set_wait_limit(shci_batch *b, long long naps) {
    if (!b) return SHCI_ERR_INVALID;
    b->spin_limit = naps < 0 ? shci::BARRIER_SPIN_LIMIT : naps;
    return SHCI_OK;
}

int shci_batch_get_stats(shci_batch *b, shci_batch_stats_t *out) {
    if (!b || !out) return SHCI_ERR_INVALID;
    *out = b->stats;
    return SHCI_OK;
}

void shci_batch_destroy(shci_batch *b) {
    if (!b) return;
    cudaSetDevice(b->parent->device);
    cudaStreamSynchronize(b->parent->st);
    delete b;
}

}  // extern "C"
