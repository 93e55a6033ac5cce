// sigma = H c: the matrix-vector product of each Davidson step (Sec. V.B).
//
// SHCI_STORED keeps both triangles of H as CSR rows (diagonal separate), so a
// row's product is a pure gather: one FP64 FMA per stored nonzero per vector
// and no atomics.  SHCI_STORED_UPPER keeps the upper triangle alone, as the
// paper does (half the memory), and adds the transposed half with FP64 atomic
// adds into L2; on GB300 those run at about 0.4 of the FP64 FMA rate, so this
// form is used when both triangles do not fit.
#include <algorithm>
#include <atomic>

#include "enum_launch.cuh"


namespace shci {

constexpr int SIGMA_THREADS = 256;

// Shape of the stored product for up to two vectors: rows per warp group,
// nonzeros per lane per step, CTAs per SM the kernel is compiled for.  On the
// 1e6-determinant heat-bath space (two vectors, GB300) 4 / 8 / 4 (64
// registers) took 4.83 ms and 8 / 4 / 4 4.93 ms; shapes that fit more CTAs
// were slower (4 / 4 / 5 5.16 ms, 4 / 2 / 5 5.39, 2 / 4 / 6 5.85, 4 / 2 / 6
// 6.30), and so were deeper steps at fewer CTAs (8 / 6 / 3 5.18, 4 / 8 / 3
// 5.25, 8 / 8 / 3 5.32, 8 / 8 / 2 5.59); deeper steps at 4 CTAs spill.
#ifndef SHCI_SIGMA_R2
#define SHCI_SIGMA_R2 4
#endif
#ifndef SHCI_SIGMA_SR2
#define SHCI_SIGMA_SR2 8
#endif
#ifndef SHCI_SIGMA_MINB2
#define SHCI_SIGMA_MINB2 4
#endif

// Rows per warp group: a warp takes R consecutive rows one after another,
// keeps each row's per-lane partial sums in registers, and reduces the R rows
// together at the end (below); fewer rows for more vectors (registers).
template <int K, bool INTER>
struct SigmaRows {
    // the shapes the Davidson iteration launches (one vector, or two interleaved)
    static constexpr bool TUNED = K == 1 || (K == 2 && INTER);
    static constexpr int R = TUNED ? SHCI_SIGMA_R2 : (K <= 4 ? 4 : 2);
    static constexpr int SR = TUNED ? SHCI_SIGMA_SR2 : 2;
    static constexpr int MINB = TUNED ? SHCI_SIGMA_MINB2 : 1;
};

// A warp per group of R consecutive rows.  x and y are [n][K] (INTER) or
// [K][n].  For each row of the group, each lane takes SR nonzeros per step and
// issues all their loads before the FMAs (more gathers of x in flight); a step
// slot with no nonzero of the row in any lane is skipped by a warp-uniform
// branch.  The FP64 pipe is the binding unit, so the per-row cost besides the
// one FMA per nonzero and vector is kept small: instead of a 5-level shuffle
// reduction per row and vector, the R rows' partial sums are reduced together
// by a butterfly that halves the rows a lane holds at each of the first
// log2(R) levels ((R - 1) + (5 - log2 R) adds per vector for R rows), and one
// lane per row writes y = H_ii x + sum.
template <int K, bool INTER>
__global__ void __launch_bounds__(SIGMA_THREADS, SigmaRows<K, INTER>::MINB) k_sigma_stored(int64_t n,
                                                                                   const int64_t *__restrict__ rowptr,
                                                                const int32_t *__restrict__ col,
                                                                const double *__restrict__ val,
                                                                const double *__restrict__ diag,
                                                                const double *__restrict__ x, double *__restrict__ y) {
    constexpr int SR = SigmaRows<K, INTER>::SR;
    constexpr int R = SigmaRows<K, INTER>::R;
    constexpr int LOG_R = R == 8 ? 3 : (R == 4 ? 2 : (R == 2 ? 1 : 0));
    const int lane = threadIdx.x & 31;
    const int64_t n_groups = (n + R - 1) / R;
    const int64_t warps = (int64_t)gridDim.x * (SIGMA_THREADS / 32);
    for (int64_t g = ((int64_t)blockIdx.x * SIGMA_THREADS + threadIdx.x) >> 5; g < n_groups; g += warps) {
        const int64_t i0 = g * R;
        double acc[R][K];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int q = 0; q < K; q++) acc[r][q] = 0.0;
#pragma unroll
        for (int r = 0; r < R; r++) {
            if (i0 + r >= n) break;                       // warp-uniform: the last group may be short
            const int64_t beg = rowptr[i0 + r], end = rowptr[i0 + r + 1];
            for (int64_t p0 = beg; p0 < end; p0 += 32 * SR) {
                int64_t j[SR];
                double v[SR], xv[SR][K];
#pragma unroll
                for (int u = 0; u < SR; u++) {
                    const int64_t p = p0 + 32 * u + lane;
                    const bool in = p < end;
                    j[u] = in ? (int64_t)__ldg(&col[p]) : -1;
                    v[u] = in ? __ldg(&val[p]) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < SR; u++) {
                    if (j[u] >= 0) {
                        if (INTER && K == 2) {
                            const double2 c2 = __ldg(reinterpret_cast<const double2 *>(x) + j[u]);
                            xv[u][0] = c2.x;
                            xv[u][K - 1] = c2.y;
                        } else {
#pragma unroll
                            for (int q = 0; q < K; q++)
                                xv[u][q] = INTER ? __ldg(&x[j[u] * K + q]) : __ldg(&x[q * n + j[u]]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < K; q++) xv[u][q] = 0.0;
                    }
                }
#pragma unroll
                for (int u = 0; u < SR; u++) {
                    if (p0 + 32 * u < end) {                  // warp-uniform: some lane holds a nonzero
#pragma unroll
                        for (int q = 0; q < K; q++) acc[r][q] = fma(v[u], xv[u][q], acc[r][q]);
                    }
                }
            }
        }
        // butterfly over the group's rows: at level t (lane mask 16 >> t) a lane
        // keeps the upper or lower half of the rows it holds and adds its
        // partner's partial sums of the half it keeps
#pragma unroll
        for (int t = 0; t < LOG_R; t++) {
            const int mask = 16 >> t;
            const int half = R >> (t + 1);
            const bool upper = (lane & mask) != 0;
#pragma unroll
            for (int r = 0; r < half; r++) {
#pragma unroll
                for (int q = 0; q < K; q++) {
                    const double send = upper ? acc[r][q] : acc[r + half][q];
                    const double keep = upper ? acc[r + half][q] : acc[r][q];
                    acc[r][q] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
                }
            }
        }
        // the remaining 5 - log2(R) levels: plain sums over the lanes that hold the same row
#pragma unroll
        for (int mask = 16 >> LOG_R; mask >= 1; mask >>= 1) {
#pragma unroll
            for (int q = 0; q < K; q++) acc[0][q] += __shfl_xor_sync(0xffffffffu, acc[0][q], mask);
        }
        // the row this lane now holds: bit (4 - t) of the lane selects half R >> (t + 1)
        int r_own = 0;
#pragma unroll
        for (int t = 0; t < LOG_R; t++) r_own += ((lane >> (4 - t)) & 1) * (R >> (t + 1));
        const int64_t i = i0 + r_own;
        if ((lane & ((32 >> LOG_R) - 1)) == 0 && i < n) {
            const double d = diag[i];
#pragma unroll
            for (int q = 0; q < K; q++) {
                const int64_t xi = INTER ? i * K + q : q * n + i;
                y[xi] = fma(d, x[xi], acc[0][q]);
            }
        }
    }
}

template <int K, bool INTER>
static void launch_stored(shci_ctx *c, const double *x, double *y) {
    int blocks = c->n_sm * (2048 / SIGMA_THREADS);
    k_sigma_stored<K, INTER><<<blocks, SIGMA_THREADS, 0, c->st>>>(c->n_det, c->rowptr.p, c->col.p, c->val.p,
                                                                 c->diag.p, x, y);
    KERNEL_CHECK();
}

template <bool INTER>
static void dispatch_stored(shci_ctx *c, int k, const double *x, double *y) {
    switch (k) {
        case 1: launch_stored<1, INTER>(c, x, y); break;
        case 2: launch_stored<2, INTER>(c, x, y); break;
        case 3: launch_stored<3, INTER>(c, x, y); break;
        case 4: launch_stored<4, INTER>(c, x, y); break;
        case 5: launch_stored<5, INTER>(c, x, y); break;
        case 6: launch_stored<6, INTER>(c, x, y); break;
        case 7: launch_stored<7, INTER>(c, x, y); break;
        case 8: launch_stored<8, INTER>(c, x, y); break;
        default: throw ShciError{SHCI_ERR_INVALID, "k must be in [1, 8]"};
    }
}

void sigma_otf(shci_ctx *c, int k, const double *x, double *y, bool inter);
void sigma_upper(shci_ctx *c, int k, const double *x, double *y, bool inter);   // sigma_upper.cu

// loads every stored-sigma kernel onto the current device (with lazy module
// loading a kernel's module is otherwise loaded, and device memory taken, at
// its first launch)
template <bool INTER>
static void preload_stored() {
    cudaFuncAttributes fa;
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<1, INTER>));
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<2, INTER>));
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<3, INTER>));
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<4, INTER>));
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<5, INTER>));
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<6, INTER>));
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<7, INTER>));
    CUDA_TRY(cudaFuncGetAttributes(&fa, k_sigma_stored<8, INTER>));
}

void sigma_stored_preload() {
    preload_stored<false>();
    preload_stored<true>();
}

void sigma(shci_ctx *c, int k, const double *x, double *y, bool inter) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before sigma"};
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev0, c->st));
    if (c->mode == SHCI_STORED) {
        if (inter) dispatch_stored<true>(c, k, x, y);
        else dispatch_stored<false>(c, k, x, y);
        g_kernel_launches += 1;
    } else if (c->mode == SHCI_STORED_UPPER) {
        sigma_upper(c, k, x, y, inter);
        g_kernel_launches += 2;
    } else {
        sigma_otf(c, k, x, y, inter);               // its two launches count themselves
    }
    c->stats.sigma_launches += 1;
    c->stats.sigma_vectors += k;
    if (c->timing) {
        CUDA_TRY(cudaEventRecord(c->ev1, c->st));
        CUDA_TRY(cudaEventSynchronize(c->ev1));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        c->stats.sigma_ms_total += ms;
    }
}

// On-the-fly sigma (the "direct" method the paper proposes for larger spaces,
// Sec. VIII): every product re-enumerates the connected pairs with the helper
// lists and recomputes H_ij, so H is never stored.  Pass 1 (rows grouped by
// alpha string) writes y = diag * x + same-spin-beta and opposite-spin terms;
// pass 2 (rows grouped by beta string) adds the same-spin-alpha terms.
template <int W, int K>
static void otf_k(shci_ctx *c, const double *x, double *y) {
    EnumArgs A = enum_args(c);
    A.x = x;
    A.y = y;
    A.diag = c->diag.p;
    DevInts I = dev_ints(c);
    A.accumulate = 0;
    launch_enum<W, ENUM_SIGMA, K>(c, A, I, true);
    A.accumulate = 1;
    launch_enum<W, ENUM_SIGMA, K>(c, A, I, false);
}

template <int W>
static void otf_w(shci_ctx *c, int k, const double *x, double *y) {
    switch (k) {
        case 1: otf_k<W, 1>(c, x, y); break;
        case 2: otf_k<W, 2>(c, x, y); break;
        case 3: otf_k<W, 3>(c, x, y); break;
        case 4: otf_k<W, 4>(c, x, y); break;
        case 5: otf_k<W, 5>(c, x, y); break;
        case 6: otf_k<W, 6>(c, x, y); break;
        case 7: otf_k<W, 7>(c, x, y); break;
        case 8: otf_k<W, 8>(c, x, y); break;
        default: throw ShciError{SHCI_ERR_INVALID, "k must be in [1, 8]"};
    }
}

void sigma_otf(shci_ctx *c, int k, const double *x, double *y, bool inter) {
    if (!inter && k != 1) throw ShciError{SHCI_ERR_INVALID, "on-the-fly sigma takes interleaved vectors"};
    if (c->W == 1) otf_w<1>(c, k, x, y);
    else otf_w<2>(c, k, x, y);
}

}  // namespace shci
