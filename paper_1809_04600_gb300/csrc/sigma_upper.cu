// sigma = H c from the upper triangle of H alone (SHCI_STORED_UPPER), the form
// the paper stores (Sec. V, "Hamiltonian Matrix"): each stored pair i < j is
// applied in both directions, the transposed half by FP64 atomic adds into L2.
#include "enum_launch.cuh"

namespace shci {

constexpr int UPPER_THREADS = 256;

// Upper-triangle product: y = diag x first (k_sigma_diag), then a warp per
// group of R consecutive rows; for each stored H_ij (j > i) a lane adds
// H_ij x_j to its row sum and scatters H_ij x_i into y_j with an atomic add,
// and the row sums are added to y_i atomically too (other rows scatter into
// it concurrently).  Summation order varies from run to run.  The FP64 atomics
// bound it (four vectors on the 1e6 heat-bath space: 0.81 of the measured
// atomic rate); the shapes tried (rows per group / nonzeros per lane per step
// / CTAs per SM: 4/4/3, 4/2/4, 2/4/4, 4/4/2) were within 3 % of one another.
#ifndef SHCI_UPPER_R
#define SHCI_UPPER_R 4
#endif
#ifndef SHCI_UPPER_SR
#define SHCI_UPPER_SR 4
#endif
#ifndef SHCI_UPPER_MINB
#define SHCI_UPPER_MINB 3
#endif
template <int K, bool INTER>
struct UpperRows {
    static constexpr int R = K <= 2 ? SHCI_UPPER_R : (K <= 4 ? 2 : 1);
    static constexpr int SR = K <= 2 ? SHCI_UPPER_SR : 2;
    static constexpr int MINB = K <= 2 ? SHCI_UPPER_MINB : 1;
};

template <int K, bool INTER>
__global__ void k_sigma_diag(int64_t n, const double *__restrict__ diag, const double *__restrict__ x,
                             double *__restrict__ y) {
    const int64_t total = n * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = diag[INTER ? e / K : e % n] * x[e];
}

template <int K, bool INTER>
__global__ void __launch_bounds__(UPPER_THREADS, UpperRows<K, INTER>::MINB) k_sigma_upper(
    int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, const double *__restrict__ val,
    const double *__restrict__ x, double *y) {
    constexpr int SR = UpperRows<K, INTER>::SR;
    constexpr int R = UpperRows<K, INTER>::R;
    constexpr int LOG_R = R == 8 ? 3 : (R == 4 ? 2 : (R == 2 ? 1 : 0));
    const int lane = threadIdx.x & 31;
    const int64_t n_groups = (n + R - 1) / R;
    const int64_t warps = (int64_t)gridDim.x * (UPPER_THREADS / 32);
    auto at = [n](int64_t i, int q) { return INTER ? i * K + q : q * n + i; };
    for (int64_t g = ((int64_t)blockIdx.x * UPPER_THREADS + threadIdx.x) >> 5; g < n_groups; g += warps) {
        const int64_t i0 = g * R;
        double acc[R][K];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int q = 0; q < K; q++) acc[r][q] = 0.0;
#pragma unroll
        for (int r = 0; r < R; r++) {
            if (i0 + r >= n) break;                       // warp-uniform: the last group may be short
            const int64_t i = i0 + r;
            const int64_t beg = rowptr[i], end = rowptr[i + 1];
            if (beg == end) continue;
            double xi[K];
#pragma unroll
            for (int q = 0; q < K; q++) xi[q] = __ldg(&x[at(i, q)]);
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
                for (int u = 0; u < SR; u++)
#pragma unroll
                    for (int q = 0; q < K; q++) xv[u][q] = j[u] >= 0 ? __ldg(&x[at(j[u], q)]) : 0.0;
#pragma unroll
                for (int u = 0; u < SR; u++) {
                    if (j[u] >= 0) {
#pragma unroll
                        for (int q = 0; q < K; q++) {
                            acc[r][q] = fma(v[u], xv[u][q], acc[r][q]);
                            atomicAdd(&y[at(j[u], q)], v[u] * xi[q]);
                        }
                    }
                }
            }
        }
        // the butterfly of k_sigma_stored over the group's rows
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
#pragma unroll
        for (int mask = 16 >> LOG_R; mask >= 1; mask >>= 1) {
#pragma unroll
            for (int q = 0; q < K; q++) acc[0][q] += __shfl_xor_sync(0xffffffffu, acc[0][q], mask);
        }
        int r_own = 0;
#pragma unroll
        for (int t = 0; t < LOG_R; t++) r_own += ((lane >> (4 - t)) & 1) * (R >> (t + 1));
        const int64_t i = i0 + r_own;
        if ((lane & ((32 >> LOG_R) - 1)) == 0 && i < n) {
#pragma unroll
            for (int q = 0; q < K; q++)
                if (acc[0][q] != 0.0) atomicAdd(&y[at(i, q)], acc[0][q]);
        }
    }
}

template <int K, bool INTER>
static void launch_upper(shci_ctx *c, const double *x, double *y) {
    const int blocks = c->n_sm * (2048 / UPPER_THREADS);
    k_sigma_diag<K, INTER><<<blocks, UPPER_THREADS, 0, c->st>>>(c->n_det, c->diag.p, x, y);
    k_sigma_upper<K, INTER><<<blocks, UPPER_THREADS, 0, c->st>>>(c->n_det, c->rowptr.p, c->col.p, c->val.p, x, y);
    KERNEL_CHECK();
}

template <bool INTER>
static void dispatch_upper(shci_ctx *c, int k, const double *x, double *y) {
    switch (k) {
        case 1: launch_upper<1, INTER>(c, x, y); break;
        case 2: launch_upper<2, INTER>(c, x, y); break;
        case 3: launch_upper<3, INTER>(c, x, y); break;
        case 4: launch_upper<4, INTER>(c, x, y); break;
        case 5: launch_upper<5, INTER>(c, x, y); break;
        case 6: launch_upper<6, INTER>(c, x, y); break;
        case 7: launch_upper<7, INTER>(c, x, y); break;
        case 8: launch_upper<8, INTER>(c, x, y); break;
        default: throw ShciError{SHCI_ERR_INVALID, "k must be in [1, 8]"};
    }
}

void sigma_upper(shci_ctx *c, int k, const double *x, double *y, bool inter) {
    if (inter) dispatch_upper<true>(c, k, x, y);
    else dispatch_upper<false>(c, k, x, y);
}

}  // namespace shci
