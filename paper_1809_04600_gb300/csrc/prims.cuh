// Device-wide primitives: exclusive scan and a stable LSD radix sort of
// multi-word uint64 keys with uint32 payloads.  Used by the helper-list build.
#pragma once
#include "common.cuh"

namespace shci {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive scan of one value per thread across the block; returns the prefix,
// *total receives the block total
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *total) {
    __shared__ T warp_sums[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? warp_sums[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < nw) warp_sums[lane] = si - s;
        if (lane == nw - 1) warp_sums[32] = si;
    }
    __syncthreads();
    T res = warp_sums[wid] + inc - v;
    *total = warp_sums[32];
    __syncthreads();
    return res;
}

template <typename T>
__global__ void k_scan_reduce(const T *__restrict__ in, int64_t n, T *__restrict__ block_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++)
        if (base + k < n) s += in[base + k];
    T tot;
    block_excl_scan<T>(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// in-place exclusive scan of nb block sums by one block; block_sums[nb] = total
template <typename T>
__global__ void k_scan_blocksums(T *block_sums, int64_t nb) {
    T carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        T v = i < nb ? block_sums[i] : T(0);
        T tot;
        T ex = block_excl_scan<T>(v, &tot);
        if (i < nb) block_sums[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) block_sums[nb] = carry;
}

template <typename T>
__global__ void k_scan_apply(const T *__restrict__ in, int64_t n, const T *__restrict__ block_sums,
                             T *__restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = base + k < n ? in[base + k] : T(0);
        s += v[k];
    }
    T tot;
    T ex = block_excl_scan<T>(s, &tot) + block_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = block_sums[gridDim.x];
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.  `tmp` needs
// ceil(n / SCAN_TILE) + 1 elements.  in and out may alias.
template <typename T>
inline void exclusive_scan(const T *in, T *out, int64_t n, T *tmp, cudaStream_t st) {
    if (n == 0) {
        CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(T), st));
        return;
    }
    int64_t nb = ceil_div(n, SCAN_TILE);
    k_scan_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, tmp);
    k_scan_blocksums<T><<<1, 1024, 0, st>>>(tmp, nb);
    k_scan_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, tmp, out);
    KERNEL_CHECK();
    g_kernel_launches += 3;
}

inline int64_t scan_tmp_len(int64_t n) { return ceil_div(n, SCAN_TILE) + 1; }

// ---------------------------------------------------------------- radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;                       // 32-element rounds per warp
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;    // 2048 elements per tile

template <int KW>
__global__ void k_key_or_and(const uint64_t *__restrict__ keys, int64_t n, unsigned long long *orand) {
    unsigned long long o[KW], a[KW];
#pragma unroll
    for (int w = 0; w < KW; w++) { o[w] = 0; a[w] = ~0ull; }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int w = 0; w < KW; w++) { uint64_t k = keys[i * KW + w]; o[w] |= k; a[w] &= k; }
    }
#pragma unroll
    for (int w = 0; w < KW; w++) {
        atomicOr(&orand[w], o[w]);
        atomicAnd(&orand[KW + w], a[w]);
    }
}

template <int KW>
__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int word, int shift,
                          uint32_t *__restrict__ hist, int64_t n_tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
        int64_t i = base + k;
        if (i < n) atomicAdd(&h[(keys[i * KW + word] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

template <int KW>
__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                             int word, int shift, const uint32_t *__restrict__ offs, int64_t n_tiles) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_ROUNDS);
    uint32_t rank[RS_ROUNDS];
    int dig[RS_ROUNDS];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + r * 32 + lane;
        bool valid = i < n;
        int d = valid ? (int)((kin[i * KW + word] >> shift) & 255u) : 256 + lane;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? wcnt[w][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
        dig[r] = d;
    }
    __syncthreads();
    // exclusive scan across warps of each digit's count
    {
        int d = threadIdx.x;   // RS_THREADS == 256 digits
        uint32_t run = 0;
#pragma unroll
        for (int x = 0; x < RS_WARPS; x++) {
            uint32_t t = wcnt[x][d];
            wcnt[x][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + r * 32 + lane;
        if (i < n) {
            int d = dig[r];
            int64_t pos = (int64_t)offs[(int64_t)d * n_tiles + blockIdx.x] + wcnt[w][d] + rank[r];
#pragma unroll
            for (int q = 0; q < KW; q++) kout[pos * KW + q] = kin[i * KW + q];
            vout[pos] = vin[i];
        }
    }
}

// Workspace for sorting up to n elements with KW-word keys.
struct SortWork {
    DevBuf<uint64_t> keys_alt;
    DevBuf<uint32_t> vals_alt;
    DevBuf<uint32_t> hist;
    DevBuf<uint32_t> scan_tmp;
    DevBuf<unsigned long long> orand;
};

// Stable sort of (keys[n][KW], vals[n]) in place (ping-pong through ws).
// Word 0 is the least significant.  Digits that are equal for every key are
// skipped (found by an OR/AND reduction), so short keys cost few passes.
template <int KW>
inline void radix_sort(uint64_t *keys, uint32_t *vals, int64_t n, SortWork &ws, cudaStream_t st) {
    if (n <= 1) return;
    if (n > 0xFFFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "radix_sort: too many elements"};
    int64_t n_tiles = ceil_div(n, RS_TILE);
    ws.keys_alt.alloc((size_t)n * KW);
    ws.vals_alt.alloc((size_t)n);
    ws.hist.alloc((size_t)(256 * n_tiles + 1));
    ws.scan_tmp.alloc((size_t)scan_tmp_len(256 * n_tiles));
    ws.orand.alloc(2 * KW);
    std::vector<unsigned long long> init(2 * KW);
    for (int w = 0; w < KW; w++) { init[w] = 0ull; init[KW + w] = ~0ull; }
    CUDA_TRY(cudaMemcpyAsync(ws.orand.p, init.data(), sizeof(unsigned long long) * 2 * KW,
                             cudaMemcpyHostToDevice, st));
    k_key_or_and<KW><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(keys, n, ws.orand.p);
    KERNEL_CHECK();
    g_kernel_launches += 1;
    std::vector<unsigned long long> oa(2 * KW);
    CUDA_TRY(cudaMemcpyAsync(oa.data(), ws.orand.p, sizeof(unsigned long long) * 2 * KW,
                             cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    uint64_t *ka = keys, *kb = ws.keys_alt.p;
    uint32_t *va = vals, *vb = ws.vals_alt.p;
    int passes = 0;
    for (int w = 0; w < KW; w++) {
        uint64_t varying = oa[w] ^ oa[KW + w];
        for (int shift = 0; shift < 64; shift += 8) {
            if (((varying >> shift) & 255u) == 0) continue;
            k_rs_hist<KW><<<(unsigned)n_tiles, RS_THREADS, 0, st>>>(ka, n, w, shift, ws.hist.p, n_tiles);
            exclusive_scan<uint32_t>(ws.hist.p, ws.hist.p, 256 * n_tiles, ws.scan_tmp.p, st);
            k_rs_scatter<KW><<<(unsigned)n_tiles, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, w, shift, ws.hist.p,
                                                                       n_tiles);
            KERNEL_CHECK();
            g_kernel_launches += 2;
            std::swap(ka, kb);
            std::swap(va, vb);
            passes++;
        }
    }
    if (ka != keys) {
        CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n * KW, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
}

}  // namespace shci
