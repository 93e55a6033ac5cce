// Peak-rate microbenchmarks for the roofline of the SHCI kernels on this GPU.
//
// The stored and on-the-fly sigma kernels are bound by FP64 and integer issue,
// not by a dense contraction, so their roofline denominators are measured
// here: the rate of independent FP64 fused multiply-adds and adds, 32-bit
// integer multiply-adds, the XOR + 64-bit popcount pair that screens a
// candidate determinant, FP64 atomic adds to random L2-resident addresses and
// random 8-byte gathers from L2.  Each kernel runs a fixed count of
// independent operations per thread (`chains` independent dependency chains,
// the iteration loop unrolled four times) on a grid of `ctas_per_sm` CTAs per
// SM (256 threads each) and is timed with CUDA events after one warm-up
// launch; the caller takes the best over a few launch shapes.
// Results are only stored when a data-dependent test that never holds in
// practice passes, so the compiler keeps every operation.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int THREADS = 256;
constexpr int CHAINS = 8;                  // independent dependency chains per thread (integer kernels)

template <int CH>
__global__ void k_dfma(int iters, double a, double b, double *sink) {
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = 1e-3 * (threadIdx.x + c);
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; c++) s += x[c];
    if (s == -1.0) sink[blockIdx.x] = s;
}

template <int CH>
__global__ void k_dadd(int iters, double b, double *sink) {
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = 1e-3 * (threadIdx.x + c);
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) x[c] = x[c] + b;
        b = -b;
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; c++) s += x[c];
    if (s == -1.0) sink[blockIdx.x] = s;
}

__global__ void k_imad(int iters, unsigned a, unsigned b, double *sink) {
    unsigned x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = threadIdx.x * 7u + c;
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = x[c] * a + b;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s ^= x[c];
    if (s == 0x9E3779B9u) sink[blockIdx.x] = s;
}

// one "screen" = XOR of two 64-bit words + popcount + accumulate: the core of
// a candidate test
__global__ void k_xorpopc(int iters, unsigned long long key, double *sink) {
    unsigned long long w[CHAINS];
    unsigned acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        w[c] = (unsigned long long)(threadIdx.x + 1) * 0x9E3779B97F4A7C15ull + c;
        acc[c] = 0;
    }
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            acc[c] += __popcll(w[c] ^ key);
            w[c] += key;
        }
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += acc[c];
    if (s == 0xFFFFFFFFu) sink[blockIdx.x] = s;
}

__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// FP64 atomic adds to random addresses of a table that fits in L2
__global__ void k_atomic(int iters, double *table, unsigned long long mask) {
    unsigned long long r = mix(blockIdx.x * (unsigned long long)THREADS + threadIdx.x + 1);
    for (int i = 0; i < iters; i++) {
        r = mix(r + i);
        atomicAdd(&table[r & mask], 1.0);
    }
}

// random 8-byte gathers from a table that fits in L2
__global__ void k_gather(int iters, const double *__restrict__ table, unsigned long long mask, double *sink) {
    unsigned long long r[CHAINS];
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) r[c] = mix(blockIdx.x * (unsigned long long)THREADS * CHAINS + threadIdx.x * CHAINS + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            r[c] = r[c] * 6364136223846793005ull + 1442695040888963407ull;
            s += __ldcg(&table[(r[c] >> 20) & mask]);
        }
    }
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" {

// which: 0 DFMA, 1 DADD, 2 IMAD (32-bit), 3 XOR+POPC (64-bit), 4 FP64 atomic
// add to L2, 5 random 8-byte L2 gather.  chains: 8 or 16 independent chains
// per thread for the FP64 kernels (others use 8).  ops_per_s: operations per
// second (one FMA counts as one operation); ms: the timed launch.  Returns 0
// or a cudaError_t.
int shci_peak_rate(int device, int which, int ctas_per_sm, int chains, double *ops_per_s, double *ms) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = sms * (ctas_per_sm > 0 ? ctas_per_sm : 4);
    double *sink = nullptr, *table = nullptr;
    const unsigned long long table_elems = 1ull << 22;   // 32 MiB: L2-resident
    if ((e = cudaMalloc(&sink, sizeof(double) * grid)) != cudaSuccess) return (int)e;
    if (which >= 4 && (e = cudaMalloc(&table, sizeof(double) * table_elems)) != cudaSuccess) {
        cudaFree(sink);
        return (int)e;
    }
    if (table) cudaMemset(table, 0, sizeof(double) * table_elems);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = which >= 4 ? 4096 : 65536;
    auto launch = [&]() {
        switch (which) {
            case 0:
                if (chains == 16) k_dfma<16><<<grid, THREADS>>>(iters, 0.999999, 1e-7, sink);
                else k_dfma<8><<<grid, THREADS>>>(iters, 0.999999, 1e-7, sink);
                break;
            case 1:
                if (chains == 16) k_dadd<16><<<grid, THREADS>>>(iters, 1e-7, sink);
                else k_dadd<8><<<grid, THREADS>>>(iters, 1e-7, sink);
                break;
            case 2: k_imad<<<grid, THREADS>>>(iters, 1664525u, 1013904223u, sink); break;
            case 3: k_xorpopc<<<grid, THREADS>>>(iters, 0x5851F42D4C957F2Dull, sink); break;
            case 4: k_atomic<<<grid, THREADS>>>(iters, table, table_elems - 1); break;
            default: k_gather<<<grid, THREADS>>>(iters, table, table_elems - 1, sink); break;
        }
    };
    launch();
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    const int ch = (which <= 1 && chains == 16) ? 16 : CHAINS;
    const double per_thread = (which == 4) ? (double)iters : (double)iters * ch;
    *ms = t;
    *ops_per_s = per_thread * THREADS * grid / (t * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (table) cudaFree(table);
    return (int)e;
}

}  // extern "C"
