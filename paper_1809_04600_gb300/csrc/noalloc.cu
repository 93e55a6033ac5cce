// shci_sigma_noalloc: sigma = H c without any device allocation.
//
// The regular shci_sigma converts k > 1 vectors between the caller's
// vector-major layout and the interleaved layout of the sigma kernel through
// buffers the context allocates on first use.  Some callers cannot let a
// library call cudaMalloc: a process whose device memory is already handed
// out to another allocator (a framework's caching pool that reserved nearly
// all of HBM), or a latency-critical loop that must not pay the implicit
// device-wide synchronisation of cudaMalloc/cudaFree.  This entry point keeps
// its layout scratch in one file-scope __device__ array of fixed size instead.
//
// Limits and behaviour:
//  - scratch: SHCI_NOALLOC_MAX_ELEMS doubles per buffer, two buffers (8 MiB in
//    total); every GPU that loads the library holds this array until the
//    process exits.  Calls with k * n_det > SHCI_NOALLOC_MAX_ELEMS return
//    SHCI_ERR_INVALID.
//  - set-up, once per device, with that device current: shci_create looks up
//    the array's device address (cudaGetSymbolAddress) and loads the kernels
//    this call launches (cudaFuncGetAttributes), so that with lazy module
//    loading (CUDA 12's default) the module holding the array is loaded --
//    and its 8 MiB taken -- when a context is created, not inside a call.  If
//    that look-up failed at shci_create, the first call on the device retries
//    it, and that call then loads the module and takes the 8 MiB itself.
//  - the call restores the caller's current device before returning.
//  - every call shares the one array: calls that overlap on the GPU (other
//    streams, other contexts, other host threads) race on it.
//  - nothing in the scratch has to start at zero: each element a call reads
//    was written earlier in the same call.
#include <algorithm>
#include <mutex>

#include "context.cuh"

#define SHCI_NOALLOC_MAX_ELEMS (1 << 19)   // 524,288 doubles = 4 MiB per buffer

namespace {

static __device__ __align__(256) double g_noalloc_scratch[2 * SHCI_NOALLOC_MAX_ELEMS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

// src [rows][cols] -> dst [cols][rows]
__global__ void k_noalloc_transpose(const double *__restrict__ src, int rows, int64_t cols,
                                    double *__restrict__ dst);

// device address of the scratch array on `device` (which must be current);
// the first look-up on a device also loads the kernels the call launches
double *noalloc_scratch(int device) {
    if (device < 0 || device >= kMaxDevices) throw ShciError{SHCI_ERR_INVALID, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw ShciError{SHCI_ERR_CUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") +
                                               cudaGetErrorString(e)};
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_noalloc_transpose);
        if (e != cudaSuccess)
            throw ShciError{SHCI_ERR_CUDA, std::string("loading the noalloc transpose: ") + cudaGetErrorString(e)};
        shci::sigma_stored_preload();
        g_noalloc_ptr[device] = static_cast<double *>(p);
    }
    return g_noalloc_ptr[device];
}

// restores the caller's current device when the call returns
struct DeviceRestore {
    int prev = -1;
    explicit DeviceRestore(int want) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != want) CUDA_TRY(cudaSetDevice(want));
    }
    ~DeviceRestore() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

__global__ void k_noalloc_transpose(const double *__restrict__ src, int rows, int64_t cols,
                                    double *__restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % rows);
        int64_t c = e / rows;
        dst[e] = src[(int64_t)r * cols + c];
    }
}

}  // namespace

namespace shci {

// set-up at context creation (device current); a failure here is left for the
// first call to report
void noalloc_prepare(int device) {
    try {
        noalloc_scratch(device);
    } catch (const ShciError &) {
        cudaGetLastError();
    }
}

}  // namespace shci

extern "C" int shci_sigma_noalloc(shci_ctx *c, int k, const double *x, double *y) {
    if (!c) return SHCI_ERR_INVALID;
    try {
        DeviceRestore on_device(c->device);
        c->err.clear();
        if (!c->built || c->mode != SHCI_STORED)
            throw ShciError{SHCI_ERR_STATE, "shci_sigma_noalloc needs a Hamiltonian built in SHCI_STORED mode"};
        if (k < 1 || k > SHCI_MAX_K) throw ShciError{SHCI_ERR_INVALID, "k must be in [1, 8]"};
        if (!x || !y) throw ShciError{SHCI_ERR_INVALID, "null vector pointer"};
        const int64_t n = c->n_det;
        if ((int64_t)k * n > SHCI_NOALLOC_MAX_ELEMS)
            throw ShciError{SHCI_ERR_INVALID,
                            "k * n_det exceeds the static scratch of shci_sigma_noalloc (524288 elements)"};
        const char *xb = (const char *)x, *yb = (const char *)y;
        const size_t bytes = sizeof(double) * k * n;
        if (xb < yb + bytes && yb < xb + bytes) throw ShciError{SHCI_ERR_INVALID, "c and sigma overlap"};
        double *scratch = noalloc_scratch(c->device);
        if (k == 1) {
            shci::sigma(c, 1, x, y, false);
        } else {
            double *xi = scratch;                              // interleaved input  [n][k]
            double *yi = scratch + SHCI_NOALLOC_MAX_ELEMS;     // interleaved output [n][k]
            unsigned g = (unsigned)std::min<int64_t>(ceil_div((int64_t)k * n, 256), 152 * 64);
            k_noalloc_transpose<<<g, 256, 0, c->st>>>(x, k, n, xi);
            CUDA_TRY(cudaGetLastError());
            shci::sigma(c, k, xi, yi, true);
            k_noalloc_transpose<<<g, 256, 0, c->st>>>(yi, (int)n, k, y);
            CUDA_TRY(cudaGetLastError());
            g_kernel_launches += 2;
        }
        CUDA_TRY(cudaStreamSynchronize(c->st));
        return SHCI_OK;
    } catch (const ShciError &e) {
        c->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        c->err = e.what();
        return SHCI_ERR_INVALID;
    }
}
