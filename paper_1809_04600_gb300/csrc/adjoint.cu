// Adjoint of the variational energy: dE/dh_pq and dE/d(pq|rs).
//
// For a normalised real eigenvector c of H, E = c^T H c and, H being linear
// in the integrals, dE/dX = c^T (dH/dX) c (Hellmann-Feynman).  dE/dh_pq is the
// spin-summed one-body density matrix gamma_pq; dE/d(packed slot) is one half
// of the two-body density matrix summed over the index permutations that the
// slot stores.  Nothing is stored: the connected pairs are enumerated again
// (the same kernels as the on-the-fly sigma) and every pair i < j adds
// c_i c_j times the integral coefficients of its Slater-Condon element.
// FP64 atomics go to GRAD_REPLICAS copies of the gradient (chosen by CTA) to
// spread contention, and one reduction sums the copies.
#include <algorithm>

#include "enum_launch.cuh"

namespace shci {

// diagonal: H_ii = E_core + sum_k h_kk n_k + sum_{k<l} [(kk|ll) - delta_spin (kl|lk)]
template <int W>
__global__ void k_grad_diag(const uint64_t *__restrict__ dets, int64_t n, const double *__restrict__ c, int n_orb,
                            double *__restrict__ gdh, double *__restrict__ geri, int64_t geri_len) {
    const int rep = blockIdx.x % GRAD_REPLICAS;
    double *dh = gdh + (int64_t)rep * n_orb * n_orb;
    double *de = geri + rep * geri_len;
    int oa[SHCI_MAX_ORB], ob[SHCI_MAX_ORB];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double w = c[i] * c[i];
        if (w == 0.0) continue;
        int na = 0, nb = 0;
#pragma unroll
        for (int k = 0; k < W; k++) {
            uint64_t m = dets[i * 2 * W + k];
            while (m) { oa[na++] = 64 * k + __ffsll((long long)m) - 1; m &= m - 1; }
            m = dets[i * 2 * W + W + k];
            while (m) { ob[nb++] = 64 * k + __ffsll((long long)m) - 1; m &= m - 1; }
        }
        for (int x = 0; x < na; x++) {
            const int k = oa[x];
            atomicAdd(&dh[k * n_orb + k], w);
            for (int y = x + 1; y < na; y++) {
                const int l = oa[y];
                atomicAdd(&de[eri_slot(k, k, l, l)], w);
                atomicAdd(&de[eri_slot(k, l, l, k)], -w);
            }
            for (int y = 0; y < nb; y++) atomicAdd(&de[eri_slot(k, k, ob[y], ob[y])], w);
        }
        for (int x = 0; x < nb; x++) {
            const int k = ob[x];
            atomicAdd(&dh[k * n_orb + k], w);
            for (int y = x + 1; y < nb; y++) {
                const int l = ob[y];
                atomicAdd(&de[eri_slot(k, k, l, l)], w);
                atomicAdd(&de[eri_slot(k, l, l, k)], -w);
            }
        }
    }
}

// out[e] = scale * sum_r rep[r][e]
__global__ void k_grad_reduce(const double *__restrict__ rep, int64_t len, double scale, double *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll 4
        for (int r = 0; r < GRAD_REPLICAS; r++) s += rep[r * len + e];
        out[e] = scale * s;
    }
}

template <int W>
static void backward_w(shci_ctx *c, const double *cv, double *gdh, double *geri, int64_t eri_len) {
    const int64_t n = c->n_det;
    const unsigned blocks = (unsigned)std::max<int64_t>(GRAD_REPLICAS,
                                                        std::min<int64_t>(ceil_div(n, 128), c->n_sm * 16));
    k_grad_diag<W><<<blocks, 128, 0, c->st>>>(c->dets.p, n, cv, c->n_orb, gdh, geri, eri_len);
    KERNEL_CHECK();
    g_kernel_launches += 1;
    EnumArgs A = enum_args(c);
    A.x = cv;
    A.gdh = gdh;
    A.geri = geri;
    A.geri_len = eri_len;
    DevInts I = dev_ints(c);
    launch_enum<W, ENUM_GRAD, 1>(c, A, I, true);
    launch_enum<W, ENUM_GRAD, 1>(c, A, I, false);
}

void energy_backward(shci_ctx *c, const double *cvec, double scale, double *dh, double *deri, int mem) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before the backward pass"};
    if (!cvec || !dh || !deri) throw ShciError{SHCI_ERR_INVALID, "null pointer"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    const int64_t n = c->n_det;
    const int n_orb = c->n_orb;
    const int64_t n2 = (int64_t)n_orb * n_orb;
    const int64_t npair = (int64_t)n_orb * (n_orb + 1) / 2;
    const int64_t eri_len = npair * (npair + 1) / 2;
    cudaStream_t st = c->st;
    DevBuf<double> rep_dh, rep_eri, cbuf, out_dh, out_eri;
    rep_dh.alloc((size_t)GRAD_REPLICAS * n2);
    rep_eri.alloc((size_t)GRAD_REPLICAS * eri_len);
    CUDA_TRY(cudaMemsetAsync(rep_dh.p, 0, sizeof(double) * GRAD_REPLICAS * n2, st));
    CUDA_TRY(cudaMemsetAsync(rep_eri.p, 0, sizeof(double) * GRAD_REPLICAS * eri_len, st));
    const double *cv = cvec;
    if (mem == SHCI_MEM_HOST) {
        cbuf.alloc((size_t)n);
        CUDA_TRY(cudaMemcpyAsync(cbuf.p, cvec, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        cv = cbuf.p;
    }
    if (c->W == 1) backward_w<1>(c, cv, rep_dh.p, rep_eri.p, eri_len);
    else backward_w<2>(c, cv, rep_dh.p, rep_eri.p, eri_len);
    double *odh = dh, *oeri = deri;
    if (mem == SHCI_MEM_HOST) {
        out_dh.alloc((size_t)n2);
        out_eri.alloc((size_t)eri_len);
        odh = out_dh.p;
        oeri = out_eri.p;
    }
    k_grad_reduce<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n2, 256), 1024)), 256, 0, st>>>(
        rep_dh.p, n2, scale, odh);
    k_grad_reduce<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(eri_len, 256), 4096)), 256, 0, st>>>(
        rep_eri.p, eri_len, scale, oeri);
    KERNEL_CHECK();
    g_kernel_launches += 2;
    if (mem == SHCI_MEM_HOST) {
        CUDA_TRY(cudaMemcpyAsync(dh, odh, sizeof(double) * n2, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(deri, oeri, sizeof(double) * eri_len, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace shci

extern "C" int shci_energy_backward(shci_ctx *c, const double *cvec, double grad_out_scale, double *dE_dh,
                                    double *dE_deri_packed, int mem_space) {
    if (!c) return SHCI_ERR_INVALID;
    try {
        int dev = -1;
        cudaGetDevice(&dev);
        if (dev != c->device) CUDA_TRY(cudaSetDevice(c->device));
        c->err.clear();
        shci::energy_backward(c, cvec, grad_out_scale, dE_dh, dE_deri_packed, mem_space);
        return SHCI_OK;
    } catch (const ShciError &e) {
        c->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        c->err = e.what();
        return SHCI_ERR_INVALID;
    }
}
