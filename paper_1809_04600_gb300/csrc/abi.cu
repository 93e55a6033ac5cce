// extern "C" entry points declared in include/shci.h: argument checks, error
// capture and layout conversion around the internal pipeline.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "context.cuh"


namespace {
thread_local std::string g_create_error;

template <typename F>
int guarded(shci_ctx *c, F &&f) {
    if (!c) return SHCI_ERR_INVALID;
    try {
        int dev = -1;
        cudaGetDevice(&dev);
        if (dev != c->device) CUDA_TRY(cudaSetDevice(c->device));
        c->err.clear();
        int rc = f();
        if (rc == SHCI_ERR_NOT_CONVERGED) c->err = "Davidson did not converge within max_iter";
        return rc;
    } catch (const ShciError &e) {
        c->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        c->err = e.what();
        return SHCI_ERR_INVALID;
    }
}

__global__ void k_transpose(const double *__restrict__ src, int rows, int64_t cols, double *__restrict__ dst) {
    // src [rows][cols] -> dst [cols][rows]
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % rows);
        int64_t c = e / rows;
        dst[e] = src[(int64_t)r * cols + c];
    }
}
}  // namespace

extern "C" {

int shci_create(shci_ctx **out, int device, void *cuda_stream) {
    if (!out) return SHCI_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        g_create_error = "no such CUDA device";
        cudaGetLastError();
        return SHCI_ERR_INVALID;
    }
    shci_ctx *c = new shci_ctx();
    c->device = device;
    try {
        CUDA_TRY(cudaSetDevice(device));
        int sms = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        c->n_sm = sms;
        if (cuda_stream) {
            c->st = (cudaStream_t)cuda_stream;
        } else {
            CUDA_TRY(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        CUDA_TRY(cudaEventCreate(&c->ev0));
        CUDA_TRY(cudaEventCreate(&c->ev1));
        shci::noalloc_prepare(device);
    } catch (const ShciError &e) {
        g_create_error = e.msg;
        delete c;
        return e.code;
    }
    *out = c;
    return SHCI_OK;
}

void shci_destroy(shci_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->st);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
}

const char *shci_last_error(const shci_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int shci_load_integrals(shci_ctx *c, int n_orb, double e_core, const double *h, const double *eri, int mem) {
    return guarded(c, [&] {
        if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
        shci::load_integrals(c, n_orb, e_core, h, eri, mem);
        return SHCI_OK;
    });
}

int shci_build_connectivity(shci_ctx *c, int n_alpha, int n_beta, int64_t n_det, const uint64_t *dets, int mem,
                            int mode, int64_t *nnz_upper_out) {
    return guarded(c, [&] {
        shci::build(c, n_alpha, n_beta, n_det, dets, mem, mode);
        if (nnz_upper_out) *nnz_upper_out = c->nnz_upper;
        return SHCI_OK;
    });
}

int shci_extend_connectivity(shci_ctx *c, int64_t n_new, const uint64_t *new_dets, int mem, double full_fraction,
                             int64_t *nnz_upper_out) {
    return guarded(c, [&] {
        shci::extend(c, n_new, new_dets, mem, full_fraction);
        if (nnz_upper_out) *nnz_upper_out = c->nnz_upper;
        return SHCI_OK;
    });
}

int shci_get_diag(shci_ctx *c, double *diag, int mem) {
    return guarded(c, [&] {
        if (!c->built) throw ShciError{SHCI_ERR_STATE, "not built"};
        if (!diag) throw ShciError{SHCI_ERR_INVALID, "null pointer"};
        CUDA_TRY(cudaMemcpyAsync(diag, c->diag.p, sizeof(double) * c->n_det,
                                 mem == SHCI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
        return SHCI_OK;
    });
}

int shci_get_pairs(shci_ctx *c, int64_t cap, int64_t *i_out, int64_t *j_out, double *hij_out, int64_t *n_out) {
    return guarded(c, [&] {
        shci::export_pairs(c, cap, i_out, j_out, hij_out, n_out);
        return SHCI_OK;
    });
}

int shci_get_row(shci_ctx *c, int64_t row, int64_t cap, int64_t *cols, double *vals, int64_t *n_out) {
    return guarded(c, [&] {
        if (!c->built || c->mode != SHCI_STORED) throw ShciError{SHCI_ERR_STATE, "no stored Hamiltonian"};
        if (row < 0 || row >= c->n_det) throw ShciError{SHCI_ERR_INVALID, "row out of range"};
        int64_t rp[2];
        CUDA_TRY(cudaMemcpyAsync(rp, c->rowptr.p + row, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
        const int64_t len = rp[1] - rp[0];
        if (n_out) *n_out = len;
        if (cap < len) return SHCI_OK;
        if (!cols || !vals) throw ShciError{SHCI_ERR_INVALID, "null output pointer"};
        std::vector<int32_t> cl((size_t)len);
        std::vector<double> vl((size_t)len);
        CUDA_TRY(cudaMemcpyAsync(cl.data(), c->col.p + rp[0], sizeof(int32_t) * len, cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaMemcpyAsync(vl.data(), c->val.p + rp[0], sizeof(double) * len, cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
        std::vector<int64_t> order((size_t)len);
        for (int64_t t = 0; t < len; t++) order[t] = t;
        std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cl[a] < cl[b]; });
        for (int64_t t = 0; t < len; t++) {
            cols[t] = cl[order[t]];
            vals[t] = vl[order[t]];
        }
        return SHCI_OK;
    });
}

int shci_sigma(shci_ctx *c, int k, const double *x, double *y, int mem) {
    return guarded(c, [&] {
        if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before sigma"};
        if (k < 1 || k > SHCI_MAX_K) throw ShciError{SHCI_ERR_INVALID, "k must be in [1, 8]"};
        if (!x || !y) throw ShciError{SHCI_ERR_INVALID, "null vector pointer"};
        if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
        const int64_t n = c->n_det;
        if (mem == SHCI_MEM_DEVICE) {
            const char *xb = (const char *)x, *yb = (const char *)y;
            size_t bytes = sizeof(double) * k * n;
            if (xb < yb + bytes && yb < xb + bytes) throw ShciError{SHCI_ERR_INVALID, "c and sigma overlap"};
        }
        c->vec_a.alloc((size_t)k * n);
        c->vec_b.alloc((size_t)k * n);
        const double *xin = x;
        if (mem == SHCI_MEM_HOST) {
            CUDA_TRY(cudaMemcpyAsync(c->vec_b.p, x, sizeof(double) * k * n, cudaMemcpyHostToDevice, c->st));
            xin = c->vec_b.p;
        }
        if (k == 1) {
            double *yout = mem == SHCI_MEM_HOST ? c->vec_a.p : y;
            shci::sigma(c, 1, xin, yout, false);
            if (mem == SHCI_MEM_HOST)
                CUDA_TRY(cudaMemcpyAsync(y, yout, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
        } else {
            // interleave [k][n] -> [n][k], multiply, de-interleave
            unsigned g = (unsigned)std::min<int64_t>(ceil_div(k * n, 256), 152 * 64);
            k_transpose<<<g, 256, 0, c->st>>>(xin, k, n, c->vec_a.p);
            KERNEL_CHECK();
            double *tmp = c->vec_b.p;   // free again once xin is consumed by the transpose
            shci::sigma(c, k, c->vec_a.p, tmp, true);
            double *yout = mem == SHCI_MEM_HOST ? c->vec_a.p : y;
            k_transpose<<<g, 256, 0, c->st>>>(tmp, (int)n, k, yout);   // [n][k] -> [k][n]
            KERNEL_CHECK();
            g_kernel_launches += 2;
            if (mem == SHCI_MEM_HOST)
                CUDA_TRY(cudaMemcpyAsync(y, yout, sizeof(double) * k * n, cudaMemcpyDeviceToHost, c->st));
        }
        CUDA_TRY(cudaStreamSynchronize(c->st));
        return SHCI_OK;
    });
}

int shci_davidson(shci_ctx *c, int k, double tol, int max_iter, const double *guess, double *energies, double *vecs,
                  int mem, int *iters_out) {
    return guarded(c, [&] { return shci::davidson(c, k, tol, max_iter, guess, energies, vecs, mem, iters_out); });
}

int shci_davidson_history(shci_ctx *c, int cap, double *theta, double *rnorm, double *t_s, int *n_out) {
    return guarded(c, [&] {
        if (cap < 0 || !n_out) throw ShciError{SHCI_ERR_INVALID, "cap must be >= 0 and n_out non-null"};
        const int n = (int)c->hist_t.size(), k = c->hist_k;
        const int w = std::min(cap, n);
        for (int it = 0; it < w; it++) {
            if (t_s) t_s[it] = c->hist_t[it];
            for (int l = 0; l < k; l++) {
                if (theta) theta[it * k + l] = c->hist_theta[(size_t)it * k + l];
                if (rnorm) rnorm[it * k + l] = c->hist_rn[(size_t)it * k + l];
            }
        }
        *n_out = n;
        return SHCI_OK;
    });
}

int shci_select(shci_ctx *c, int k, const double *coef, double eps1, int64_t cap, uint64_t *out, int64_t *n_out,
                int mem) {
    return guarded(c, [&] {
        shci::select_dets(c, k, coef, eps1, cap, out, n_out, mem);
        return SHCI_OK;
    });
}

int shci_pt2(shci_ctx *c, const double *coef, double e_var, double eps2, int n_batches, double *e2,
             int64_t *n_pert, int mem) {
    return guarded(c, [&] {
        shci::pt2(c, coef, e_var, eps2, n_batches, e2, n_pert, mem);
        return SHCI_OK;
    });
}

int shci_alias_draw(shci_ctx *c, const double *coef, int64_t n_draws, uint64_t seed, int64_t *draws, int mem) {
    return guarded(c, [&] {
        shci::alias_draw(c, coef, n_draws, seed, draws, mem);
        return SHCI_OK;
    });
}

int shci_pt2_samples(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_d, int64_t n_d,
                     int n_samples, const int64_t *draws, double *out, int mem, int n_batches, const int *batches) {
    return guarded(c, [&] {
        if (n_batches > 1 && !batches) throw ShciError{SHCI_ERR_INVALID, "batches must be given for n_batches > 1"};
        shci::pt2_samples(c, coef, e_var, eps2, eps2_d, n_d, n_samples, draws, out, mem, n_batches < 1 ? 1 : n_batches,
                          n_batches > 1 ? batches : nullptr);
        return SHCI_OK;
    });
}

int shci_pt2_3step(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_psto, double eps2_dtm,
                   double target, int nb_psto, int nb_sto, int64_t n_d, int n_samples, uint64_t seed,
                   shci_pt2_3step_t *out, int mem) {
    return guarded(c, [&] {
        shci::pt2_3step(c, coef, e_var, eps2, eps2_psto, eps2_dtm, target, nb_psto, nb_sto, n_d, n_samples, seed, out,
                        mem);
        return SHCI_OK;
    });
}

int shci_pt2_semistochastic(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_d, int64_t n_d,
                            int n_samples, uint64_t seed, double *e2, double *e2_err, int mem) {
    return guarded(c, [&] {
        shci::pt2_semistochastic(c, coef, e_var, eps2, eps2_d, n_d, n_samples, seed, e2, e2_err, mem);
        return SHCI_OK;
    });
}

int shci_get_stats(shci_ctx *c, shci_stats_t *out) {
    return guarded(c, [&] {
        if (!out) throw ShciError{SHCI_ERR_INVALID, "null pointer"};
        shci_stats_t s = c->stats;
        s.n_det = c->n_det;
        s.nnz_upper = c->nnz_upper;
        s.n_alpha_strings = c->Ua;
        s.n_beta_strings = c->Ub;
        s.n_alpha_singles = c->n_alpha_singles;
        s.candidates = c->candidates;
        s.kernel_launches = g_kernel_launches.load();
        s.mode = c->mode;
        s.n_words = c->W;
        *out = s;
        return SHCI_OK;
    });
}

int shci_set_timing(shci_ctx *c, int enable) {
    return guarded(c, [&] {
        c->timing = (enable & 1) != 0;
        c->timing_dav = (enable & 2) != 0;
        c->stats.sigma_ms_total = 0.0;
        c->stats.sigma_launches = 0;
        c->stats.sigma_vectors = 0;
        return SHCI_OK;
    });
}

}  // extern "C"
