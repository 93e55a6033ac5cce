// Shared device/host definitions of the CUDA library (sm_103a).
#pragma once
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/shci.h"

#include <atomic>
// number of kernels this library has launched (reported by shci_get_stats)
extern std::atomic<long long> g_kernel_launches;

#define SHCI_MAX_ORB 128
#define SHCI_MAX_W 2
#define SHCI_MAX_K 8
#define SHCI_MAX_SUB 64

// ---------------------------------------------------------------- host errors

struct ShciError {
    int code;
    std::string msg;
};

#define CUDA_TRY(expr)                                                              \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            throw ShciError{e_ == cudaErrorMemoryAllocation ? SHCI_ERR_OOM : SHCI_ERR_CUDA, \
                            std::string(#expr) + ": " + cudaGetErrorString(e_)};    \
        }                                                                           \
    } while (0)

#define KERNEL_CHECK() CUDA_TRY(cudaGetLastError())

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- device buffers

// A device allocation owned by the context; freed by reset() or the destructor.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    void reset() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        if (count <= n && p) return;
        reset();
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = sizeof(T);
        CUDA_TRY(cudaMalloc((void **)&p, bytes));
        n = count;
    }
    T *get() const { return p; }
    void swap(DevBuf &o) {
        std::swap(p, o.p);
        std::swap(n, o.n);
    }
};

// ---------------------------------------------------------------- device helpers

// *p += v as a global-memory reduction (no result returned).  For a pointer
// the compiler cannot place in global memory (one read from a struct in
// memory or a struct argument), atomicAdd compiles to a returning atomic that
// waits for L2 (measured in the batched solver: every scatter made a round
// trip, 1.4x slower); red.global does not wait.  p must point to global memory.
__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v) : "memory");
}

__device__ __forceinline__ int popc2(uint64_t a, uint64_t b) { return __popcll(a ^ b); }

template <int W>
struct Str {
    uint64_t w[W];
};

template <int W>
__device__ __forceinline__ int xor_popc(const Str<W> &a, const Str<W> &b) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < W; k++) c += __popcll(a.w[k] ^ b.w[k]);
    return c;
}

template <int W>
__device__ __forceinline__ Str<W> load_str(const uint64_t *base, int64_t idx) {
    Str<W> s;
#pragma unroll
    for (int k = 0; k < W; k++) s.w[k] = base[idx * W + k];
    return s;
}

// index of the lowest set bit of a multi-word string, or -1
template <int W>
__device__ __forceinline__ int lowest_bit(const Str<W> &s) {
#pragma unroll
    for (int k = 0; k < W; k++)
        if (s.w[k]) return 64 * k + __ffsll((long long)s.w[k]) - 1;
    return -1;
}

template <int W>
__device__ __forceinline__ void clear_bit(Str<W> &s, int b) {
    s.w[b >> 6] &= ~(1ull << (b & 63));
}

template <int W>
__device__ __forceinline__ void flip_bit(Str<W> &s, int b) {
    s.w[b >> 6] ^= (1ull << (b & 63));
}

// number of set bits of s strictly between orbitals lo and hi (lo < hi)
template <int W>
__device__ __forceinline__ int bits_between(const Str<W> &s, int lo, int hi) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < W; k++) {
        // bits of word k with global index in (lo, hi)
        int b0 = 64 * k;
        int from = lo + 1 - b0;   // first bit in word
        int to = hi - b0;         // one past last bit in word
        if (from < 0) from = 0;
        if (to > 64) to = 64;
        if (to > from) {
            uint64_t m = (to == 64 ? ~0ull : ((1ull << to) - 1)) & ~((1ull << from) - 1);
            c += __popcll(s.w[k] & m);
        }
    }
    return c;
}

__device__ __forceinline__ double flip_sign(double v, int neg) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(neg & 1) << 63));
}

// ---------------------------------------------------------------- integrals on device

// Packed chemists' two-electron integrals and the one-electron matrix.
struct DevInts {
    const double *h;        // n*n
    const double *eri;      // packed, 8-fold
    const double *jk1;      // [n*n][n]: (pq|kk) - (pk|kq)   (same-spin mean field)
    const double *j1;       // [n*n][n]: (pq|kk)             (opposite-spin mean field)
    const double *jdiag;    // [n][n]:   (kk|ll)
    const double *kdiag;    // [n][n]:   (kl|lk)
    double e_core;
    int n;
};

__device__ __forceinline__ int pair_idx(int p, int q) {
    int a = p > q ? p : q, b = p > q ? q : p;
    return a * (a + 1) / 2 + b;
}

__device__ __forceinline__ double eri_get(const DevInts &I, int p, int q, int r, int s) {
    int a = pair_idx(p, q), b = pair_idx(r, s);
    int hi = a > b ? a : b, lo = a > b ? b : a;
    return __ldg(&I.eri[(int64_t)hi * (hi + 1) / 2 + lo]);
}

// ---------------------------------------------------------------- Slater-Condon (string form)

// <D_i|H|D_j> for two distinct determinants that differ by one or two
// excitations (the caller has screened the pair).  ai/bi: alpha/beta strings
// of D_i; aj/bj of D_j.  Sign convention: alpha creators left of beta
// creators, each ascending, so a single q->p in one spin string has the sign
// of the number of that string's common electrons strictly between p and q,
// and an opposite-spin double is the product of its two single signs.
template <int W>
__device__ __forceinline__ double hij_offdiag(const DevInts &I, const Str<W> &ai, const Str<W> &bi,
                                              const Str<W> &aj, const Str<W> &bj) {
    int na = xor_popc<W>(ai, aj) >> 1;
    int nb = xor_popc<W>(bi, bj) >> 1;
    const int n = I.n;
    if (na + nb == 1) {
        // single excitation within one spin string; 'same' is that string, 'other' the other
        const Str<W> &si = na ? ai : bi;
        const Str<W> &sj = na ? aj : bj;
        const Str<W> &other = na ? bi : ai;
        Str<W> pi, qj, common;
#pragma unroll
        for (int k = 0; k < W; k++) {
            uint64_t d = si.w[k] ^ sj.w[k];
            pi.w[k] = si.w[k] & d;   // particle: in D_i only
            qj.w[k] = sj.w[k] & d;   // hole: in D_j only
            common.w[k] = si.w[k] & sj.w[k];
        }
        int p = lowest_bit<W>(pi), q = lowest_bit<W>(qj);
        int lo = p < q ? p : q, hi = p < q ? q : p;
        int neg = bits_between<W>(common, lo, hi) & 1;
        const double *jk = I.jk1 + (int64_t)(p * n + q) * n;
        const double *jo = I.j1 + (int64_t)(p * n + q) * n;
        double v = __ldg(&I.h[p * n + q]);
#pragma unroll
        for (int k = 0; k < W; k++) {
            uint64_t m = common.w[k];
            while (m) {
                int b = __ffsll((long long)m) - 1;
                m &= m - 1;
                v += __ldg(&jk[64 * k + b]);
            }
            uint64_t o = other.w[k];
            while (o) {
                int b = __ffsll((long long)o) - 1;
                o &= o - 1;
                v += __ldg(&jo[64 * k + b]);
            }
        }
        return flip_sign(v, neg);
    }
    if (na == 1 && nb == 1) {
        Str<W> pa, qa, pb, qb;
#pragma unroll
        for (int k = 0; k < W; k++) {
            uint64_t da = ai.w[k] ^ aj.w[k], db = bi.w[k] ^ bj.w[k];
            pa.w[k] = ai.w[k] & da; qa.w[k] = aj.w[k] & da;
            pb.w[k] = bi.w[k] & db; qb.w[k] = bj.w[k] & db;
        }
        int p = lowest_bit<W>(pa), q = lowest_bit<W>(qa);
        int r = lowest_bit<W>(pb), s = lowest_bit<W>(qb);
        int neg = bits_between<W>(aj, p < q ? p : q, p < q ? q : p) +
                  bits_between<W>(bj, r < s ? r : s, r < s ? s : r);
        return flip_sign(eri_get(I, p, q, r, s), neg);
    }
    // same-spin double: holes q1 < q2 in D_j, particles p1 < p2 in D_i
    const Str<W> &si = na ? ai : bi;
    const Str<W> &sj = na ? aj : bj;
    Str<W> pm, qm;
#pragma unroll
    for (int k = 0; k < W; k++) {
        uint64_t d = si.w[k] ^ sj.w[k];
        pm.w[k] = si.w[k] & d;
        qm.w[k] = sj.w[k] & d;
    }
    int p1 = lowest_bit<W>(pm); clear_bit<W>(pm, p1); int p2 = lowest_bit<W>(pm);
    int q1 = lowest_bit<W>(qm); clear_bit<W>(qm, q1); int q2 = lowest_bit<W>(qm);
    // q1 -> p1 on D_j, then q2 -> p2 on the intermediate string
    int neg = bits_between<W>(sj, p1 < q1 ? p1 : q1, p1 < q1 ? q1 : p1);
    Str<W> x = sj;
    flip_bit<W>(x, q1);
    flip_bit<W>(x, p1);
    neg += bits_between<W>(x, p2 < q2 ? p2 : q2, p2 < q2 ? q2 : p2);
    double v = eri_get(I, p1, q1, p2, q2) - eri_get(I, p1, q2, p2, q1);
    return flip_sign(v, neg);
}

// H_ii
template <int W>
__device__ __forceinline__ double hii(const DevInts &I, const Str<W> &a, const Str<W> &b) {
    const int n = I.n;
    double e = I.e_core;
    int oa[SHCI_MAX_ORB], ob[SHCI_MAX_ORB];
    int na = 0, nb = 0;
#pragma unroll
    for (int k = 0; k < W; k++) {
        uint64_t m = a.w[k];
        while (m) { oa[na++] = 64 * k + __ffsll((long long)m) - 1; m &= m - 1; }
        m = b.w[k];
        while (m) { ob[nb++] = 64 * k + __ffsll((long long)m) - 1; m &= m - 1; }
    }
    for (int x = 0; x < na; x++) {
        int k = oa[x];
        e += __ldg(&I.h[k * n + k]);
        for (int y = x + 1; y < na; y++) {
            int l = oa[y];
            e += __ldg(&I.jdiag[k * n + l]) - __ldg(&I.kdiag[k * n + l]);
        }
        for (int y = 0; y < nb; y++) e += __ldg(&I.jdiag[k * n + ob[y]]);
    }
    for (int x = 0; x < nb; x++) {
        int k = ob[x];
        e += __ldg(&I.h[k * n + k]);
        for (int y = x + 1; y < nb; y++) {
            int l = ob[y];
            e += __ldg(&I.jdiag[k * n + l]) - __ldg(&I.kdiag[k * n + l]);
        }
    }
    return e;
}
