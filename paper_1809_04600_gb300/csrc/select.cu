// Heat-bath selection of new determinants (Sec. II.A, Eq. 2): D_a outside V is
// selected when some D_i in V has |H_ai c_i| >= eps1.
//
// Double excitations are found the way the paper describes: for every pair
// of occupied orbitals, the magnitudes of the matrix elements of all double
// excitations from that pair depend only on the four orbitals, so they are
// computed once per set of integrals and stored sorted in decreasing order;
// a determinant walks the list of each of its occupied pairs and stops at
// the first element below eps1 / |c_i|.  Single excitations depend on the
// whole determinant and are evaluated exactly (Slater-Condon) for every
// occupied -> virtual move.  Candidates are written per determinant (count
// pass, scan, fill pass), sorted as multi-word integers, made unique and
// removed when already in V.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "context.cuh"
#include "enumerate.cuh"

namespace shci {

constexpr int SEL_THREADS = 256;

// ---------------------------------------------------------------- sorted double-excitation lists

// Tuple t = ((p n + q) n + r) n + s.  List 0 (same spin): p < q, r < s,
// {r, s} disjoint from {p, q}, magnitude |(pr|qs) - (ps|qr)|.  List 1
// (opposite spin, p and r alpha, q and s beta): r != p, s != q, magnitude
// |(pr|qs)|.  Entries with magnitude 0 never meet eps1 > 0 and are dropped.
__device__ __forceinline__ bool hb_entry(const DevInts &I, int same, int64_t t, int &slot, int &r, int &s,
                                         double &v) {
    const int n = I.n;
    s = (int)(t % n);
    r = (int)((t / n) % n);
    const int q = (int)((t / ((int64_t)n * n)) % n);
    const int p = (int)(t / ((int64_t)n * n * n));
    slot = p * n + q;
    if (same) {
        if (!(p < q && r < s) || r == p || r == q || s == p || s == q) return false;
        v = fabs(eri_get(I, p, r, q, s) - eri_get(I, p, s, q, r));
    } else {
        if (r == p || s == q) return false;
        v = fabs(eri_get(I, p, r, q, s));
    }
    return v > 0.0;
}

// key: slot in the high word, then the magnitude rounded toward zero to FP32
// with its bits inverted (ascending keys = decreasing magnitude); excluded
// tuples get the largest key and sort last
__global__ void k_hb_gen(const DevInts I, int same, int64_t total, uint64_t *__restrict__ keys,
                         uint32_t *__restrict__ vals, unsigned long long *__restrict__ cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int slot, r, s;
        double v;
        vals[t] = (uint32_t)t;
        if (!hb_entry(I, same, t, slot, r, s, v)) {
            keys[t] = ~0ull;
            continue;
        }
        const uint32_t fb = __float_as_uint(__double2float_rz(v));
        keys[t] = ((uint64_t)slot << 32) | (uint64_t)(~fb);
        atomicAdd(&cnt[slot], 1ull);
    }
}

__global__ void k_hb_final(const DevInts I, int same, int64_t n_valid, const uint32_t *__restrict__ vals,
                           uint32_t *__restrict__ rs, double *__restrict__ val, float *__restrict__ kf) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_valid;
         e += (int64_t)gridDim.x * blockDim.x) {
        int slot, r, s;
        double v = 0.0;
        hb_entry(I, same, (int64_t)vals[e], slot, r, s, v);
        rs[e] = (uint32_t)r | ((uint32_t)s << 16);
        val[e] = v;
        kf[e] = __double2float_rz(v);
    }
}

static void build_hb_list(shci_ctx *c, int same, HBList &L) {
    cudaStream_t st = c->st;
    const int n = c->n_orb;
    const int64_t total = (int64_t)n * n * n * n;
    const DevInts I = dev_ints(c);
    DevBuf<uint64_t> keys;
    DevBuf<uint32_t> vals;
    DevBuf<unsigned long long> cnt;
    keys.alloc((size_t)total);
    vals.alloc((size_t)total);
    cnt.alloc((size_t)n * n + 1);
    CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (n * n + 1), st));
    const int blocks = (int)std::min<int64_t>(ceil_div(total, SEL_THREADS), (int64_t)c->n_sm * 16);
    k_hb_gen<<<blocks, SEL_THREADS, 0, st>>>(I, same, total, keys.p, vals.p, cnt.p);
    KERNEL_CHECK();
    g_kernel_launches += 1;
    radix_sort<1>(keys.p, vals.p, total, c->sw, st);
    L.off.alloc((size_t)n * n + 1);
    DevBuf<int64_t> tmp;
    tmp.alloc((size_t)scan_tmp_len(n * n + 1));
    exclusive_scan<int64_t>(reinterpret_cast<const int64_t *>(cnt.p), L.off.p, (int64_t)n * n, tmp.p, st);
    int64_t n_valid = 0;
    CUDA_TRY(cudaMemcpyAsync(&n_valid, L.off.p + (int64_t)n * n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    L.rs.alloc((size_t)std::max<int64_t>(n_valid, 1));
    L.val.alloc((size_t)std::max<int64_t>(n_valid, 1));
    L.kf.alloc((size_t)std::max<int64_t>(n_valid, 1));
    if (n_valid > 0) {
        k_hb_final<<<(int)std::min<int64_t>(ceil_div(n_valid, SEL_THREADS), (int64_t)c->n_sm * 16), SEL_THREADS, 0,
                     st>>>(I, same, n_valid, vals.p, L.rs.p, L.val.p, L.kf.p);
        KERNEL_CHECK();
        g_kernel_launches += 1;
    }
    L.entries = n_valid;
    CUDA_TRY(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- selection kernels

struct SelArgs {
    int64_t n_det;
    const uint64_t *dets;                   // [n][2W]
    int k;
    const double *c;                        // [k][n]
    double eps1;
    int n, na, nb;
    const int64_t *ss_off, *os_off;
    const uint32_t *ss_rs, *os_rs;
    const double *ss_v, *os_v;
    const float *ss_kf, *os_kf;
    unsigned long long *cnt;                // count pass: candidates per determinant
    const int64_t *off;                     // fill pass: first slot of each determinant
    uint64_t *out;                          // fill pass: [total][2W]
    // second-order energy: the terms H_ai c_i of determinants a in hash batch `batch` of `nbatch`
    int nbatch, batch;
    double *terms;                          // fill pass: [total]
    // stochastic estimator (Eq. 9): per sampled determinant w/p and
    // w (n_d - 1) / p - w^2 / p^2; second term and |H_ai c_i| per candidate
    const double *f1, *f2;
    double *terms2, *mags;
};

// batch of a determinant (a SplitMix64-style mix of its words)
template <int W>
__device__ __forceinline__ int det_batch(const Str<W> &a, const Str<W> &b, int nbatch) {
    uint64_t z = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int k = 0; k < 2 * W; k++) {
        z ^= k < W ? a.w[k] : b.w[k - W];
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
    }
    return (int)(z % (uint64_t)nbatch);
}

// orbital of the x-th (0-based) set bit of s
template <int W>
__device__ __forceinline__ int nth_set(const Str<W> &s, int x) {
#pragma unroll
    for (int k = 0; k < W; k++) {
        const int c = __popcll(s.w[k]);
        if (x < c) {
            uint64_t m = s.w[k];
            for (int j = 0; j < x; j++) m &= m - 1;
            return 64 * k + __ffsll((long long)m) - 1;
        }
        x -= c;
    }
    return -1;
}

// orbital of the y-th (0-based) empty orbital below n
template <int W>
__device__ __forceinline__ int nth_unset(const Str<W> &s, int y, int n) {
#pragma unroll
    for (int k = 0; k < W; k++) {
        const int lo = 64 * k;
        if (lo >= n) break;
        const int nb = min(64, n - lo);
        const uint64_t mask = nb == 64 ? ~0ull : ((1ull << nb) - 1);
        uint64_t m = ~s.w[k] & mask;
        const int c = __popcll(m);
        if (y < c) {
            for (int j = 0; j < y; j++) m &= m - 1;
            return lo + __ffsll((long long)m) - 1;
        }
        y -= c;
    }
    return -1;
}

template <int W>
__device__ __forceinline__ bool has_bit(const Str<W> &s, int b) {
    return (s.w[b >> 6] >> (b & 63)) & 1ull;
}

// Above this bound no later entry of a list can meet the threshold: a key is
// the magnitude rounded toward zero to FP32, so the magnitude is below
// key (1 + 2^-23) for normal keys and below FLT_MIN otherwise.
__device__ __forceinline__ double key_bound(float kf) {
    return kf < FLT_MIN ? (double)FLT_MIN : (double)kf * (1.0 + 0x1p-22);
}

// Record a candidate (a, b).  Second-order mode (PT): only determinants of
// the current hash batch, with the term H_ai c_i (signed, exact Slater-Condon).
template <int W, bool FILL, bool PT>
__device__ __forceinline__ void sel_emit(const SelArgs &S, const DevInts &I, unsigned long long &cnt, int64_t base,
                                         unsigned *cursor, const Str<W> &A, const Str<W> &B, double ci,
                                         double f1, double f2, const Str<W> &a, const Str<W> &b) {
    if (PT && S.nbatch > 1 && det_batch<W>(a, b, S.nbatch) != S.batch) return;
    if (!FILL) {
        cnt++;
        return;
    }
    const int64_t pos = base + atomicAdd(cursor, 1u);
    uint64_t *o = S.out + pos * 2 * W;
#pragma unroll
    for (int k = 0; k < W; k++) {
        o[k] = a.w[k];
        o[W + k] = b.w[k];
    }
    if (PT) {
        const double hv = hij_offdiag<W>(I, A, B, a, b);
        if (S.f1) {
            S.terms[pos] = f1 * ci * hv;
            S.terms2[pos] = f2 * ci * ci * hv * hv;
            S.mags[pos] = fabs(hv) * fabs(ci);
        } else {
            S.terms[pos] = hv * ci;
            if (S.mags) S.mags[pos] = fabs(hv) * fabs(ci);
        }
    }
}

// walk one sorted list from slot; `spin` 0: both moves in a (same spin alpha),
// 1: both in b (same spin beta), 2: p -> r in a and q -> s in b
template <int W, bool FILL, bool PT>
__device__ __forceinline__ void sel_walk(const SelArgs &S, const DevInts &I, const int64_t *off, const uint32_t *rs,
                                         const double *val, const float *kf, int slot, int p, int q, int spin,
                                         double cmax, double ci, double f1, double f2, const Str<W> &A,
                                         const Str<W> &B, unsigned long long &cnt, int64_t base, unsigned *cursor) {
    const int64_t e0 = __ldg(&off[slot]), e1 = __ldg(&off[slot + 1]);
    for (int64_t e = e0; e < e1; e++) {
        if (key_bound(__ldg(&kf[e])) * cmax < S.eps1) break;
        const uint32_t x = __ldg(&rs[e]);
        const int r = (int)(x & 0xFFFFu), s = (int)(x >> 16);
        Str<W> a = A, b = B;
        if (spin == 0) {
            if (has_bit(A, r) || has_bit(A, s)) continue;
            flip_bit(a, p); flip_bit(a, q); flip_bit(a, r); flip_bit(a, s);
        } else if (spin == 1) {
            if (has_bit(B, r) || has_bit(B, s)) continue;
            flip_bit(b, p); flip_bit(b, q); flip_bit(b, r); flip_bit(b, s);
        } else {
            if (has_bit(A, r) || has_bit(B, s)) continue;
            flip_bit(a, p); flip_bit(a, r); flip_bit(b, q); flip_bit(b, s);
        }
        if (!(__ldg(&val[e]) * cmax >= S.eps1)) continue;
        sel_emit<W, FILL, PT>(S, I, cnt, base, cursor, A, B, ci, f1, f2, a, b);
    }
}

// One warp per determinant; the lanes share its units of work: every single
// move (alpha then beta) and every occupied pair (alpha-alpha, beta-beta,
// alpha-beta), whose sorted list the lane walks.
template <int W, bool FILL, bool PT>
__global__ void __launch_bounds__(SEL_THREADS) k_select(SelArgs S, DevInts I) {
    __shared__ unsigned cursor[SEL_THREADS / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n = S.n, na = S.na, nb = S.nb;
    const int64_t u_sa = (int64_t)na * (n - na), u_sb = (int64_t)nb * (n - nb);
    const int64_t u_paa = (int64_t)na * (na - 1) / 2, u_pbb = (int64_t)nb * (nb - 1) / 2, u_pab = (int64_t)na * nb;
    const int64_t units = u_sa + u_sb + u_paa + u_pbb + u_pab;
    const int64_t warps = (int64_t)gridDim.x * (SEL_THREADS / 32);
    for (int64_t i = ((int64_t)blockIdx.x * SEL_THREADS + threadIdx.x) >> 5; i < S.n_det; i += warps) {
        double cmax = 0.0, ci = 0.0, f1 = 0.0, f2 = 0.0;
        if (PT) {
            ci = __ldg(&S.c[i]);
            cmax = fabs(ci);
            if (S.f1) {
                f1 = __ldg(&S.f1[i]);
                f2 = __ldg(&S.f2[i]);
            }
        } else {
            for (int l = 0; l < S.k; l++) cmax = fmax(cmax, fabs(__ldg(&S.c[(int64_t)l * S.n_det + i])));
        }
        const Str<W> A = load_str<W>(S.dets, 2 * i), B = load_str<W>(S.dets, 2 * i + 1);
        unsigned long long cnt = 0;
        const int64_t base = FILL ? __ldg(&S.off[i]) : 0;
        if (FILL && lane == 0) cursor[wib] = 0u;
        __syncwarp();
        if (cmax > 0.0) {
            for (int64_t u = lane; u < units; u += 32) {
                int64_t v = u;
                if (v < u_sa + u_sb) {                               // single move p -> r
                    const bool alpha = v < u_sa;
                    if (!alpha) v -= u_sa;
                    const int ne = alpha ? na : nb;
                    const Str<W> &si = alpha ? A : B;
                    const int p = nth_set(si, (int)(v / (n - ne)));
                    const int r = nth_unset(si, (int)(v % (n - ne)), n);
                    Str<W> sj = si;
                    flip_bit(sj, p);
                    flip_bit(sj, r);
                    const double hv = single_exc<W>(I, si, sj, alpha ? B : A);
                    if (!(fabs(hv) * cmax >= S.eps1)) continue;
                    if (alpha) sel_emit<W, FILL, PT>(S, I, cnt, base, &cursor[wib], A, B, ci, f1, f2, sj, B);
                    else sel_emit<W, FILL, PT>(S, I, cnt, base, &cursor[wib], A, B, ci, f1, f2, A, sj);
                    continue;
                }
                v -= u_sa + u_sb;
                if (v < u_paa + u_pbb) {                             // same-spin pair (p < q)
                    const bool alpha = v < u_paa;
                    if (!alpha) v -= u_paa;
                    // pair rank v -> (x < y): y is the largest with y (y - 1) / 2 <= v
                    int y = (int)((1.0 + sqrt(1.0 + 8.0 * (double)v)) * 0.5);
                    while ((int64_t)y * (y - 1) / 2 > v) y--;
                    while ((int64_t)(y + 1) * y / 2 <= v) y++;
                    const int x = (int)(v - (int64_t)y * (y - 1) / 2);
                    const Str<W> &si = alpha ? A : B;
                    const int p = nth_set(si, x), q = nth_set(si, y);
                    sel_walk<W, FILL, PT>(S, I, S.ss_off, S.ss_rs, S.ss_v, S.ss_kf, p * n + q, p, q, alpha ? 0 : 1,
                                          cmax, ci, f1, f2, A, B, cnt, base, &cursor[wib]);
                    continue;
                }
                v -= u_paa + u_pbb;                                  // opposite-spin pair
                const int p = nth_set(A, (int)(v / nb)), q = nth_set(B, (int)(v % nb));
                sel_walk<W, FILL, PT>(S, I, S.os_off, S.os_rs, S.os_v, S.os_kf, p * n + q, p, q, 2, cmax, ci, f1, f2,
                                      A, B, cnt, base, &cursor[wib]);
            }
        }
        if (!FILL) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if (lane == 0) S.cnt[i] = cnt;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- unique, minus V

// lexicographic comparison with the last word most significant
template <int KW>
__device__ __forceinline__ int cmp_words(const uint64_t *a, const uint64_t *b) {
#pragma unroll
    for (int w = KW - 1; w >= 0; w--)
        if (a[w] != b[w]) return a[w] < b[w] ? -1 : 1;
    return 0;
}

// flag[e] = candidate e is the first of its run and not in the sorted V
template <int KW>
__global__ void k_sel_mark(const uint64_t *__restrict__ cand, int64_t total, const uint64_t *__restrict__ vs,
                           int64_t nv, int64_t *__restrict__ flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *x = cand + e * KW;
        int keep = e == 0 || cmp_words<KW>(cand + (e - 1) * KW, x) != 0;
        if (keep) {
            int64_t lo = 0, hi = nv;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (cmp_words<KW>(vs + mid * KW, x) < 0) lo = mid + 1;
                else hi = mid;
            }
            if (lo < nv && cmp_words<KW>(vs + lo * KW, x) == 0) keep = 0;
        }
        flag[e] = keep;
    }
}

template <int KW>
__global__ void k_sel_compact(const uint64_t *__restrict__ cand, int64_t total, const int64_t *__restrict__ pos,
                              uint64_t *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (pos[e + 1] == pos[e]) continue;
#pragma unroll
        for (int w = 0; w < KW; w++) out[pos[e] * KW + w] = cand[e * KW + w];
    }
}

template <int W>
static void select_w(shci_ctx *c, int k, const double *cd, double eps1, DevBuf<uint64_t> &result, int64_t &n_new) {
    cudaStream_t st = c->st;
    constexpr int KW = 2 * W;
    const int64_t n = c->n_det;
    SelArgs S{};
    S.n_det = n;
    S.dets = c->dets.p;
    S.k = k;
    S.c = cd;
    S.eps1 = eps1;
    S.n = c->n_orb;
    S.na = c->n_alpha;
    S.nb = c->n_beta;
    S.ss_off = c->hb_same.off.p;
    S.ss_rs = c->hb_same.rs.p;
    S.ss_v = c->hb_same.val.p;
    S.ss_kf = c->hb_same.kf.p;
    S.os_off = c->hb_opp.off.p;
    S.os_rs = c->hb_opp.rs.p;
    S.os_v = c->hb_opp.val.p;
    S.os_kf = c->hb_opp.kf.p;
    const DevInts I = dev_ints(c);
    const int blocks = c->n_sm * (2048 / SEL_THREADS);
    DevBuf<unsigned long long> cnt;
    cnt.alloc((size_t)n + 1);
    S.cnt = cnt.p;
    k_select<W, false, false><<<blocks, SEL_THREADS, 0, st>>>(S, I);
    KERNEL_CHECK();
    DevBuf<int64_t> off, tmp;
    off.alloc((size_t)n + 1);
    tmp.alloc((size_t)scan_tmp_len(n + 1));
    exclusive_scan<int64_t>(reinterpret_cast<const int64_t *>(cnt.p), off.p, n, tmp.p, st);
    int64_t total = 0;
    CUDA_TRY(cudaMemcpyAsync(&total, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    c->stats.select_candidates = total;
    n_new = 0;
    g_kernel_launches += 1;
    if (total == 0) return;
    if (total > 0xFFFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many candidates: raise eps1"};
    DevBuf<uint64_t> cand;
    cand.alloc((size_t)total * KW);
    S.off = off.p;
    S.out = cand.p;
    k_select<W, true, false><<<blocks, SEL_THREADS, 0, st>>>(S, I);
    KERNEL_CHECK();
    g_kernel_launches += 1;
    DevBuf<uint32_t> dummy;
    dummy.alloc((size_t)std::max(total, n));
    radix_sort<KW>(cand.p, dummy.p, total, c->sw, st);
    // V sorted the same way
    DevBuf<uint64_t> vs;
    vs.alloc((size_t)n * KW);
    CUDA_TRY(cudaMemcpyAsync(vs.p, c->dets.p, sizeof(uint64_t) * n * KW, cudaMemcpyDeviceToDevice, st));
    radix_sort<KW>(vs.p, dummy.p, n, c->sw, st);
    DevBuf<int64_t> flag, pos, tmp2;
    flag.alloc((size_t)total + 1);
    pos.alloc((size_t)total + 1);
    tmp2.alloc((size_t)scan_tmp_len(total + 1));
    const int gb = (int)std::min<int64_t>(ceil_div(total, SEL_THREADS), (int64_t)c->n_sm * 16);
    k_sel_mark<KW><<<gb, SEL_THREADS, 0, st>>>(cand.p, total, vs.p, n, flag.p);
    KERNEL_CHECK();
    exclusive_scan<int64_t>(flag.p, pos.p, total, tmp2.p, st);
    CUDA_TRY(cudaMemcpyAsync(&n_new, pos.p + total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    result.alloc((size_t)std::max<int64_t>(n_new, 1) * KW);
    k_sel_compact<KW><<<gb, SEL_THREADS, 0, st>>>(cand.p, total, pos.p, result.p);
    KERNEL_CHECK();
    g_kernel_launches += 2;
    CUDA_TRY(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- second-order energy

__global__ void k_iota(uint32_t *__restrict__ v, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = (uint32_t)e;
}

// Over the sorted candidates of one batch: for each first entry of a run of
// equal determinants a outside V, num = sum of the run's terms (in generation
// order, i.e. by determinant i of V), and num^2 / (E_V - H_aa); per-block
// sums of the contributions and of the determinants.
template <int W>
__global__ void __launch_bounds__(SEL_THREADS) k_pt_reduce(const uint64_t *__restrict__ cand,
                                                          const uint32_t *__restrict__ idx,
                                                          const double *__restrict__ terms, int64_t total,
                                                          const uint64_t *__restrict__ vs, int64_t nv, DevInts I,
                                                          double e_var, double *__restrict__ part,
                                                          unsigned long long *__restrict__ npart) {
    constexpr int KW = 2 * W;
    double acc = 0.0;
    unsigned long long cnt = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *x = cand + e * KW;
        if (e > 0 && cmp_words<KW>(cand + (e - 1) * KW, x) == 0) continue;
        int64_t lo = 0, hi = nv;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cmp_words<KW>(vs + mid * KW, x) < 0) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nv && cmp_words<KW>(vs + lo * KW, x) == 0) continue;
        double num = 0.0;
        for (int64_t f = e; f < total && cmp_words<KW>(cand + f * KW, x) == 0; f++) num += terms[idx[f]];
        Str<W> a, b;
#pragma unroll
        for (int k = 0; k < W; k++) {
            a.w[k] = x[k];
            b.w[k] = x[W + k];
        }
        acc += num * num / (e_var - hii<W>(I, a, b));
        cnt++;
    }
    __shared__ double red[SEL_THREADS / 32];
    __shared__ unsigned long long redc[SEL_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        red[w] = acc;
        redc[w] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        unsigned long long sc = 0;
        for (int x = 0; x < SEL_THREADS / 32; x++) {
            s += red[x];
            sc += redc[x];
        }
        part[blockIdx.x] = s;
        npart[blockIdx.x] = sc;
    }
}

template <int W>
static double pt2_w(shci_ctx *c, const double *cd, double e_var, double eps2, int nbatch, int64_t &n_pert,
                    int &nbatch_used, int64_t &candidates) {
    cudaStream_t st = c->st;
    constexpr int KW = 2 * W;
    const int64_t n = c->n_det;
    SelArgs S{};
    S.n_det = n;
    S.dets = c->dets.p;
    S.k = 1;
    S.c = cd;
    S.eps1 = eps2;
    S.n = c->n_orb;
    S.na = c->n_alpha;
    S.nb = c->n_beta;
    S.ss_off = c->hb_same.off.p;
    S.ss_rs = c->hb_same.rs.p;
    S.ss_v = c->hb_same.val.p;
    S.ss_kf = c->hb_same.kf.p;
    S.os_off = c->hb_opp.off.p;
    S.os_rs = c->hb_opp.rs.p;
    S.os_v = c->hb_opp.val.p;
    S.os_kf = c->hb_opp.kf.p;
    const DevInts I = dev_ints(c);
    const int blocks = c->n_sm * (2048 / SEL_THREADS);
    DevBuf<unsigned long long> cnt;
    cnt.alloc((size_t)n + 1);
    S.cnt = cnt.p;
    DevBuf<int64_t> off, tmp;
    off.alloc((size_t)n + 1);
    tmp.alloc((size_t)scan_tmp_len(n + 1));
    auto count_pass = [&]() -> int64_t {
        k_select<W, false, true><<<blocks, SEL_THREADS, 0, st>>>(S, I);
        KERNEL_CHECK();
        g_kernel_launches += 1;
        exclusive_scan<int64_t>(reinterpret_cast<const int64_t *>(cnt.p), off.p, n, tmp.p, st);
        int64_t total = 0;
        CUDA_TRY(cudaMemcpyAsync(&total, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return total;
    };
    // batches: enough that one batch's candidates and their sort fit a quarter of free memory
    constexpr double BYTES_PER_CAND = 2.0 * 8 * KW + 8 + 2 * 4;
    if (nbatch <= 0) {
        S.nbatch = 1;
        S.batch = 0;
        const int64_t all = count_pass();
        size_t fr = 0, tot = 0;
        CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        const double budget = 0.25 * (double)fr;
        nbatch = (int)std::max<double>(1.0, std::ceil((double)all * BYTES_PER_CAND / budget));
        nbatch = std::max(nbatch, (int)((all + 0xFFFFFFFEll) / 0xFFFFFFFFll));
    }
    nbatch_used = nbatch;
    // V sorted as multi-word integers
    DevBuf<uint64_t> vs;
    DevBuf<uint32_t> vdummy;
    vs.alloc((size_t)n * KW);
    vdummy.alloc((size_t)n);
    CUDA_TRY(cudaMemcpyAsync(vs.p, c->dets.p, sizeof(uint64_t) * n * KW, cudaMemcpyDeviceToDevice, st));
    radix_sort<KW>(vs.p, vdummy.p, n, c->sw, st);
    const int rblocks = c->n_sm * 4;
    DevBuf<double> part;
    DevBuf<unsigned long long> npart;
    part.alloc((size_t)rblocks);
    npart.alloc((size_t)rblocks);
    std::vector<double> hp(rblocks);
    std::vector<unsigned long long> hn(rblocks);
    double e2 = 0.0;
    n_pert = 0;
    candidates = 0;
    for (int b = 0; b < nbatch; b++) {
        S.nbatch = nbatch;
        S.batch = b;
        const int64_t total = count_pass();
        candidates += total;
        if (total == 0) continue;
        if (total > 0xFFFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many candidates in one batch: more batches"};
        DevBuf<uint64_t> cand;
        DevBuf<double> terms;
        DevBuf<uint32_t> idx;
        cand.alloc((size_t)total * KW);
        terms.alloc((size_t)total);
        idx.alloc((size_t)total);
        S.off = off.p;
        S.out = cand.p;
        S.terms = terms.p;
        k_select<W, true, true><<<blocks, SEL_THREADS, 0, st>>>(S, I);
        KERNEL_CHECK();
        const int gb = (int)std::min<int64_t>(ceil_div(total, SEL_THREADS), (int64_t)c->n_sm * 16);
        k_iota<<<gb, SEL_THREADS, 0, st>>>(idx.p, total);
        KERNEL_CHECK();
        g_kernel_launches += 2;
        radix_sort<KW>(cand.p, idx.p, total, c->sw, st);
        k_pt_reduce<W><<<rblocks, SEL_THREADS, 0, st>>>(cand.p, idx.p, terms.p, total, vs.p, n, I, e_var, part.p,
                                                        npart.p);
        KERNEL_CHECK();
        g_kernel_launches += 1;
        CUDA_TRY(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * rblocks, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(hn.data(), npart.p, sizeof(unsigned long long) * rblocks, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int x = 0; x < rblocks; x++) {
            e2 += hp[x];
            n_pert += (int64_t)hn[x];
        }
    }
    return e2;
}

// ---------------------------------------------------------------- stochastic second-order energy

// sum |c_i| in a fixed order: per-block partials, then one block over them
__global__ void k_abs_partial(const double *__restrict__ c, int64_t n, double *__restrict__ part) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += fabs(c[i]);
    __shared__ double red[SEL_THREADS / 32];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < SEL_THREADS / 32; w++) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_sum_in_order(const double *__restrict__ part, int m, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < m; b++) t += part[b];
    *out = t;
}

// Walker's alias table for p_i = |c_i| / sum (Eq. 10), built by Vose's
// two-list method; one thread, O(n).  small/large: scratch stacks of n.
__global__ void k_alias_table(const double *__restrict__ c, int64_t n, const double *__restrict__ sum,
                              double *__restrict__ prob, int64_t *__restrict__ alias, double *__restrict__ q,
                              int64_t *__restrict__ small, int64_t *__restrict__ large) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double scale = (double)n / *sum;
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; i++) {
        q[i] = fabs(c[i]) * scale;
        alias[i] = i;
        if (q[i] < 1.0) small[ns++] = i;
        else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        const int64_t l = small[--ns], g = large[--nl];
        prob[l] = q[l];
        alias[l] = g;
        q[g] = (q[g] + q[l]) - 1.0;
        if (q[g] < 1.0) small[ns++] = g;
        else large[nl++] = g;
    }
    while (nl > 0) prob[large[--nl]] = 1.0;
    while (ns > 0) prob[small[--ns]] = 1.0;      // rounding leftovers
}

// draw d: r = SplitMix64 output for the counter seed + (d + 1) * golden
// gamma; column = high 32 bits * n >> 32, uniform u = low 32 bits / 2^32;
// the column itself when u < prob[column], else its alias
__global__ void k_alias_draw(const double *__restrict__ prob, const int64_t *__restrict__ alias, int64_t n,
                             uint64_t seed, int64_t n_draws, int64_t *__restrict__ out) {
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < n_draws;
         d += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(d + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const int64_t col = (int64_t)(((z >> 32) * (uint64_t)n) >> 32);
        const double u = (double)(uint32_t)z * 0x1p-32;
        out[d] = u < prob[col] ? col : alias[col];
    }
}

static double abs_sum(shci_ctx *c, const double *cd, int64_t n) {
    cudaStream_t st = c->st;
    const int nb = (int)std::min<int64_t>(ceil_div(n, SEL_THREADS), (int64_t)c->n_sm * 4);
    DevBuf<double> part, tot;
    part.alloc((size_t)nb);
    tot.alloc(1);
    k_abs_partial<<<nb, SEL_THREADS, 0, st>>>(cd, n, part.p);
    k_sum_in_order<<<1, 32, 0, st>>>(part.p, nb, tot.p);
    KERNEL_CHECK();
    g_kernel_launches += 2;
    double h = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&h, tot.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return h;
}

// sample prep: run heads of the sorted draws -> distinct index, count, and the
// per-determinant compact arrays (strings, c_i, w/p, w (n_d - 1)/p - w^2/p^2)
template <int W>
__global__ void k_sample_prep(const uint64_t *__restrict__ sorted, int64_t n_d, const int64_t *__restrict__ pos,
                              const uint64_t *__restrict__ dets, const double *__restrict__ c, double csum,
                              uint64_t *__restrict__ sdets, double *__restrict__ sc, double *__restrict__ f1,
                              double *__restrict__ f2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_d; e += (int64_t)gridDim.x * blockDim.x) {
        if (e > 0 && sorted[e - 1] == sorted[e]) continue;
        int64_t f = e + 1;
        while (f < n_d && sorted[f] == sorted[e]) f++;
        const int64_t i = (int64_t)sorted[e], u = pos[e];
        const double w = (double)(f - e), p = fabs(c[i]) / csum;
#pragma unroll
        for (int k = 0; k < 2 * W; k++) sdets[u * 2 * W + k] = dets[i * 2 * W + k];
        sc[u] = c[i];
        f1[u] = w / p;
        f2[u] = w * (double)(n_d - 1) / p - w * w / (p * p);
    }
}

__global__ void k_run_heads(const uint64_t *__restrict__ sorted, int64_t n, int64_t *__restrict__ flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = (e == 0 || sorted[e - 1] != sorted[e]) ? 1 : 0;
}

// the runs of one sample: (S1^2 + S2) / (E_V - H_aa) at eps2 (all kept terms)
// and at eps2_d (terms with |H_ai c_i| >= eps2_d); per-block partials
template <int W>
__global__ void __launch_bounds__(SEL_THREADS) k_pts_reduce(const uint64_t *__restrict__ cand,
                                                           const uint32_t *__restrict__ idx,
                                                           const double *__restrict__ t1,
                                                           const double *__restrict__ t2,
                                                           const double *__restrict__ mag, int64_t total,
                                                           const uint64_t *__restrict__ vs, int64_t nv, DevInts I,
                                                           double e_var, double eps2_d, double *__restrict__ part) {
    constexpr int KW = 2 * W;
    double acc = 0.0, accd = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *x = cand + e * KW;
        if (e > 0 && cmp_words<KW>(cand + (e - 1) * KW, x) == 0) continue;
        int64_t lo = 0, hi = nv;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cmp_words<KW>(vs + mid * KW, x) < 0) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nv && cmp_words<KW>(vs + lo * KW, x) == 0) continue;
        double s1 = 0.0, s2 = 0.0, s1d = 0.0, s2d = 0.0;
        for (int64_t f = e; f < total && cmp_words<KW>(cand + f * KW, x) == 0; f++) {
            const uint32_t j = idx[f];
            s1 += t1[j];
            s2 += t2[j];
            if (mag[j] >= eps2_d) {
                s1d += t1[j];
                s2d += t2[j];
            }
        }
        Str<W> a, b;
#pragma unroll
        for (int k = 0; k < W; k++) {
            a.w[k] = x[k];
            b.w[k] = x[W + k];
        }
        const double den = e_var - hii<W>(I, a, b);
        acc += (s1 * s1 + s2) / den;
        accd += (s1d * s1d + s2d) / den;
    }
    __shared__ double red[2][SEL_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        accd += __shfl_xor_sync(0xffffffffu, accd, o);
    }
    if (lane == 0) {
        red[0][w] = acc;
        red[1][w] = accd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int x = 0; x < SEL_THREADS / 32; x++) {
            s0 += red[0][x];
            s1 += red[1][x];
        }
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
    }
}

template <int W>
static void pt2_samples_w(shci_ctx *c, const double *cd, double e_var, double eps2, double eps2_d, int64_t n_d,
                          int n_samples, const int64_t *draws, double *out, int nbatch, const int *batch_of_sample) {
    cudaStream_t st = c->st;
    constexpr int KW = 2 * W;
    const int64_t n = c->n_det;
    const double csum = abs_sum(c, cd, n);
    if (!(csum > 0.0)) throw ShciError{SHCI_ERR_INVALID, "all coefficients are zero"};
    DevBuf<uint64_t> vs;
    DevBuf<uint32_t> vdummy;
    vs.alloc((size_t)n * KW);
    vdummy.alloc((size_t)std::max<int64_t>(n, n_d));
    CUDA_TRY(cudaMemcpyAsync(vs.p, c->dets.p, sizeof(uint64_t) * n * KW, cudaMemcpyDeviceToDevice, st));
    radix_sort<KW>(vs.p, vdummy.p, n, c->sw, st);
    const DevInts I = dev_ints(c);
    const int blocks = c->n_sm * (2048 / SEL_THREADS);
    const int rblocks = c->n_sm * 4;
    DevBuf<uint64_t> sorted, sdets;
    DevBuf<int64_t> flag, pos, tmp, off, tmp2;
    DevBuf<double> sc, f1, f2, part;
    DevBuf<unsigned long long> cnt;
    sorted.alloc((size_t)n_d);
    flag.alloc((size_t)n_d + 1);
    pos.alloc((size_t)n_d + 1);
    tmp.alloc((size_t)scan_tmp_len(n_d + 1));
    sdets.alloc((size_t)n_d * KW);
    sc.alloc((size_t)n_d);
    f1.alloc((size_t)n_d);
    f2.alloc((size_t)n_d);
    cnt.alloc((size_t)n_d + 1);
    off.alloc((size_t)n_d + 1);
    tmp2.alloc((size_t)scan_tmp_len(n_d + 1));
    part.alloc((size_t)2 * rblocks);
    std::vector<double> hp(2 * rblocks);
    const int gb = (int)std::min<int64_t>(ceil_div(n_d, SEL_THREADS), (int64_t)c->n_sm * 16);
    for (int smp = 0; smp < n_samples; smp++) {
        CUDA_TRY(cudaMemcpyAsync(sorted.p, draws + (int64_t)smp * n_d, sizeof(int64_t) * n_d,
                                 cudaMemcpyDeviceToDevice, st));
        radix_sort<1>(sorted.p, vdummy.p, n_d, c->sw, st);
        k_run_heads<<<gb, SEL_THREADS, 0, st>>>(sorted.p, n_d, flag.p);
        exclusive_scan<int64_t>(flag.p, pos.p, n_d, tmp.p, st);
        int64_t n_dist = 0;
        CUDA_TRY(cudaMemcpyAsync(&n_dist, pos.p + n_d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        k_sample_prep<W><<<gb, SEL_THREADS, 0, st>>>(sorted.p, n_d, pos.p, c->dets.p, cd, csum, sdets.p, sc.p, f1.p,
                                                     f2.p);
        KERNEL_CHECK();
        g_kernel_launches += 2;
        CUDA_TRY(cudaStreamSynchronize(st));
        SelArgs S{};
        S.n_det = n_dist;
        S.dets = sdets.p;
        S.k = 1;
        S.c = sc.p;
        S.eps1 = eps2;
        S.n = c->n_orb;
        S.na = c->n_alpha;
        S.nb = c->n_beta;
        S.ss_off = c->hb_same.off.p;
        S.ss_rs = c->hb_same.rs.p;
        S.ss_v = c->hb_same.val.p;
        S.ss_kf = c->hb_same.kf.p;
        S.os_off = c->hb_opp.off.p;
        S.os_rs = c->hb_opp.rs.p;
        S.os_v = c->hb_opp.val.p;
        S.os_kf = c->hb_opp.kf.p;
        S.nbatch = nbatch;
        S.batch = batch_of_sample ? batch_of_sample[smp] : 0;
        S.f1 = f1.p;
        S.f2 = f2.p;
        S.cnt = cnt.p;
        k_select<W, false, true><<<blocks, SEL_THREADS, 0, st>>>(S, I);
        KERNEL_CHECK();
        exclusive_scan<int64_t>(reinterpret_cast<const int64_t *>(cnt.p), off.p, n_dist, tmp2.p, st);
        int64_t total = 0;
        CUDA_TRY(cudaMemcpyAsync(&total, off.p + n_dist, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        g_kernel_launches += 1;
        const double norm = 1.0 / ((double)n_d * (double)(n_d - 1));
        if (total == 0) {
            out[2 * smp] = 0.0;
            out[2 * smp + 1] = 0.0;
            continue;
        }
        if (total > 0xFFFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many terms in one sample: raise eps2"};
        DevBuf<uint64_t> cand;
        DevBuf<double> t1, t2, mg;
        DevBuf<uint32_t> idx;
        cand.alloc((size_t)total * KW);
        t1.alloc((size_t)total);
        t2.alloc((size_t)total);
        mg.alloc((size_t)total);
        idx.alloc((size_t)total);
        S.off = off.p;
        S.out = cand.p;
        S.terms = t1.p;
        S.terms2 = t2.p;
        S.mags = mg.p;
        k_select<W, true, true><<<blocks, SEL_THREADS, 0, st>>>(S, I);
        KERNEL_CHECK();
        const int gt = (int)std::min<int64_t>(ceil_div(total, SEL_THREADS), (int64_t)c->n_sm * 16);
        k_iota<<<gt, SEL_THREADS, 0, st>>>(idx.p, total);
        KERNEL_CHECK();
        radix_sort<KW>(cand.p, idx.p, total, c->sw, st);
        k_pts_reduce<W><<<rblocks, SEL_THREADS, 0, st>>>(cand.p, idx.p, t1.p, t2.p, mg.p, total, vs.p, n, I, e_var,
                                                         eps2_d, part.p);
        KERNEL_CHECK();
        g_kernel_launches += 3;
        CUDA_TRY(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * 2 * rblocks, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        double a0 = 0.0, a1 = 0.0;
        for (int x = 0; x < rblocks; x++) {
            a0 += hp[2 * x];
            a1 += hp[2 * x + 1];
        }
        out[2 * smp] = a0 * norm;
        out[2 * smp + 1] = a1 * norm;
    }
}

static void ensure_lists(shci_ctx *c) {
    if (!c->hb_valid) {
        build_hb_list(c, 1, c->hb_same);
        build_hb_list(c, 0, c->hb_opp);
        c->hb_valid = true;
    }
}

void pt2_samples(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_d, int64_t n_d,
                 int n_samples, const int64_t *draws, double *out, int mem, int nbatch, const int *batch_of_sample) {
    if (nbatch < 1 || nbatch > 1 << 20) throw ShciError{SHCI_ERR_INVALID, "n_batches must be in [1, 2^20]"};
    if (batch_of_sample)
        for (int sm = 0; sm < n_samples; sm++)
            if (batch_of_sample[sm] < 0 || batch_of_sample[sm] >= nbatch)
                throw ShciError{SHCI_ERR_INVALID, "batch index out of range"};
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity first"};
    if (!(eps2 > 0.0) || !std::isfinite(eps2) || !(eps2_d >= eps2) || !std::isfinite(eps2_d))
        throw ShciError{SHCI_ERR_INVALID, "need 0 < eps2 <= eps2_d, finite"};
    if (!std::isfinite(e_var)) throw ShciError{SHCI_ERR_INVALID, "e_var must be finite"};
    if (n_d < 2 || n_samples < 1 || !coef || !draws || !out) throw ShciError{SHCI_ERR_INVALID, "bad sample arguments"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    if (c->n_orb > 128) throw ShciError{SHCI_ERR_INVALID, "up to 128 orbitals"};
    cudaStream_t st = c->st;
    ensure_lists(c);
    const int64_t n = c->n_det;
    const double *cd = coef;
    const int64_t *dd = draws;
    DevBuf<double> cbuf;
    DevBuf<int64_t> dbuf;
    if (mem == SHCI_MEM_HOST) {
        cbuf.alloc((size_t)n);
        CUDA_TRY(cudaMemcpyAsync(cbuf.p, coef, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        cd = cbuf.p;
        dbuf.alloc((size_t)n_samples * n_d);
        CUDA_TRY(cudaMemcpyAsync(dbuf.p, draws, sizeof(int64_t) * n_samples * n_d, cudaMemcpyHostToDevice, st));
        dd = dbuf.p;
    }
    // every draw must index a determinant of V with a nonzero coefficient
    {
        std::vector<int64_t> hd((size_t)n_samples * n_d);
        std::vector<double> hc((size_t)n);
        CUDA_TRY(cudaMemcpyAsync(hd.data(), dd, sizeof(int64_t) * hd.size(), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(hc.data(), cd, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t v : hd)
            if (v < 0 || v >= n || hc[(size_t)v] == 0.0)
                throw ShciError{SHCI_ERR_INVALID, "a draw is out of range or has a zero coefficient"};
    }
    std::vector<double> res((size_t)2 * n_samples);
    if (c->W == 1) pt2_samples_w<1>(c, cd, e_var, eps2, eps2_d, n_d, n_samples, dd, res.data(), nbatch, batch_of_sample);
    else pt2_samples_w<2>(c, cd, e_var, eps2, eps2_d, n_d, n_samples, dd, res.data(), nbatch, batch_of_sample);
    for (size_t e = 0; e < res.size(); e++) out[e] = res[e];
}

void alias_draw(shci_ctx *c, const double *coef, int64_t n_draws, uint64_t seed, int64_t *out, int mem) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity first"};
    if (n_draws < 0 || !coef || (n_draws > 0 && !out)) throw ShciError{SHCI_ERR_INVALID, "bad draw arguments"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    cudaStream_t st = c->st;
    const int64_t n = c->n_det;
    if (n > 0xFFFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many determinants for the sampler"};
    const double *cd = coef;
    DevBuf<double> cbuf;
    if (mem == SHCI_MEM_HOST) {
        cbuf.alloc((size_t)n);
        CUDA_TRY(cudaMemcpyAsync(cbuf.p, coef, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        cd = cbuf.p;
    }
    const double csum = abs_sum(c, cd, n);
    if (!(csum > 0.0)) throw ShciError{SHCI_ERR_INVALID, "all coefficients are zero"};
    DevBuf<double> prob, q, sum;
    DevBuf<int64_t> alias, small, large, obuf;
    prob.alloc((size_t)n);
    q.alloc((size_t)n);
    sum.alloc(1);
    alias.alloc((size_t)n);
    small.alloc((size_t)n);
    large.alloc((size_t)n);
    CUDA_TRY(cudaMemcpyAsync(sum.p, &csum, sizeof(double), cudaMemcpyHostToDevice, st));
    k_alias_table<<<1, 32, 0, st>>>(cd, n, sum.p, prob.p, alias.p, q.p, small.p, large.p);
    KERNEL_CHECK();
    g_kernel_launches += 1;
    if (n_draws == 0) return;
    int64_t *o = out;
    if (mem == SHCI_MEM_HOST) {
        obuf.alloc((size_t)n_draws);
        o = obuf.p;
    }
    const int gb = (int)std::min<int64_t>(ceil_div(n_draws, SEL_THREADS), (int64_t)c->n_sm * 16);
    k_alias_draw<<<gb, SEL_THREADS, 0, st>>>(prob.p, alias.p, n, seed, n_draws, o);
    KERNEL_CHECK();
    g_kernel_launches += 1;
    if (mem == SHCI_MEM_HOST)
        CUDA_TRY(cudaMemcpyAsync(out, o, sizeof(int64_t) * n_draws, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
}

void pt2(shci_ctx *c, const double *coef, double e_var, double eps2, int nbatch, double *e2, int64_t *n_pert,
         int mem) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before the second-order energy"};
    if (!(eps2 > 0.0) || !std::isfinite(eps2)) throw ShciError{SHCI_ERR_INVALID, "eps2 must be positive and finite"};
    if (!std::isfinite(e_var)) throw ShciError{SHCI_ERR_INVALID, "e_var must be finite"};
    if (!coef || !e2) throw ShciError{SHCI_ERR_INVALID, "null pointer"};
    if (nbatch < 0 || nbatch > 1 << 20) throw ShciError{SHCI_ERR_INVALID, "n_batches must be in [0, 2^20]"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    if (c->n_orb > 128) throw ShciError{SHCI_ERR_INVALID, "up to 128 orbitals"};
    cudaStream_t st = c->st;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e0, st));
    ensure_lists(c);
    const double *cd = coef;
    DevBuf<double> cbuf;
    if (mem == SHCI_MEM_HOST) {
        cbuf.alloc((size_t)c->n_det);
        CUDA_TRY(cudaMemcpyAsync(cbuf.p, coef, sizeof(double) * c->n_det, cudaMemcpyHostToDevice, st));
        cd = cbuf.p;
    }
    int64_t np = 0, cands = 0;
    int used = 0;
    const double v = c->W == 1 ? pt2_w<1>(c, cd, e_var, eps2, nbatch, np, used, cands)
                               : pt2_w<2>(c, cd, e_var, eps2, nbatch, np, used, cands);
    *e2 = v;
    if (n_pert) *n_pert = np;
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->stats.pt2_ms = ms;
    c->stats.pt2_batches = used;
    c->stats.pt2_terms = cands;
}

// pseudo-stochastic step: over the sorted terms of one batch at eps2_psto, for
// each determinant a outside V the correction
//   (num_psto^2 - num_dtm^2) / (E_V - H_aa),
// num_dtm summing only the terms with |H_ai c_i| >= eps2_dtm; per-block sums of
// the corrections, of their squares and the number of determinants
template <int W>
__global__ void __launch_bounds__(SEL_THREADS) k_psto_reduce(const uint64_t *__restrict__ cand,
                                                            const uint32_t *__restrict__ idx,
                                                            const double *__restrict__ t,
                                                            const double *__restrict__ mag, int64_t total,
                                                            const uint64_t *__restrict__ vs, int64_t nv, DevInts I,
                                                            double e_var, double eps_dtm, double *__restrict__ part,
                                                            unsigned long long *__restrict__ npart) {
    constexpr int KW = 2 * W;
    double acc = 0.0, acc2 = 0.0;
    unsigned long long cnt = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t *x = cand + e * KW;
        if (e > 0 && cmp_words<KW>(cand + (e - 1) * KW, x) == 0) continue;
        int64_t lo = 0, hi = nv;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cmp_words<KW>(vs + mid * KW, x) < 0) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nv && cmp_words<KW>(vs + lo * KW, x) == 0) continue;
        double na = 0.0, nd = 0.0;
        for (int64_t f = e; f < total && cmp_words<KW>(cand + f * KW, x) == 0; f++) {
            const uint32_t j = idx[f];
            na += t[j];
            if (mag[j] >= eps_dtm) nd += t[j];
        }
        Str<W> a, b;
#pragma unroll
        for (int k = 0; k < W; k++) {
            a.w[k] = x[k];
            b.w[k] = x[W + k];
        }
        const double corr = (na * na - nd * nd) / (e_var - hii<W>(I, a, b));
        acc += corr;
        acc2 += corr * corr;
        cnt++;
    }
    __shared__ double red[2][SEL_THREADS / 32];
    __shared__ unsigned long long redc[SEL_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        red[0][w] = acc;
        red[1][w] = acc2;
        redc[w] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        unsigned long long sc = 0;
        for (int x = 0; x < SEL_THREADS / 32; x++) {
            s0 += red[0][x];
            s1 += red[1][x];
            sc += redc[x];
        }
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
        npart[blockIdx.x] = sc;
    }
}

// Pseudo-stochastic step of the 3-step scheme: batches of the perturbative
// determinants (hash partition, at least 16) in order; after each batch the
// corrections seen so far give a mean and variance, the number of
// perturbative determinants is extrapolated from the batches done, and the
// loop stops when the standard deviation of the estimated sum of the
// unevaluated ones is below 0.4 target (all batches: exact, zero deviation).
template <int W>
static void psto_w(shci_ctx *c, const double *cd, double e_var, double eps_psto, double eps_dtm, int nbatch,
                   double target, double &est, double &err, int &done) {
    cudaStream_t st = c->st;
    constexpr int KW = 2 * W;
    const int64_t n = c->n_det;
    SelArgs S{};
    S.n_det = n;
    S.dets = c->dets.p;
    S.k = 1;
    S.c = cd;
    S.eps1 = eps_psto;
    S.n = c->n_orb;
    S.na = c->n_alpha;
    S.nb = c->n_beta;
    S.ss_off = c->hb_same.off.p;
    S.ss_rs = c->hb_same.rs.p;
    S.ss_v = c->hb_same.val.p;
    S.ss_kf = c->hb_same.kf.p;
    S.os_off = c->hb_opp.off.p;
    S.os_rs = c->hb_opp.rs.p;
    S.os_v = c->hb_opp.val.p;
    S.os_kf = c->hb_opp.kf.p;
    S.nbatch = nbatch;
    const DevInts I = dev_ints(c);
    const int blocks = c->n_sm * (2048 / SEL_THREADS);
    const int rblocks = c->n_sm * 4;
    DevBuf<unsigned long long> cnt, npart;
    DevBuf<int64_t> off, tmp;
    DevBuf<double> part;
    cnt.alloc((size_t)n + 1);
    off.alloc((size_t)n + 1);
    tmp.alloc((size_t)scan_tmp_len(n + 1));
    part.alloc((size_t)2 * rblocks);
    npart.alloc((size_t)rblocks);
    S.cnt = cnt.p;
    DevBuf<uint64_t> vs;
    DevBuf<uint32_t> vdummy;
    vs.alloc((size_t)n * KW);
    vdummy.alloc((size_t)n);
    CUDA_TRY(cudaMemcpyAsync(vs.p, c->dets.p, sizeof(uint64_t) * n * KW, cudaMemcpyDeviceToDevice, st));
    radix_sort<KW>(vs.p, vdummy.p, n, c->sw, st);
    std::vector<double> hp(2 * rblocks);
    std::vector<unsigned long long> hn(rblocks);
    double sum = 0.0, sum2 = 0.0;
    int64_t count = 0;
    est = 0.0;
    err = 0.0;
    done = 0;
    for (int b = 0; b < nbatch; b++) {
        S.batch = b;
        k_select<W, false, true><<<blocks, SEL_THREADS, 0, st>>>(S, I);
        KERNEL_CHECK();
        exclusive_scan<int64_t>(reinterpret_cast<const int64_t *>(cnt.p), off.p, n, tmp.p, st);
        int64_t total = 0;
        CUDA_TRY(cudaMemcpyAsync(&total, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        g_kernel_launches += 1;
        if (total > 0xFFFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many terms in one batch: more batches"};
        if (total > 0) {
            DevBuf<uint64_t> cand;
            DevBuf<double> t, mg;
            DevBuf<uint32_t> idx;
            cand.alloc((size_t)total * KW);
            t.alloc((size_t)total);
            mg.alloc((size_t)total);
            idx.alloc((size_t)total);
            S.off = off.p;
            S.out = cand.p;
            S.terms = t.p;
            S.mags = mg.p;
            k_select<W, true, true><<<blocks, SEL_THREADS, 0, st>>>(S, I);
            KERNEL_CHECK();
            const int gt = (int)std::min<int64_t>(ceil_div(total, SEL_THREADS), (int64_t)c->n_sm * 16);
            k_iota<<<gt, SEL_THREADS, 0, st>>>(idx.p, total);
            KERNEL_CHECK();
            radix_sort<KW>(cand.p, idx.p, total, c->sw, st);
            k_psto_reduce<W><<<rblocks, SEL_THREADS, 0, st>>>(cand.p, idx.p, t.p, mg.p, total, vs.p, n, I, e_var,
                                                              eps_dtm, part.p, npart.p);
            KERNEL_CHECK();
            g_kernel_launches += 3;
            CUDA_TRY(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * 2 * rblocks, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaMemcpyAsync(hn.data(), npart.p, sizeof(unsigned long long) * rblocks,
                                     cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            for (int x = 0; x < rblocks; x++) {
                sum += hp[2 * x];
                sum2 += hp[2 * x + 1];
                count += (int64_t)hn[x];
            }
            S.mags = nullptr;
        }
        done = b + 1;
        if (done == nbatch) {
            est = sum;
            err = 0.0;
            break;
        }
        const double n_est = (double)count * nbatch / done;             // perturbative determinants, all batches
        const double rest = n_est - (double)count;
        const double mean = count > 0 ? sum / count : 0.0;
        const double var = count > 1 ? std::max(0.0, (sum2 - count * mean * mean) / (count - 1)) : 0.0;
        est = sum + mean * rest;
        err = std::sqrt(var * rest);
        if (count > 1 && err < 0.4 * target) break;
    }
}

void pt2_3step(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_psto, double eps2_dtm,
               double target, int nbatch_psto, int nbatch_sto, int64_t n_d, int n_samples, uint64_t seed,
               shci_pt2_3step_t *out, int mem) {
    if (!out) throw ShciError{SHCI_ERR_INVALID, "null pointer"};
    if (!(eps2 > 0.0 && eps2 <= eps2_psto && eps2_psto <= eps2_dtm) || !std::isfinite(eps2_dtm))
        throw ShciError{SHCI_ERR_INVALID, "need 0 < eps2 <= eps2_psto <= eps2_dtm, finite"};
    if (!(target >= 0.0)) throw ShciError{SHCI_ERR_INVALID, "target error must be >= 0"};
    if (nbatch_psto < 16 || nbatch_psto > 1 << 20 || nbatch_sto < 1 || nbatch_sto > 1 << 20)
        throw ShciError{SHCI_ERR_INVALID, "need 16 <= pseudo-stochastic batches and 1 <= stochastic batches"};
    if (n_samples < 1 || n_d < 2) throw ShciError{SHCI_ERR_INVALID, "need n_samples >= 1 and n_d >= 2"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    cudaStream_t st = c->st;
    const double *cd = coef;
    DevBuf<double> cbuf;
    if (mem == SHCI_MEM_HOST) {
        cbuf.alloc((size_t)c->n_det);
        CUDA_TRY(cudaMemcpyAsync(cbuf.p, coef, sizeof(double) * c->n_det, cudaMemcpyHostToDevice, st));
        cd = cbuf.p;
    }
    *out = shci_pt2_3step_t{};
    // 1: deterministic at eps2_dtm (hash batches as memory requires)
    pt2(c, cd, e_var, eps2_dtm, 0, &out->dtm, nullptr, SHCI_MEM_DEVICE);
    // 2: pseudo-stochastic at eps2_psto, minus its eps2_dtm part
    ensure_lists(c);
    if (eps2_psto < eps2_dtm) {
        if (c->W == 1) psto_w<1>(c, cd, e_var, eps2_psto, eps2_dtm, nbatch_psto, target, out->psto, out->psto_err,
                                 out->psto_batches);
        else psto_w<2>(c, cd, e_var, eps2_psto, eps2_dtm, nbatch_psto, target, out->psto, out->psto_err,
                       out->psto_batches);
    }
    // 3: stochastic at eps2, minus its eps2_psto part; one batch per sample, drawn
    // from the SplitMix64 stream after the determinant draws, times the batch count
    if (eps2 < eps2_psto) {
        DevBuf<int64_t> draws;
        draws.alloc((size_t)n_samples * n_d);
        alias_draw(c, cd, (int64_t)n_samples * n_d, seed, draws.p, SHCI_MEM_DEVICE);
        std::vector<int> bsel(n_samples);
        for (int sm = 0; sm < n_samples; sm++) {
            uint64_t z = seed + (uint64_t)((int64_t)n_samples * n_d + sm + 1) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            bsel[sm] = (int)(((z >> 32) * (uint64_t)nbatch_sto) >> 32);
        }
        std::vector<double> v((size_t)2 * n_samples);
        pt2_samples(c, cd, e_var, eps2, eps2_psto, n_d, n_samples, draws.p, v.data(), SHCI_MEM_DEVICE, nbatch_sto,
                    bsel.data());
        double mean = 0.0;
        for (int sm = 0; sm < n_samples; sm++) mean += nbatch_sto * (v[2 * sm] - v[2 * sm + 1]);
        mean /= n_samples;
        double var = 0.0;
        for (int sm = 0; sm < n_samples; sm++) {
            const double d = nbatch_sto * (v[2 * sm] - v[2 * sm + 1]) - mean;
            var += d * d;
        }
        out->sto = mean;
        out->sto_err = n_samples > 1 ? std::sqrt(var / (n_samples - 1) / n_samples) : 0.0;
    }
    out->e2 = out->dtm + out->psto + out->sto;
    out->e2_err = std::sqrt(out->psto_err * out->psto_err + out->sto_err * out->sto_err);
}

void pt2_semistochastic(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_d, int64_t n_d,
                        int n_samples, uint64_t seed, double *e2, double *e2_err, int mem) {
    if (!e2) throw ShciError{SHCI_ERR_INVALID, "null pointer"};
    if (n_samples < 1 || n_d < 2) throw ShciError{SHCI_ERR_INVALID, "need n_samples >= 1 and n_d >= 2"};
    // deterministic part at eps2_d (Eq. 8)
    double e2d = 0.0;
    pt2(c, coef, e_var, eps2_d, 0, &e2d, nullptr, mem);
    // stochastic part: the same samples at eps2 and at eps2_d (Eq. 9)
    DevBuf<int64_t> draws;
    draws.alloc((size_t)n_samples * n_d);
    const double *cd = coef;
    DevBuf<double> cbuf;
    if (mem == SHCI_MEM_HOST) {
        cbuf.alloc((size_t)c->n_det);
        CUDA_TRY(cudaMemcpyAsync(cbuf.p, coef, sizeof(double) * c->n_det, cudaMemcpyHostToDevice, c->st));
        cd = cbuf.p;
    }
    alias_draw(c, cd, (int64_t)n_samples * n_d, seed, draws.p, SHCI_MEM_DEVICE);
    std::vector<double> v((size_t)2 * n_samples);
    pt2_samples(c, cd, e_var, eps2, eps2_d, n_d, n_samples, draws.p, v.data(), SHCI_MEM_DEVICE, 1, nullptr);
    double mean = 0.0;
    for (int sm = 0; sm < n_samples; sm++) mean += v[2 * sm] - v[2 * sm + 1];
    mean /= n_samples;
    double var = 0.0;
    for (int sm = 0; sm < n_samples; sm++) {
        const double d = v[2 * sm] - v[2 * sm + 1] - mean;
        var += d * d;
    }
    *e2 = e2d + mean;
    if (e2_err) *e2_err = n_samples > 1 ? std::sqrt(var / (n_samples - 1) / n_samples) : 0.0;
}

void select_dets(shci_ctx *c, int k, const double *coef, double eps1, int64_t cap, uint64_t *out, int64_t *n_out,
                 int mem) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before selecting"};
    if (k < 1 || k > SHCI_MAX_K) throw ShciError{SHCI_ERR_INVALID, "k must be in [1, 8]"};
    if (!(eps1 > 0.0) || !std::isfinite(eps1)) throw ShciError{SHCI_ERR_INVALID, "eps1 must be positive and finite"};
    if (!coef || !n_out) throw ShciError{SHCI_ERR_INVALID, "null pointer"};
    if (cap < 0) throw ShciError{SHCI_ERR_INVALID, "cap must be >= 0"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    if (c->n_orb > 128) throw ShciError{SHCI_ERR_INVALID, "selection supports up to 128 orbitals"};
    cudaStream_t st = c->st;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e0, st));
    if (!c->hb_valid) {
        build_hb_list(c, 1, c->hb_same);
        build_hb_list(c, 0, c->hb_opp);
        c->hb_valid = true;
    }
    const double *cd = coef;
    DevBuf<double> cbuf;
    if (mem == SHCI_MEM_HOST) {
        cbuf.alloc((size_t)k * c->n_det);
        CUDA_TRY(cudaMemcpyAsync(cbuf.p, coef, sizeof(double) * k * c->n_det, cudaMemcpyHostToDevice, st));
        cd = cbuf.p;
    }
    DevBuf<uint64_t> result;
    int64_t n_new = 0;
    if (c->W == 1) select_w<1>(c, k, cd, eps1, result, n_new);
    else select_w<2>(c, k, cd, eps1, result, n_new);
    *n_out = n_new;
    const int KW = 2 * c->W;
    if (n_new > 0 && cap > 0) {
        if (!out) throw ShciError{SHCI_ERR_INVALID, "null output pointer"};
        const int64_t m = std::min(cap, n_new);
        CUDA_TRY(cudaMemcpyAsync(out, result.p, sizeof(uint64_t) * m * KW,
                                 mem == SHCI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    }
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->stats.select_ms = ms;
}

}  // namespace shci
