// Integrals, helper lists (Table I), the cached diagonal and the stored
// Hamiltonian (Sec. III).  Every connected pair is found by screening
// candidates with XOR/popcount in warp-wide rounds and written, with its
// Slater-Condon value, into both rows of a symmetric sparse matrix.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <numeric>

#include "enum_launch.cuh"

std::atomic<long long> g_kernel_launches{0};
#define LAUNCHED(n) (g_kernel_launches += (n))

namespace shci {

// ====================================================================== integrals

__global__ void k_mean_field_tables(const double *__restrict__ eri, int n, double *__restrict__ jk1,
                                    double *__restrict__ j1, double *__restrict__ jdiag,
                                    double *__restrict__ kdiag) {
    DevInts I{};
    I.eri = eri;
    I.n = n;
    int64_t total = (int64_t)n * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(t % n);
        int q = (int)((t / n) % n);
        int p = (int)(t / ((int64_t)n * n));
        double j = eri_get(I, p, q, k, k);
        double x = eri_get(I, p, k, k, q);
        j1[t] = j;
        jk1[t] = j - x;
        if (p == q) {
            jdiag[p * n + k] = eri_get(I, p, p, k, k);
            kdiag[p * n + k] = eri_get(I, p, k, k, p);
        }
    }
}

void load_integrals(shci_ctx *c, int n_orb, double e_core, const double *h, const double *eri, int mem) {
    if (n_orb < 1 || n_orb > SHCI_MAX_ORB) throw ShciError{SHCI_ERR_INVALID, "n_orb must be in [1, 128]"};
    if (!h || !eri) throw ShciError{SHCI_ERR_INVALID, "null integral pointer"};
    int64_t npair = (int64_t)n_orb * (n_orb + 1) / 2;
    int64_t neri = npair * (npair + 1) / 2;
    std::vector<double> hh((size_t)n_orb * n_orb);
    cudaMemcpyKind kind = mem == SHCI_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (mem == SHCI_MEM_HOST) {
        std::copy(h, h + (size_t)n_orb * n_orb, hh.begin());
    } else {
        CUDA_TRY(cudaMemcpyAsync(hh.data(), h, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    for (int p = 0; p < n_orb; p++)
        for (int q = 0; q < p; q++)
            if (!(std::abs(hh[p * n_orb + q] - hh[q * n_orb + p]) <= 1e-12))
                throw ShciError{SHCI_ERR_INVALID, "h is not symmetric"};
    c->built = false;
    c->h.alloc(hh.size());
    c->eri.alloc((size_t)neri);
    c->jk1.alloc((size_t)n_orb * n_orb * n_orb);
    c->j1.alloc((size_t)n_orb * n_orb * n_orb);
    c->jdiag.alloc((size_t)n_orb * n_orb);
    c->kdiag.alloc((size_t)n_orb * n_orb);
    CUDA_TRY(cudaMemcpyAsync(c->h.p, hh.data(), sizeof(double) * hh.size(), cudaMemcpyHostToDevice, c->st));
    CUDA_TRY(cudaMemcpyAsync(c->eri.p, eri, sizeof(double) * neri, kind, c->st));
    int64_t total = (int64_t)n_orb * n_orb * n_orb;
    k_mean_field_tables<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 4096), 256, 0, c->st>>>(
        c->eri.p, n_orb, c->jk1.p, c->j1.p, c->jdiag.p, c->kdiag.p);
    KERNEL_CHECK();
    LAUNCHED(1);
    CUDA_TRY(cudaStreamSynchronize(c->st));
    c->n_orb = n_orb;
    c->e_core = e_core;
    c->have_ints = true;
    c->hb_valid = false;
}

DevInts dev_ints(const shci_ctx *c) {
    DevInts I;
    I.h = c->h.p;
    I.eri = c->eri.p;
    I.jk1 = c->jk1.p;
    I.j1 = c->j1.p;
    I.jdiag = c->jdiag.p;
    I.kdiag = c->kdiag.p;
    I.e_core = c->e_core;
    I.n = c->n_orb;
    return I;
}

// ====================================================================== helper lists

// flags: bit 0 wrong alpha popcount, bit 1 wrong beta popcount, bit 2 bits beyond n_orb
template <int W>
__global__ void k_validate(const uint64_t *__restrict__ dets, int64_t n, int n_orb, int na, int nb, int *flags) {
    int f = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int ca = 0, cb = 0;
#pragma unroll
        for (int k = 0; k < W; k++) {
            uint64_t a = dets[i * 2 * W + k], b = dets[i * 2 * W + W + k];
            ca += __popcll(a);
            cb += __popcll(b);
            int lo = 64 * k;
            uint64_t valid = n_orb - lo >= 64 ? ~0ull : (n_orb - lo <= 0 ? 0ull : ((1ull << (n_orb - lo)) - 1));
            if ((a | b) & ~valid) f |= 4;
        }
        if (ca != na) f |= 1;
        if (cb != nb) f |= 2;
    }
    if (f) atomicOr(flags, f);
}

// keys[i] = spin string `spin` of determinant i; vals[i] = i
template <int W>
__global__ void k_extract_strings(const uint64_t *__restrict__ dets, int64_t n, int spin, uint64_t *__restrict__ keys,
                                  uint32_t *__restrict__ vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < W; k++) keys[i * W + k] = dets[i * 2 * W + spin * W + k];
        vals[i] = (uint32_t)i;
    }
}

template <int KW>
__global__ void k_head_flags(const uint64_t *__restrict__ keys, int64_t n, int64_t *__restrict__ flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t f = 1;
        if (i > 0) {
            f = 0;
#pragma unroll
            for (int k = 0; k < KW; k++) f |= keys[i * KW + k] != keys[(i - 1) * KW + k];
        }
        flags[i] = f;
    }
}

// after an exclusive scan of head flags: write unique strings and the string index of each det
template <int W>
__global__ void k_unique_write(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                               const int64_t *__restrict__ flags, const int64_t *__restrict__ excl, int64_t n,
                               uint64_t *__restrict__ ustr, int32_t *__restrict__ sidx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t id = excl[i] + flags[i] - 1;
        if (flags[i]) {
#pragma unroll
            for (int k = 0; k < W; k++) ustr[id * W + k] = keys[i * W + k];
        }
        sidx[vals[i]] = (int32_t)id;
    }
}

// composite key (major << 32 | minor) per determinant; minor == nullptr takes
// the determinant index
__global__ void k_composite(const int32_t *__restrict__ major, const int32_t *__restrict__ minor, int64_t n,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = ((uint64_t)(uint32_t)major[i] << 32) | (minor ? (uint32_t)minor[i] : (uint32_t)i);
        vals[i] = (uint32_t)i;
    }
}

// group offsets from sorted composite keys; members and the other spin's string; duplicates -> flag
template <int W>
__global__ void k_group_build(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                              const uint64_t *__restrict__ dets, int other_spin, int64_t n_groups,
                              int64_t *__restrict__ off, int32_t *__restrict__ mdet, uint64_t *__restrict__ mstr,
                              int *flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        int64_t g = (int64_t)(k >> 32);
        if (i == 0 || (keys[i - 1] >> 32) != (uint64_t)g) off[g] = i;
        if (i > 0 && keys[i - 1] == k) atomicOr(flags, 8);   // duplicate determinant
        uint32_t d = vals[i];
        mdet[i] = (int32_t)d;
#pragma unroll
        for (int w = 0; w < W; w++) mstr[i * W + w] = dets[(int64_t)d * 2 * W + other_spin * W + w];
        if (i == n - 1) off[n_groups] = n;
    }
}

// groups whose members are in determinant order: the offset of each group's
// first member with index >= n_old (the group's end when it has none)
__global__ void k_new_start_init(const int64_t *__restrict__ off, int64_t n_groups, int64_t *__restrict__ g_new) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_groups; g += (int64_t)gridDim.x * blockDim.x)
        g_new[g] = off[g + 1];
}

__global__ void k_new_start(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                            int64_t n_old, int64_t *__restrict__ g_new) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        if ((int64_t)vals[p] < n_old) continue;
        const uint64_t g = keys[p] >> 32;
        if (p == 0 || (keys[p - 1] >> 32) != g || (int64_t)vals[p - 1] < n_old) g_new[g] = p;
    }
}

// incremental update: row lengths and the offsets of the two new parts of each
// row (old elements first, then the beta-grouped and alpha-grouped new ones)
__global__ void k_extend_rows(const int64_t *__restrict__ old_rowptr, int64_t n_old, const int64_t *__restrict__ cnt_b,
                              const int64_t *__restrict__ cnt_a, int64_t n, int64_t *__restrict__ len,
                              int64_t *__restrict__ off_b, int64_t *__restrict__ off_a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t old = i < n_old ? old_rowptr[i + 1] - old_rowptr[i] : 0;
        off_b[i] = old;
        off_a[i] = old + cnt_b[i];
        len[i] = old + cnt_b[i] + cnt_a[i];
    }
}

// incremental update: old rows to the head of their new slots, one warp per row
__global__ void k_copy_rows(const int64_t *__restrict__ old_rowptr, const int32_t *__restrict__ old_col,
                            const double *__restrict__ old_val, int64_t n_old, const int64_t *__restrict__ rowptr,
                            int32_t *__restrict__ col, double *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n_old; i += warps) {
        const int64_t src = old_rowptr[i], len = old_rowptr[i + 1] - src, dst = rowptr[i];
        for (int64_t e = lane; e < len; e += 32) {
            col[dst + e] = __ldcs(&old_col[src + e]);
            val[dst + e] = __ldcs(&old_val[src + e]);
        }
    }
}

// alpha^(-1) keys: each unique alpha string with one of its electrons removed
template <int W>
__global__ void k_minus_one_keys(const uint64_t *__restrict__ astr, int64_t Ua, int ne, uint64_t *__restrict__ keys,
                                 uint32_t *__restrict__ vals) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < Ua; a += (int64_t)gridDim.x * blockDim.x) {
        Str<W> s = load_str<W>(astr, a);
        Str<W> m = s;
        for (int e = 0; e < ne; e++) {
            int b = lowest_bit<W>(m);
            clear_bit<W>(m, b);
            Str<W> key = s;
            clear_bit<W>(key, b);
            int64_t t = a * ne + e;
#pragma unroll
            for (int w = 0; w < W; w++) keys[t * W + w] = key.w[w];
            vals[t] = (uint32_t)t;
        }
    }
}

// for each sorted entry: its segment start / length, stored at the entry's original slot
template <int W>
__global__ void k_segment_info(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                               int64_t *__restrict__ seg_start, int32_t *__restrict__ seg_len) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        auto same = [&](int64_t x, int64_t y) {
            bool eq = true;
#pragma unroll
            for (int w = 0; w < W; w++) eq &= keys[x * W + w] == keys[y * W + w];
            return eq;
        };
        if (i > 0 && same(i, i - 1)) continue;   // only segment heads work
        int64_t e = i + 1;
        while (e < n && same(e, i)) e++;
        for (int64_t t = i; t < e; t++) {
            seg_start[vals[t]] = i;
            seg_len[vals[t]] = (int32_t)(e - i);
        }
    }
}

__global__ void k_singles_count(const int32_t *__restrict__ seg_len, int64_t Ua, int ne, int64_t *__restrict__ cnt) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < Ua; a += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        for (int e = 0; e < ne; e++) c += seg_len[a * ne + e] - 1;
        cnt[a] = c;
    }
}

__global__ void k_singles_fill(const int64_t *__restrict__ seg_start, const int32_t *__restrict__ seg_len,
                               const uint32_t *__restrict__ vals, int64_t Ua, int ne, const int64_t *__restrict__ off,
                               int32_t *__restrict__ out) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < Ua; a += (int64_t)gridDim.x * blockDim.x) {
        int64_t pos = off[a];
        for (int e = 0; e < ne; e++) {
            int64_t s = seg_start[a * ne + e];
            int len = seg_len[a * ne + e];
            for (int t = 0; t < len; t++) {
                int64_t b = vals[s + t] / ne;
                if (b != a) out[pos++] = (int32_t)b;
            }
        }
    }
}

template <int W>
__global__ void k_diag(const uint64_t *__restrict__ dets, int64_t n, DevInts I, double *__restrict__ diag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Str<W> a = load_str<W>(dets, 2 * i);
        Str<W> b = load_str<W>(dets, 2 * i + 1);
        diag[i] = hii<W>(I, a, b);
    }
}

// ====================================================================== connectivity

// (kernels in enumerate.cuh)

__global__ void k_add_i64(int64_t *__restrict__ a, const int64_t *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

static void make_items(shci_ctx *c, const int64_t *off, int64_t n_groups, DevBuf<int32_t> &item_group,
                       DevBuf<int32_t> &item_first, int64_t &n_items) {
    cudaStream_t st = c->st;
    DevBuf<int64_t> cnt, start, tmp;
    cnt.alloc((size_t)n_groups + 1);
    start.alloc((size_t)n_groups + 1);
    tmp.alloc((size_t)scan_tmp_len(n_groups + 1));
    unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_groups, 256), 4096));
    k_items_count<<<g, 256, 0, st>>>(off, n_groups, cnt.p);
    exclusive_scan<int64_t>(cnt.p, start.p, n_groups, tmp.p, st);
    CUDA_TRY(cudaMemcpyAsync(&n_items, start.p + n_groups, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (n_items > 0x7FFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many work items"};
    item_group.alloc((size_t)std::max<int64_t>(n_items, 1));
    item_first.alloc((size_t)std::max<int64_t>(n_items, 1));
    k_items_fill<<<g, 256, 0, st>>>(off, start.p, n_groups, item_group.p, item_first.p);
    KERNEL_CHECK();
    g_kernel_launches += 2;
}


// incremental update: work items over the old (part 0) or new (part 1) members
// of each determinant-ordered group, with the member offset each item ends at
struct PartItems {
    DevBuf<int32_t> group, first, end;
    int64_t n = 0;
};

static void make_items_part(shci_ctx *c, const int64_t *off, const int64_t *g_new, int64_t n_groups, int part,
                            PartItems &P) {
    cudaStream_t st = c->st;
    DevBuf<int64_t> cnt, start, tmp;
    cnt.alloc((size_t)n_groups + 1);
    start.alloc((size_t)n_groups + 1);
    tmp.alloc((size_t)scan_tmp_len(n_groups + 1));
    unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_groups, 256), 4096));
    k_items_count_part<<<g, 256, 0, st>>>(off, g_new, n_groups, part, cnt.p);
    exclusive_scan<int64_t>(cnt.p, start.p, n_groups, tmp.p, st);
    CUDA_TRY(cudaMemcpyAsync(&P.n, start.p + n_groups, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (P.n > 0x7FFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many work items"};
    P.group.alloc((size_t)std::max<int64_t>(P.n, 1));
    P.first.alloc((size_t)std::max<int64_t>(P.n, 1));
    P.end.alloc((size_t)std::max<int64_t>(P.n, 1));
    k_items_fill_part<<<g, 256, 0, st>>>(off, g_new, start.p, n_groups, part, P.group.p, P.first.p, P.end.p);
    KERNEL_CHECK();
    g_kernel_launches += 2;
}

// one count or fill pass of the incremental update over the given items, rows
// taken from the determinant-ordered member lists rdet / rstr
template <int W, int MODE>
static void extend_pass(shci_ctx *c, EnumArgs E, const DevInts &I, bool alpha_part, const PartItems &items,
                        const int32_t *rdet, const uint64_t *rstr) {
    if (items.n == 0) return;
    E.item_group = items.group.p;
    E.item_first = items.first.p;
    E.item_end = items.end.p;
    E.n_items = items.n;
    E.row_det = rdet;
    E.row_str = rstr;
    launch_enum<W, MODE, 0>(c, E, I, alpha_part);
}

// ====================================================================== host pipeline

static inline unsigned grid_for(int64_t n, int threads = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), 152 * 32));
}

template <int W>
static void unique_strings(shci_ctx *c, int spin, DevBuf<uint64_t> &ustr, DevBuf<int32_t> &sidx, int64_t &U) {
    const int64_t n = c->n_det;
    cudaStream_t st = c->st;
    c->sort_keys.alloc((size_t)n * W);
    c->sort_vals.alloc((size_t)n);
    k_extract_strings<W><<<grid_for(n), 256, 0, st>>>(c->dets.p, n, spin, c->sort_keys.p, c->sort_vals.p);
    KERNEL_CHECK();
    radix_sort<W>(c->sort_keys.p, c->sort_vals.p, n, c->sw, st);
    c->i64a.alloc((size_t)n + 1);
    c->i64b.alloc((size_t)n + 1);
    c->i64c.alloc((size_t)scan_tmp_len(n + 1));
    k_head_flags<W><<<grid_for(n), 256, 0, st>>>(c->sort_keys.p, n, c->i64a.p);
    exclusive_scan<int64_t>(c->i64a.p, c->i64b.p, n, c->i64c.p, st);
    CUDA_TRY(cudaMemcpyAsync(&U, c->i64b.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    ustr.alloc((size_t)U * W);
    sidx.alloc((size_t)n);
    k_unique_write<W><<<grid_for(n), 256, 0, st>>>(c->sort_keys.p, c->sort_vals.p, c->i64a.p, c->i64b.p, n, ustr.p,
                                                   sidx.p);
    KERNEL_CHECK();
    LAUNCHED(3);
}

template <int W>
static void group_by(shci_ctx *c, const int32_t *major, const int32_t *minor, int64_t n_groups, int other_spin,
                     DevBuf<int64_t> &off, DevBuf<int32_t> &mdet, DevBuf<uint64_t> &mstr) {
    const int64_t n = c->n_det;
    cudaStream_t st = c->st;
    k_composite<<<grid_for(n), 256, 0, st>>>(major, minor, n, c->sort_keys.p, c->sort_vals.p);
    KERNEL_CHECK();
    radix_sort<1>(c->sort_keys.p, c->sort_vals.p, n, c->sw, st);
    off.alloc((size_t)n_groups + 1);
    mdet.alloc((size_t)n);
    mstr.alloc((size_t)n * W);
    k_group_build<W><<<grid_for(n), 256, 0, st>>>(c->sort_keys.p, c->sort_vals.p, n, c->dets.p, other_spin,
                                                  n_groups, off.p, mdet.p, mstr.p, c->counter.p);
    KERNEL_CHECK();
    LAUNCHED(2);
}

// Groups by `major` with members in determinant order (the incremental
// update's list order, Sec. III): members and their other-spin strings into
// mdet / mstr, and the offset of each group's first new member into g_new.
// The offsets equal those of group_by over the same strings.
template <int W>
static void group_by_index(shci_ctx *c, const int32_t *major, int64_t n_groups, int other_spin, int64_t n_old,
                           DevBuf<int64_t> &off, DevBuf<int32_t> &mdet, DevBuf<uint64_t> &mstr,
                           DevBuf<int64_t> &g_new) {
    const int64_t n = c->n_det;
    cudaStream_t st = c->st;
    k_composite<<<grid_for(n), 256, 0, st>>>(major, nullptr, n, c->sort_keys.p, c->sort_vals.p);
    KERNEL_CHECK();
    radix_sort<1>(c->sort_keys.p, c->sort_vals.p, n, c->sw, st);
    off.alloc((size_t)n_groups + 1);
    mdet.alloc((size_t)n);
    mstr.alloc((size_t)n * W);
    g_new.alloc((size_t)n_groups);
    k_group_build<W><<<grid_for(n), 256, 0, st>>>(c->sort_keys.p, c->sort_vals.p, n, c->dets.p, other_spin,
                                                  n_groups, off.p, mdet.p, mstr.p, c->counter.p);
    k_new_start_init<<<grid_for(n_groups), 256, 0, st>>>(off.p, n_groups, g_new.p);
    k_new_start<<<grid_for(n), 256, 0, st>>>(c->sort_keys.p, c->sort_vals.p, n, n_old, g_new.p);
    KERNEL_CHECK();
    LAUNCHED(4);
}

// Single-excitation lists (Table I's alpha-singles, and the beta mirror) over
// the U unique strings `ustr` with ne electrons: keys are the strings with one
// electron removed (alpha^(-1)); strings sharing a key are single excitations
// of one another, and each such pair shares exactly one key (Sec. III).
template <int W>
static int64_t string_singles(shci_ctx *c, const uint64_t *ustr, int64_t U, int ne, DevBuf<int64_t> &off,
                              DevBuf<int32_t> &idx) {
    cudaStream_t st = c->st;
    const int64_t nk = U * ne;
    off.alloc((size_t)U + 1);
    if (ne == 0 || nk == 0) {
        CUDA_TRY(cudaMemsetAsync(off.p, 0, sizeof(int64_t) * (U + 1), st));
        idx.alloc(1);
        return 0;
    }
    if (nk > 0x7FFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "too many unique strings"};
    c->sort_keys.alloc((size_t)std::max<int64_t>(nk * W, c->n_det * W));
    c->sort_vals.alloc((size_t)std::max<int64_t>(nk, c->n_det));
    k_minus_one_keys<W><<<grid_for(U), 256, 0, st>>>(ustr, U, ne, c->sort_keys.p, c->sort_vals.p);
    KERNEL_CHECK();
    radix_sort<W>(c->sort_keys.p, c->sort_vals.p, nk, c->sw, st);
    DevBuf<int64_t> seg_start;
    DevBuf<int32_t> seg_len;
    seg_start.alloc((size_t)nk);
    seg_len.alloc((size_t)nk);
    k_segment_info<W><<<grid_for(nk), 256, 0, st>>>(c->sort_keys.p, c->sort_vals.p, nk, seg_start.p, seg_len.p);
    c->i64a.alloc((size_t)std::max<int64_t>(U + 1, c->n_det + 1));
    c->i64c.alloc((size_t)scan_tmp_len(std::max<int64_t>(U + 1, c->n_det + 1)));
    k_singles_count<<<grid_for(U), 256, 0, st>>>(seg_len.p, U, ne, c->i64a.p);
    exclusive_scan<int64_t>(c->i64a.p, off.p, U, c->i64c.p, st);
    int64_t total = 0;
    CUDA_TRY(cudaMemcpyAsync(&total, off.p + U, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    idx.alloc((size_t)std::max<int64_t>(total, 1));
    k_singles_fill<<<grid_for(U), 256, 0, st>>>(seg_start.p, seg_len.p, c->sort_vals.p, U, ne, off.p, idx.p);
    KERNEL_CHECK();
    LAUNCHED(4);
    CUDA_TRY(cudaStreamSynchronize(st));
    return total;
}

template <int W>
static void alpha_singles(shci_ctx *c) {
    c->n_alpha_singles = string_singles<W>(c, c->astr.p, c->Ua, c->n_alpha, c->as_off, c->as_idx);
}

// occupancy bitmap over (unique alpha, unique beta) and, per 64-bit word, the
// number of set bits before it in its row: the rank of a present (a, b) among
// the members of alpha group a (sorted by beta index) is its member offset
__global__ void k_occ_set(const int32_t *__restrict__ ia, const int32_t *__restrict__ ib, int64_t n, int64_t ow,
                          unsigned long long *__restrict__ occ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = ib[i];
        atomicOr(&occ[(int64_t)ia[i] * ow + (b >> 6)], 1ull << (b & 63));
    }
}

__global__ void k_occ_prefix(const unsigned long long *__restrict__ occ, int64_t Ua, int64_t ow,
                             int32_t *__restrict__ pref) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < Ua; a += (int64_t)gridDim.x * blockDim.x) {
        int32_t run = 0;
        for (int64_t w = 0; w < ow; w++) {
            pref[a * ow + w] = run;
            run += __popcll(occ[a * ow + w]);
        }
    }
}


// Beta-single lists and the occupancy bitmap for the opposite-spin doubles.
// SHCI_OPP_SPIN=scan: no bitmap, every alpha single's group is scanned;
// lookup: every (alpha single, beta single) pair is looked up; auto (default):
// the enumeration chooses per alpha single (scan the group when it is short
// compared with the CTA's beta-single lists, SHCI_OPP_FACTOR times at most).
// The bitmap is skipped when it would take more than 4 GB.
template <int W>
static void opposite_spin_setup(shci_ctx *c) {
    cudaStream_t st = c->st;
    c->n_beta_singles = string_singles<W>(c, c->bstr.p, c->Ub, c->n_beta, c->bs_off, c->bs_idx);
    c->occ_words = (c->Ub + 63) / 64;
    const double bytes = (double)c->Ua * c->occ_words * 12.0;
    const char *env = getenv("SHCI_OPP_SPIN");
    std::string pref = env ? env : "auto";
    c->opp_lookup = false;
    c->opp_hybrid = false;
    if (pref == "scan" || bytes > 4.0e9) {
        c->occ.reset();
        c->occ_pref.reset();
        return;
    }
    c->occ.alloc((size_t)(c->Ua * c->occ_words));
    c->occ_pref.alloc((size_t)(c->Ua * c->occ_words));
    CUDA_TRY(cudaMemsetAsync(c->occ.p, 0, sizeof(unsigned long long) * c->Ua * c->occ_words, st));
    k_occ_set<<<grid_for(c->n_det), 256, 0, st>>>(c->ia.p, c->ib.p, c->n_det, c->occ_words, c->occ.p);
    k_occ_prefix<<<grid_for(c->Ua), 256, 0, st>>>(c->occ.p, c->Ua, c->occ_words, c->occ_pref.p);
    KERNEL_CHECK();
    LAUNCHED(2);
    c->opp_lookup = true;
    c->opp_hybrid = pref != "lookup";
    // the crossover of the per-alpha-single choice (SHCI_OPP_FACTOR overrides):
    // 0.5 measured fastest on GB300 among 0.5-4 (24- and 76-orbital shapes)
    const char *fenv = getenv("SHCI_OPP_FACTOR");
    c->opp_factor = fenv ? (float)atof(fenv) : 0.5f;
    if (!(c->opp_factor >= 0.0f)) c->opp_factor = 0.5f;
}

// SHCI_AUTO: store both triangles of H when their nnz_full elements (12 bytes
// each) fit 80 % of the free device memory and the context's budget, else the
// upper triangle alone when its nnz_full / 2 elements fit, else apply H on the fly
static int decide_mode(shci_ctx *c, int mode, int64_t nnz_full) {
    if (mode != SHCI_AUTO) return mode;
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    double need = (double)nnz_full * 12.0;
    double cap = 0.8 * (double)free_b;
    if (c->stored_budget >= 0.0) cap = std::min(cap, c->stored_budget);
    if (need < cap) return SHCI_STORED;
    return 0.5 * need < cap ? SHCI_STORED_UPPER : SHCI_ON_THE_FLY;
}

// entries held by a stored matrix: both triangles or the upper one
static int64_t stored_entries(const shci_ctx *c) {
    return c->mode == SHCI_STORED_UPPER ? c->nnz_upper : c->nnz_full;
}

// validation, helper lists (Table I), the diagonal and the work items of V
template <int W>
static void lists_w(shci_ctx *c) {
    cudaStream_t st = c->st;
    const int64_t n = c->n_det;
    c->counter.alloc(4);
    CUDA_TRY(cudaMemsetAsync(c->counter.p, 0, 4 * sizeof(int), st));
    k_validate<W><<<grid_for(n), 256, 0, st>>>(c->dets.p, n, c->n_orb, c->n_alpha, c->n_beta, c->counter.p);
    KERNEL_CHECK();
    LAUNCHED(1);
    int flags = 0;
    CUDA_TRY(cudaMemcpyAsync(&flags, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (flags & 1) throw ShciError{SHCI_ERR_INVALID, "an alpha string does not hold n_alpha electrons"};
    if (flags & 2) throw ShciError{SHCI_ERR_INVALID, "a beta string does not hold n_beta electrons"};
    if (flags & 4) throw ShciError{SHCI_ERR_INVALID, "a determinant occupies an orbital >= n_orb"};

    unique_strings<W>(c, 0, c->astr, c->ia, c->Ua);
    unique_strings<W>(c, 1, c->bstr, c->ib, c->Ub);
    group_by<W>(c, c->ia.p, c->ib.p, c->Ua, 1, c->ga_off, c->ga_det, c->ga_str);
    group_by<W>(c, c->ib.p, c->ia.p, c->Ub, 0, c->gb_off, c->gb_det, c->gb_str);
    CUDA_TRY(cudaMemcpyAsync(&flags, c->counter.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (flags & 8) throw ShciError{SHCI_ERR_INVALID, "duplicate determinants in V"};
    alpha_singles<W>(c);
    opposite_spin_setup<W>(c);

    DevInts I = dev_ints(c);
    c->diag.alloc((size_t)n);
    k_diag<W><<<grid_for(n, 128), 128, 0, st>>>(c->dets.p, n, I, c->diag.p);
    KERNEL_CHECK();
    LAUNCHED(1);

    // work items: chunks of ENUM_NW rows of one alpha (beta) group
    make_items(c, c->ga_off.p, c->Ua, c->item_a_group, c->item_a_first, c->n_items_a);
    make_items(c, c->gb_off.p, c->Ub, c->item_b_group, c->item_b_first, c->n_items_b);
}

// count pass: entries of the beta-grouped part and of the alpha-grouped part
// of each row, their offsets (rowptr) and the pair counts; with upper set,
// only the pairs j > i
template <int W>
static void count_w(shci_ctx *c, bool upper) {
    cudaStream_t st = c->st;
    const int64_t n = c->n_det;
    DevInts I = dev_ints(c);
    DevBuf<unsigned long long> cand;
    cand.alloc(1);
    CUDA_TRY(cudaMemsetAsync(cand.p, 0, sizeof(unsigned long long), st));
    c->rowptr.alloc((size_t)n + 1);
    c->cnt_b.alloc((size_t)n);
    c->i64a.alloc((size_t)n + 1);
    c->i64c.alloc((size_t)scan_tmp_len(n + 1));
    EnumArgs A = enum_args(c);
    A.cand = cand.p;
    A.cnt = c->cnt_b.p;
    if (upper) launch_enum<W, ENUM_COUNT_UP, 0>(c, A, I, false);
    else launch_enum<W, ENUM_COUNT, 0>(c, A, I, false);
    A.cnt = c->i64a.p;
    if (upper) launch_enum<W, ENUM_COUNT_UP, 0>(c, A, I, true);
    else launch_enum<W, ENUM_COUNT, 0>(c, A, I, true);
    k_add_i64<<<grid_for(n), 256, 0, st>>>(c->i64a.p, c->cnt_b.p, n);
    KERNEL_CHECK();
    LAUNCHED(1);
    exclusive_scan<int64_t>(c->i64a.p, c->rowptr.p, n, c->i64c.p, st);
    int64_t nnz = 0;
    unsigned long long ncand = 0;
    CUDA_TRY(cudaMemcpyAsync(&nnz, c->rowptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&ncand, cand.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    c->nnz_full = upper ? 2 * nnz : nnz;
    c->nnz_upper = upper ? nnz : nnz / 2;
    c->candidates = (int64_t)ncand;
    c->rows_upper = upper;
}

// Store H in mode SHCI_STORED or SHCI_STORED_UPPER after the lists and a
// count pass (recounted when the row lengths held are of the other form).
template <int W>
static void store_w(shci_ctx *c, int mode) {
    const bool upper = mode == SHCI_STORED_UPPER;
    if (c->rows_upper != upper) count_w<W>(c, upper);
    c->mode = mode;
    const int64_t nnz = stored_entries(c);
    c->col.alloc((size_t)std::max<int64_t>(nnz, 1));
    c->val.alloc((size_t)std::max<int64_t>(nnz, 1));
    DevInts I = dev_ints(c);
    EnumArgs A = enum_args(c);
    A.rowptr = c->rowptr.p;
    A.col = c->col.p;
    A.val = c->val.p;
    A.part_off = nullptr;
    if (upper) launch_enum<W, ENUM_FILL_UP, 0>(c, A, I, false);
    else launch_enum<W, ENUM_FILL, 0>(c, A, I, false);
    A.part_off = c->cnt_b.p;
    if (upper) launch_enum<W, ENUM_FILL_UP, 0>(c, A, I, true);
    else launch_enum<W, ENUM_FILL, 0>(c, A, I, true);
    CUDA_TRY(cudaStreamSynchronize(c->st));
}

template <int W>
static void build_w(shci_ctx *c, int mode) {
    lists_w<W>(c);
    count_w<W>(c, mode == SHCI_STORED_UPPER);
    mode = decide_mode(c, mode, c->nnz_full);
    if (mode == SHCI_STORED || mode == SHCI_STORED_UPPER) {
        store_w<W>(c, mode);
    } else {
        c->mode = mode;
        c->col.reset();
        c->val.reset();
    }
    CUDA_TRY(cudaStreamSynchronize(c->st));
}

void store(shci_ctx *c, int mode) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before storing it"};
    if (mode != SHCI_STORED && mode != SHCI_STORED_UPPER) throw ShciError{SHCI_ERR_INVALID, "unknown stored form"};
    if (c->mode == mode) return;
    c->built = false;
    c->col.reset();
    c->val.reset();
    if (c->W == 1) store_w<1>(c, mode);
    else store_w<2>(c, mode);
    c->built = true;
}

// Incremental update after V grew from n_old determinants (Sec. III,
// Algorithms 1 and 2).  The lists are rebuilt for all of V; a second copy of
// the per-string groups with members in determinant order puts each group's
// new members in a suffix.  New rows take every candidate from the usual
// lists (group scans or bitmap lookups, as in a full build); old rows take
// only the new candidates, the suffixes of the determinant-ordered groups
// (j >= s), each warp reading its row's suffixes directly.  The old rows are
// copied into the grown matrix ahead of their new elements.
// events on the context's stream marking the parts of an incremental update
struct PhaseMarks {
    cudaEvent_t e[5] = {};
    explicit PhaseMarks(cudaStream_t st) : st_(st) {
        for (auto &x : e) CUDA_TRY(cudaEventCreate(&x));
    }
    ~PhaseMarks() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
    void mark(int i) { CUDA_TRY(cudaEventRecord(e[i], st_)); }
    // after the stream has been synchronised: milliseconds between marks
    void read(double *ms, int parts) {
        for (int i = 0; i < parts; i++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e[i], e[i + 1]);
            ms[i] = t;
        }
    }
    cudaStream_t st_;
};

// Returns false, with nothing built, when SHCI_AUTO finds that both triangles
// of the grown matrix no longer fit but its upper triangle would: the row
// lengths counted here are the full ones, so the caller rebuilds V.
template <int W>
static bool extend_w(shci_ctx *c, int64_t n_old) {
    cudaStream_t st = c->st;
    const int64_t n = c->n_det;
    PhaseMarks pm(st);
    pm.mark(0);
    lists_w<W>(c);
    DevInts I = dev_ints(c);
    DevBuf<int64_t> off_tmp, ga_new, gb_new;
    DevBuf<int32_t> gad, gbd;
    DevBuf<uint64_t> gas, gbs;
    group_by_index<W>(c, c->ia.p, c->Ua, 1, n_old, off_tmp, gad, gas, ga_new);
    group_by_index<W>(c, c->ib.p, c->Ub, 0, n_old, off_tmp, gbd, gbs, gb_new);
    PartItems ia_old, ia_new, ib_old, ib_new;
    make_items_part(c, c->ga_off.p, ga_new.p, c->Ua, 0, ia_old);
    make_items_part(c, c->ga_off.p, ga_new.p, c->Ua, 1, ia_new);
    make_items_part(c, c->gb_off.p, gb_new.p, c->Ub, 0, ib_old);
    make_items_part(c, c->gb_off.p, gb_new.p, c->Ub, 1, ib_new);
    // new rows: every candidate, the context's lists
    EnumArgs An = enum_args(c);
    // old rows: new candidates only, determinant-ordered lists
    EnumArgs Ao = enum_args(c);
    Ao.ga_det = gad.p;
    Ao.ga_str = gas.p;
    Ao.gb_det = gbd.p;
    Ao.gb_str = gbs.p;
    Ao.opp_lookup = 0;
    Ao.opp_hybrid = 0;
    Ao.n_old = n_old;
    Ao.ga_new = ga_new.p;
    Ao.gb_new = gb_new.p;

    pm.mark(1);
    // count pass: new elements of each row, beta-grouped and alpha-grouped
    DevBuf<unsigned long long> cand;
    cand.alloc(1);
    CUDA_TRY(cudaMemsetAsync(cand.p, 0, sizeof(unsigned long long), st));
    DevBuf<int64_t> cnt_a, len, off_a, off_b, rowptr;
    c->cnt_b.alloc((size_t)n);
    cnt_a.alloc((size_t)n);
    len.alloc((size_t)n + 1);
    off_a.alloc((size_t)n);
    off_b.alloc((size_t)n);
    rowptr.alloc((size_t)n + 1);
    c->i64c.alloc((size_t)scan_tmp_len(n + 1));
    // an upper-triangle matrix grows by its new pairs j > i only
    An.upper_only = Ao.upper_only = c->mode == SHCI_STORED_UPPER ? 1 : 0;
    An.cand = Ao.cand = cand.p;
    An.cnt = Ao.cnt = c->cnt_b.p;
    extend_pass<W, ENUM_COUNT_INC>(c, An, I, false, ib_new, gbd.p, gbs.p);
    extend_pass<W, ENUM_COUNT_INC>(c, Ao, I, false, ib_old, gbd.p, gbs.p);
    An.cnt = Ao.cnt = cnt_a.p;
    extend_pass<W, ENUM_COUNT_INC>(c, An, I, true, ia_new, gad.p, gas.p);
    extend_pass<W, ENUM_COUNT_INC>(c, Ao, I, true, ia_old, gad.p, gas.p);
    k_extend_rows<<<grid_for(n), 256, 0, st>>>(c->rowptr.p, n_old, c->cnt_b.p, cnt_a.p, n, len.p, off_b.p, off_a.p);
    KERNEL_CHECK();
    LAUNCHED(1);
    exclusive_scan<int64_t>(len.p, rowptr.p, n, c->i64c.p, st);
    int64_t nnz = 0;
    unsigned long long ncand = 0;
    CUDA_TRY(cudaMemcpyAsync(&nnz, rowptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&ncand, cand.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    c->candidates = (int64_t)ncand;
    pm.mark(2);
    const bool upper = c->mode == SHCI_STORED_UPPER;
    const int64_t nnz_full = upper ? 2 * nnz : nnz;
    // a stored matrix stays stored unless SHCI_AUTO finds no room for the grown
    // one (both triangles may then fall back to the upper one, by a rebuild)
    int mode = c->mode;
    if (mode != SHCI_ON_THE_FLY && c->mode_req == SHCI_AUTO) {
        const int fit = decide_mode(c, SHCI_AUTO, nnz_full);
        if (fit == SHCI_ON_THE_FLY) mode = SHCI_ON_THE_FLY;
        else if (mode == SHCI_STORED && fit == SHCI_STORED_UPPER) return false;
    }
    if (mode == SHCI_STORED || mode == SHCI_STORED_UPPER) {
        DevBuf<int32_t> col;
        DevBuf<double> val;
        col.alloc((size_t)std::max<int64_t>(nnz, 1));
        val.alloc((size_t)std::max<int64_t>(nnz, 1));
        const unsigned gw = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_old, 8), (int64_t)c->n_sm * 8));
        k_copy_rows<<<gw, 256, 0, st>>>(c->rowptr.p, c->col.p, c->val.p, n_old, rowptr.p, col.p, val.p);
        KERNEL_CHECK();
        LAUNCHED(1);
        pm.mark(3);
        for (EnumArgs *E : {&An, &Ao}) {
            E->rowptr = rowptr.p;
            E->col = col.p;
            E->val = val.p;
            E->part_off = off_b.p;
        }
        extend_pass<W, ENUM_FILL_INC>(c, An, I, false, ib_new, gbd.p, gbs.p);
        extend_pass<W, ENUM_FILL_INC>(c, Ao, I, false, ib_old, gbd.p, gbs.p);
        An.part_off = Ao.part_off = off_a.p;
        extend_pass<W, ENUM_FILL_INC>(c, An, I, true, ia_new, gad.p, gas.p);
        extend_pass<W, ENUM_FILL_INC>(c, Ao, I, true, ia_old, gad.p, gas.p);
        c->col.swap(col);
        c->val.swap(val);
    } else {
        pm.mark(3);
        c->col.reset();
        c->val.reset();
    }
    pm.mark(4);
    c->mode = mode;
    c->rowptr.swap(rowptr);
    c->nnz_full = nnz_full;
    c->nnz_upper = upper ? nnz : nnz / 2;
    c->rows_upper = upper;
    CUDA_TRY(cudaStreamSynchronize(st));
    pm.read(c->stats.extend_phase_ms, 4);
    return true;
}

void extend(shci_ctx *c, int64_t n_new, const uint64_t *new_dets, int mem, double full_fraction) {
    if (!c->built) throw ShciError{SHCI_ERR_STATE, "build the connectivity before extending it"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    if (n_new < 0) throw ShciError{SHCI_ERR_INVALID, "n_new must be >= 0"};
    if (n_new == 0) return;
    if (!new_dets) throw ShciError{SHCI_ERR_INVALID, "null determinant pointer"};
    const int64_t n_old = c->n_det, n = n_old + n_new;
    if (n > 0x7FFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "n_old + n_new must be <= 2^31-1"};
    if (!(full_fraction > 0.0)) full_fraction = 0.2;
    const int W = c->W;
    c->built = false;
    {
        DevBuf<uint64_t> grown;
        grown.alloc((size_t)n * 2 * W);
        CUDA_TRY(cudaMemcpyAsync(grown.p, c->dets.p, sizeof(uint64_t) * n_old * 2 * W, cudaMemcpyDeviceToDevice,
                                 c->st));
        CUDA_TRY(cudaMemcpyAsync(grown.p + n_old * 2 * W, new_dets, sizeof(uint64_t) * n_new * 2 * W,
                                 mem == SHCI_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st));
        CUDA_TRY(cudaStreamSynchronize(c->st));
        c->dets.swap(grown);
    }
    c->n_det = n;
    bool incremental = (double)n_new < full_fraction * (double)n;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e0, c->st));
    if (incremental) incremental = W == 1 ? extend_w<1>(c, n_old) : extend_w<2>(c, n_old);
    if (!incremental) {
        // the rebuild replaces the stored matrix: release it first, so that
        // SHCI_AUTO decides against the memory the new one can have
        c->col.reset();
        c->val.reset();
        const int mode = c->mode_req == SHCI_AUTO ? SHCI_AUTO : c->mode;
        if (W == 1) build_w<1>(c, mode);
        else build_w<2>(c, mode);
    }
    CUDA_TRY(cudaEventRecord(e1, c->st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->stats.extend_ms = ms;
    c->stats.extend_incremental = incremental ? 1 : 0;
    if (!incremental)
        for (double &x : c->stats.extend_phase_ms) x = 0.0;
    c->stats.extend_n_old = n_old;
    c->built = true;
}

void build(shci_ctx *c, int n_alpha, int n_beta, int64_t n_det, const uint64_t *dets, int mem, int mode) {
    if (!c->have_ints) throw ShciError{SHCI_ERR_STATE, "load integrals before building"};
    if (n_det < 1 || n_det > 0x7FFFFFFFll) throw ShciError{SHCI_ERR_INVALID, "n_det must be in [1, 2^31-1]"};
    if (!dets) throw ShciError{SHCI_ERR_INVALID, "null determinant pointer"};
    if (n_alpha < 0 || n_beta < 0 || n_alpha > c->n_orb || n_beta > c->n_orb)
        throw ShciError{SHCI_ERR_INVALID, "electron counts out of range"};
    if (mode != SHCI_STORED && mode != SHCI_ON_THE_FLY && mode != SHCI_AUTO && mode != SHCI_STORED_UPPER)
        throw ShciError{SHCI_ERR_INVALID, "unknown mode"};
    if (mem != SHCI_MEM_HOST && mem != SHCI_MEM_DEVICE) throw ShciError{SHCI_ERR_INVALID, "unknown mem_space"};
    const int W = (c->n_orb + 63) / 64;
    c->built = false;
    c->mode_req = mode;
    c->W = W;
    c->n_alpha = n_alpha;
    c->n_beta = n_beta;
    c->n_det = n_det;
    c->dets.alloc((size_t)n_det * 2 * W);
    CUDA_TRY(cudaMemcpyAsync(c->dets.p, dets, sizeof(uint64_t) * n_det * 2 * W,
                             mem == SHCI_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e0, c->st));
    if (W == 1) build_w<1>(c, mode);
    else build_w<2>(c, mode);
    CUDA_TRY(cudaEventRecord(e1, c->st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->stats.build_ms = ms;
    c->built = true;
}

// ====================================================================== export

void export_pairs(shci_ctx *c, int64_t cap, int64_t *i_out, int64_t *j_out, double *v_out, int64_t *n_out) {
    if (!c->built || (c->mode != SHCI_STORED && c->mode != SHCI_STORED_UPPER))
        throw ShciError{SHCI_ERR_STATE, "no stored Hamiltonian"};
    if (n_out) *n_out = c->nnz_upper;
    if (cap < c->nnz_upper || c->nnz_upper == 0) return;
    if (!i_out || !j_out) throw ShciError{SHCI_ERR_INVALID, "null output pointer"};
    const int64_t n = c->n_det;
    std::vector<int64_t> rp((size_t)n + 1);
    const int64_t held = stored_entries(c);
    std::vector<int32_t> cl((size_t)held);
    std::vector<double> vl((size_t)held);
    CUDA_TRY(cudaMemcpyAsync(rp.data(), c->rowptr.p, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaMemcpyAsync(cl.data(), c->col.p, sizeof(int32_t) * held, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaMemcpyAsync(vl.data(), c->val.p, sizeof(double) * held, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    int64_t o = 0;
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = 0; i < n; i++) {
        row.clear();
        for (int64_t p = rp[i]; p < rp[i + 1]; p++)
            if (cl[p] > i) row.emplace_back(cl[p], vl[p]);
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int32_t, double> &x, const std::pair<int32_t, double> &y) { return x.first < y.first; });
        for (auto &e : row) {
            i_out[o] = i;
            j_out[o] = e.first;
            if (v_out) v_out[o] = e.second;
            o++;
        }
    }
}

}  // namespace shci
