// Enumeration of the connected determinant pairs of V (Sec. III, Algorithms
// 1 and 2) with a per-pair action: count, write H_ij (stored H), or
// accumulate H_ij c_j (on-the-fly sigma).
//
// Two kernels cover every pair (i, j), i != j, of one row i exactly once:
//   k_enum_alpha: rows grouped by alpha string a.  Candidates are the
//     determinants whose alpha string is a itself (same-spin beta
//     excitations) or one of a's alpha singles k (opposite-spin doubles when
//     the beta strings differ by one electron).  A CTA takes up to NW rows of
//     one alpha group (one warp each), so every candidate list it needs is the
//     same for all its warps: the list is staged tile by tile in shared memory
//     and screened by each warp with XOR + popcount + ballot.
//   k_enum_beta: rows grouped by beta string b; candidates share b
//     (same-spin alpha excitations), staged the same way.
// Row i's entries are laid out [beta-grouped part | alpha-grouped part].
//
// Only a few percent of the screened candidates are connected, so matches are
// not evaluated where they are found: each warp appends them to a queue in
// shared memory and evaluates H_ij 32 at a time, one per lane.
#pragma once
#include "common.cuh"

namespace shci {

constexpr int ENUM_NW = 8;                  // warps (rows) per CTA
constexpr int ENUM_THREADS = 32 * ENUM_NW;
constexpr int ENUM_TILE = 1024;             // candidates staged per tile
constexpr int ENUM_QCAP = 64;               // per-warp queue of found pairs

// ENUM_COUNT_INC / ENUM_FILL_INC: count / fill for the incremental update
// (rows from separate member lists and item ranges; with n_old > 0 the items
// hold old rows only, which take only the new candidates).
// ENUM_COUNT_UP / ENUM_FILL_UP: count / fill of the upper triangle (pairs
// j > i only); the incremental modes take that choice from EnumArgs::upper_only.
enum {
    ENUM_COUNT = 0, ENUM_FILL = 1, ENUM_SIGMA = 2, ENUM_GRAD = 3, ENUM_COUNT_INC = 4, ENUM_FILL_INC = 5,
    ENUM_COUNT_UP = 6, ENUM_FILL_UP = 7
};

template <int MODE>
struct ModeOf {
    static constexpr bool count = MODE == ENUM_COUNT || MODE == ENUM_COUNT_INC || MODE == ENUM_COUNT_UP;
    static constexpr bool fill = MODE == ENUM_FILL || MODE == ENUM_FILL_INC || MODE == ENUM_FILL_UP;
    static constexpr bool inc = MODE == ENUM_COUNT_INC || MODE == ENUM_FILL_INC;
    static constexpr bool up = MODE == ENUM_COUNT_UP || MODE == ENUM_FILL_UP;
};


constexpr int GRAD_REPLICAS = 32;           // gradient copies that spread the atomics

struct EnumArgs {
    const uint64_t *dets;
    const uint64_t *astr, *bstr;            // unique strings
    const int64_t *ga_off, *gb_off;         // groups by alpha / beta string
    const int32_t *ga_det, *gb_det;         // member determinant
    const uint64_t *ga_str, *gb_str;        // member's other string
    const int64_t *as_off;                  // alpha singles
    const int32_t *as_idx;
    // opposite-spin lookups (used when opp_lookup != 0); with opp_hybrid the
    // choice is made per alpha single k: scan group k when it has at most
    // opp_factor times as many members as the CTA's rows have beta singles,
    // else look up
    int opp_lookup;
    int opp_hybrid;
    float opp_factor;
    // incremental update (ENUM_COUNT_INC / ENUM_FILL_INC only): the items'
    // rows come from row_det / row_str (the groups with members in
    // determinant order) and end at member offset item_end[item]; with
    // n_old > 0 every row is old (< n_old) and takes only the new members of
    // its candidate groups, from ga_new / gb_new (offset of each group's first
    // new member) on, read directly by each warp
    const int32_t *row_det;
    const uint64_t *row_str;
    const int32_t *item_end;
    int64_t n_old;
    const int64_t *ga_new, *gb_new;
    const int32_t *ib;                      // beta string index of each determinant
    const int64_t *bs_off;                  // beta singles
    const int32_t *bs_idx;
    const unsigned long long *occ;          // [Ua][occ_words] occupancy bitmap over (alpha, beta)
    const int32_t *occ_pref;                // [Ua][occ_words] set bits before each word in its row
    int64_t occ_words;
    const int32_t *item_group;              // work item -> group index
    const int32_t *item_first;              // work item -> first member offset within the group
    int64_t n_items;
    int *work_counter;
    // incremental count / fill: with upper_only set, only the pairs j > i of
    // each row (the upper triangle) are counted and stored
    int upper_only;
    // count
    int64_t *cnt;                           // entries per row of this kernel's part
    unsigned long long *cand;               // candidates screened (statistics)
    // fill
    const int64_t *rowptr;
    const int64_t *part_off;                // offset of this kernel's part within the row (may be null)
    int32_t *col;
    double *val;
    // sigma
    const double *x;                        // [n][K] interleaved
    double *y;                              // [n][K]
    const double *diag;
    int accumulate;                         // 0: y = diag x + part, 1: y += part
    int k_active;                           // vectors in use (<= K; 0 means K)
    // gradient (x = the root c, [n])
    double *gdh;                            // [GRAD_REPLICAS][n_orb * n_orb]
    double *geri;                           // [GRAD_REPLICAS][packed length]
    int64_t geri_len;
};

// pairs j > i only: always in the upper-triangle modes, by the run-time flag in
// the incremental ones, never otherwise (compiled away there)
template <int MODE>
__device__ __forceinline__ bool upper_only(const EnumArgs &A) {
    return ModeOf<MODE>::up || (ModeOf<MODE>::inc && A.upper_only != 0);
}

// ---------------------------------------------------------------- matrix element pieces

// single excitation q -> p inside one spin string: D_i has string si, D_j has sj,
// both determinants have the other-spin string `other`
template <int W>
__device__ __forceinline__ double single_exc(const DevInts &I, const Str<W> &si, const Str<W> &sj,
                                             const Str<W> &other) {
    const int n = I.n;
    Str<W> pi, qj, common;
#pragma unroll
    for (int k = 0; k < W; k++) {
        uint64_t d = si.w[k] ^ sj.w[k];
        pi.w[k] = si.w[k] & d;
        qj.w[k] = sj.w[k] & d;
        common.w[k] = si.w[k] & sj.w[k];
    }
    const int p = lowest_bit<W>(pi), q = lowest_bit<W>(qj);
    const int neg = bits_between<W>(common, p < q ? p : q, p < q ? q : p);
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

// same-spin double: holes q1 < q2 in sj, particles p1 < p2 in si
template <int W>
__device__ __forceinline__ double same_double(const DevInts &I, const Str<W> &si, const Str<W> &sj) {
    Str<W> pm, qm;
#pragma unroll
    for (int k = 0; k < W; k++) {
        uint64_t d = si.w[k] ^ sj.w[k];
        pm.w[k] = si.w[k] & d;
        qm.w[k] = sj.w[k] & d;
    }
    int p1 = lowest_bit<W>(pm); clear_bit<W>(pm, p1); int p2 = lowest_bit<W>(pm);
    int q1 = lowest_bit<W>(qm); clear_bit<W>(qm, q1); int q2 = lowest_bit<W>(qm);
    int neg = bits_between<W>(sj, p1 < q1 ? p1 : q1, p1 < q1 ? q1 : p1);
    Str<W> x = sj;
    flip_bit<W>(x, q1);
    flip_bit<W>(x, p1);
    neg += bits_between<W>(x, p2 < q2 ? p2 : q2, p2 < q2 ? q2 : p2);
    return flip_sign(eri_get(I, p1, q1, p2, q2) - eri_get(I, p1, q2, p2, q1), neg);
}

// one-electron move inside a string: particle p (in si only), hole q (in sj
// only), pair index of (p, q) and the parity of sj's electrons between them
template <int W>
__device__ __forceinline__ void move_info(const Str<W> &si, const Str<W> &sj, int &pq, int &neg) {
    Str<W> pi, qj;
#pragma unroll
    for (int k = 0; k < W; k++) {
        uint64_t d = si.w[k] ^ sj.w[k];
        pi.w[k] = si.w[k] & d;
        qj.w[k] = sj.w[k] & d;
    }
    const int p = lowest_bit<W>(pi), q = lowest_bit<W>(qj);
    pq = pair_idx(p, q);
    neg = bits_between<W>(sj, p < q ? p : q, p < q ? q : p);
}

__device__ __forceinline__ double eri_pairs(const DevInts &I, int pq, int rs) {
    int hi = pq > rs ? pq : rs, lo = pq > rs ? rs : pq;
    return __ldg(&I.eri[(int64_t)hi * (hi + 1) / 2 + lo]);
}

// H_ij for a queued pair.  si / other: the row's string of the spin that
// differs and of the spin that does not (for an opposite-spin double: the
// row's beta and alpha strings); sj: D_j's string of the differing spin.
// ctx & 1 marks an opposite-spin double whose alpha part (pair index ctx >> 2,
// sign bit (ctx >> 1) & 1) was computed once for the whole candidate group.
template <int W>
__device__ __forceinline__ double eval_pair(const DevInts &I, const Str<W> &si, const Str<W> &other,
                                            const Str<W> &sj, int ctx) {
    if (ctx & 1) {
        int pq_b, neg_b;
        move_info<W>(si, sj, pq_b, neg_b);
        return flip_sign(eri_pairs(I, ctx >> 2, pq_b), ((ctx >> 1) & 1) + neg_b);
    }
    return xor_popc<W>(si, sj) == 2 ? single_exc<W>(I, si, sj, other) : same_double<W>(I, si, sj);
}

__device__ __forceinline__ int64_t eri_slot(int p, int q, int r, int s) {
    int a = pair_idx(p, q), b = pair_idx(r, s);
    int hi = a > b ? a : b, lo = a > b ? b : a;
    return (int64_t)hi * (hi + 1) / 2 + lo;
}

// Adjoint of one connected pair i < j: add c_i c_j dH_ij/d(integral) for
// both orders (i, j) and (j, i).  h entries are independent, so H_ij's h_pq
// and H_ji's h_qp go to different slots (weight w = c_i c_j each); a packed
// two-electron slot is shared by both orders (weight w2 = 2 c_i c_j).
template <int W>
__device__ __forceinline__ void grad_pair(const DevInts &I, double *__restrict__ gdh, double *__restrict__ geri,
                                          const Str<W> &si, const Str<W> &other, const Str<W> &sj, int ctx,
                                          double w) {
    const double w2 = 2.0 * w;
    if (ctx & 1) {
        int pq_b, neg_b;
        move_info<W>(si, sj, pq_b, neg_b);
        const int pq_a = ctx >> 2;
        const int hi = pq_a > pq_b ? pq_a : pq_b, lo = pq_a > pq_b ? pq_b : pq_a;
        red_add(&geri[(int64_t)hi * (hi + 1) / 2 + lo], flip_sign(w2, ((ctx >> 1) & 1) + neg_b));
        return;
    }
    const int n = I.n;
    Str<W> pm, qm;
#pragma unroll
    for (int k = 0; k < W; k++) {
        uint64_t d = si.w[k] ^ sj.w[k];
        pm.w[k] = si.w[k] & d;
        qm.w[k] = sj.w[k] & d;
    }
    if (xor_popc<W>(si, sj) == 2) {
        const int p = lowest_bit<W>(pm), q = lowest_bit<W>(qm);
        Str<W> common;
#pragma unroll
        for (int k = 0; k < W; k++) common.w[k] = si.w[k] & sj.w[k];
        const int neg = bits_between<W>(common, p < q ? p : q, p < q ? q : p);
        const double sw = flip_sign(w, neg), sw2 = flip_sign(w2, neg);
        red_add(&gdh[p * n + q], sw);
        red_add(&gdh[q * n + p], sw);
#pragma unroll
        for (int k = 0; k < W; k++) {
            uint64_t m = common.w[k];
            while (m) {
                const int b = 64 * k + __ffsll((long long)m) - 1;
                m &= m - 1;
                red_add(&geri[eri_slot(p, q, b, b)], sw2);
                red_add(&geri[eri_slot(p, b, b, q)], -sw2);
            }
            uint64_t o = other.w[k];
            while (o) {
                const int b = 64 * k + __ffsll((long long)o) - 1;
                o &= o - 1;
                red_add(&geri[eri_slot(p, q, b, b)], sw2);
            }
        }
        return;
    }
    int p1 = lowest_bit<W>(pm); clear_bit<W>(pm, p1); int p2 = lowest_bit<W>(pm);
    int q1 = lowest_bit<W>(qm); clear_bit<W>(qm, q1); int q2 = lowest_bit<W>(qm);
    int neg = bits_between<W>(sj, p1 < q1 ? p1 : q1, p1 < q1 ? q1 : p1);
    Str<W> x = sj;
    flip_bit<W>(x, q1);
    flip_bit<W>(x, p1);
    neg += bits_between<W>(x, p2 < q2 ? p2 : q2, p2 < q2 ? q2 : p2);
    const double sw2 = flip_sign(w2, neg);
    red_add(&geri[eri_slot(p1, q1, p2, q2)], sw2);
    red_add(&geri[eri_slot(p1, q2, p2, q1)], -sw2);
}

// ---------------------------------------------------------------- per-row state

template <int W>
struct WarpQueue {
    int32_t j[ENUM_QCAP];
    int32_t ctx[ENUM_QCAP];
    uint64_t s[ENUM_QCAP * W];
};

template <int MODE, int K>
struct RowAcc {
    int64_t found = 0;
    int64_t pos = 0;
    int qn = 0;
    int64_t i = 0;          // the row's determinant (gradient mode)
    int ka = K;             // vectors in use (sigma mode)
    double ci = 0.0;        // its coefficient (gradient mode)
    double acc[K > 0 ? K : 1];
};

// evaluate the first `cnt` (<= 32) queued pairs, one per lane, and apply the action
template <int W, int MODE, int K>
__device__ __forceinline__ void flush(RowAcc<MODE, K> &R, const EnumArgs &A, const DevInts &I, WarpQueue<W> &Q,
                                      const Str<W> &si, const Str<W> &other, int cnt) {
    const int lane = threadIdx.x & 31;
    if (MODE == ENUM_GRAD) {
        if (lane < cnt) {
            const int32_t j = Q.j[lane];
            if ((int64_t)j > R.i) {
                Str<W> sj;
#pragma unroll
                for (int k = 0; k < W; k++) sj.w[k] = Q.s[lane * W + k];
                const int rep = blockIdx.x % GRAD_REPLICAS;
                grad_pair<W>(I, A.gdh + (int64_t)rep * I.n * I.n, A.geri + rep * A.geri_len, si, other, sj,
                             Q.ctx[lane], R.ci * __ldg(&A.x[j]));
            }
        }
        return;
    }
    if (lane < cnt) {
        Str<W> sj;
#pragma unroll
        for (int k = 0; k < W; k++) sj.w[k] = Q.s[lane * W + k];
        const int32_t j = Q.j[lane];
        const double v = eval_pair<W>(I, si, other, sj, Q.ctx[lane]);
        if (ModeOf<MODE>::fill) {
            A.col[R.pos + lane] = j;
            A.val[R.pos + lane] = v;
        } else if (MODE == ENUM_SIGMA) {
            // x is read through L2 (ld.global.cg): the batched solver rewrites it
            // between phases of one persistent launch
            if (K == 2) {
                const double2 c2 = __ldcg(reinterpret_cast<const double2 *>(A.x) + j);
                R.acc[0] = fma(v, c2.x, R.acc[0]);
                R.acc[K - 1] = fma(v, c2.y, R.acc[K - 1]);
            } else {
                const int ka = R.ka;
#pragma unroll
                for (int q = 0; q < K; q++)
                    if (q < ka) R.acc[q] = fma(v, __ldcg(&A.x[(int64_t)j * K + q]), R.acc[q]);
            }
        }
    }
    if (ModeOf<MODE>::fill) R.pos += cnt;
}

// Record this round's matches: count them, or queue them and evaluate full
// rounds of 32.
template <int W, int MODE, int K>
__device__ __forceinline__ void emit(RowAcc<MODE, K> &R, const EnumArgs &A, const DevInts &I, WarpQueue<W> &Q,
                                     const Str<W> &si, const Str<W> &other, bool match, int32_t j, const Str<W> &sj,
                                     int ctx) {
    const int lane = threadIdx.x & 31;
    if (upper_only<MODE>(A)) match = match && (int64_t)j > R.i;
    const unsigned mask = __ballot_sync(0xffffffffu, match);
    const int nm = __popc(mask);
    R.found += nm;
    if (ModeOf<MODE>::count || nm == 0) return;
    if (match) {
        const int slot = R.qn + __popc(mask & ((1u << lane) - 1u));
        Q.j[slot] = j;
        Q.ctx[slot] = ctx;
#pragma unroll
        for (int k = 0; k < W; k++) Q.s[slot * W + k] = sj.w[k];
    }
    R.qn += nm;
    __syncwarp();
    if (R.qn >= 32) {
        flush<W, MODE, K>(R, A, I, Q, si, other, 32);
        __syncwarp();
        const int rest = R.qn - 32;
        if (lane < rest) {
            Q.j[lane] = Q.j[32 + lane];
            Q.ctx[lane] = Q.ctx[32 + lane];
#pragma unroll
            for (int k = 0; k < W; k++) Q.s[lane * W + k] = Q.s[(32 + lane) * W + k];
        }
        R.qn = rest;
        __syncwarp();
    }
}

// ---------------------------------------------------------------- tile staging

template <int W>
struct Tile {
    uint64_t str[ENUM_TILE * W];
    int32_t det[ENUM_TILE];
};

template <int W>
__device__ __forceinline__ void stage(Tile<W> &T, const uint64_t *__restrict__ mstr, const int32_t *__restrict__ mdet,
                                      int64_t start, int cnt, bool need_det) {
    for (int e = threadIdx.x; e < cnt * W; e += ENUM_THREADS) T.str[e] = __ldg(&mstr[start * W + e]);
    if (need_det)
        for (int e = threadIdx.x; e < cnt; e += ENUM_THREADS) T.det[e] = __ldg(&mdet[start + e]);
}

template <int W>
__device__ __forceinline__ Str<W> tile_str(const Tile<W> &T, int e) {
    Str<W> s;
#pragma unroll
    for (int k = 0; k < W; k++) s.w[k] = T.str[e * W + k];
    return s;
}

template <int MODE, int K>
__device__ __forceinline__ void row_begin(RowAcc<MODE, K> &R, const EnumArgs &A, int64_t i, bool valid) {
    R.found = 0;
    R.qn = 0;
    R.i = i;
#pragma unroll
    for (int q = 0; q < (K > 0 ? K : 1); q++) R.acc[q] = 0.0;
    if (ModeOf<MODE>::fill && valid) R.pos = A.rowptr[i] + (A.part_off ? A.part_off[i] : 0);
    if (MODE == ENUM_GRAD) R.ci = valid ? A.x[i] : 0.0;
}

template <int W, int MODE, int K>
__device__ __forceinline__ void row_end(RowAcc<MODE, K> &R, const EnumArgs &A, const DevInts &I, WarpQueue<W> &Q,
                                        const Str<W> &si, const Str<W> &other, int64_t i, bool valid) {
    const int lane = threadIdx.x & 31;
    if (!ModeOf<MODE>::count && R.qn > 0) {
        flush<W, MODE, K>(R, A, I, Q, si, other, R.qn);
        R.qn = 0;
        __syncwarp();
    }
    if (MODE == ENUM_SIGMA) {
        // only the R.ka vectors in use (warp-uniform); the others' outputs are not read
#pragma unroll
        for (int q = 0; q < K; q++) {
            if (q < R.ka) {
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) R.acc[q] += __shfl_xor_sync(0xffffffffu, R.acc[q], o);
            }
        }
        if (valid && lane == 0) {
#pragma unroll
            for (int q = 0; q < K; q++) {
                if (q >= R.ka) continue;
                const int64_t xi = i * K + q;
                if (A.accumulate) A.y[xi] = __ldcg(&A.y[xi]) + R.acc[q];
                else A.y[xi] = fma(A.diag[i], __ldcg(&A.x[xi]), R.acc[q]);
            }
        }
    } else if (ModeOf<MODE>::count) {
        if (valid && lane == 0) A.cnt[i] = R.found;
    }
}

// ---------------------------------------------------------------- kernels

// Incremental update, old rows (Sec. III, Algorithms 1 and 2: row i takes only
// candidates j >= s, the first new determinant): the same-spin single and
// double excitations among the new members of the row's own group,
// [m_beg, m_end) of the determinant-ordered member lists, screened by this
// warp alone (read directly; they are few).
template <int W, int MODE, int K>
__device__ __forceinline__ void old_row_suffix(RowAcc<MODE, K> &R, const EnumArgs &A, const DevInts &I,
                                               WarpQueue<W> &Q, const Str<W> &si, const Str<W> &other,
                                               const uint64_t *mstr, const int32_t *mdet, int64_t m_beg,
                                               int64_t m_end, unsigned long long &cand_local) {
    const int lane = threadIdx.x & 31;
    cand_local += lane == 0 ? (unsigned long long)(m_end - m_beg) : 0ull;
    for (int64_t m0 = m_beg; m0 < m_end; m0 += 32) {
        const int64_t m = m0 + lane;
        bool match = false;
        int32_t j = 0;
        Str<W> sj{};
        if (m < m_end) {
            sj = load_str<W>(mstr, m);
            const int d = xor_popc<W>(si, sj);
            match = (d == 2) | (d == 4);
            if (match) j = __ldg(&mdet[m]);
        }
        emit<W, MODE, K>(R, A, I, Q, si, other, match, j, sj, 0);
    }
}

// Rows grouped by alpha string: same-spin beta excitations (candidates in the
// row's own alpha group) and opposite-spin doubles (candidates in the alpha
// groups of the alpha singles of the row's alpha string).  One work item:
// up to ENUM_NW rows of one alpha group, one per warp; called by the whole CTA.
template <int W, int MODE, int K>
__device__ __forceinline__ void enum_alpha_item(const EnumArgs &A, const DevInts &I, int64_t item, Tile<W> &T,
                                                WarpQueue<W> &Q, unsigned long long &cand_local, int k_active = 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // member determinant indices: always outside the count modes; in them only
    // for an upper-triangle count (the filter compares j with the row)
    const bool need_det = !ModeOf<MODE>::count || upper_only<MODE>(A);
    constexpr bool XM = ModeOf<MODE>::inc;
    const int a = A.item_group[item];
    const int64_t g_beg = A.ga_off[a], g_len = A.ga_off[a + 1] - g_beg;
    const int32_t *rdet = XM ? A.row_det : A.ga_det;
    const uint64_t *rstr = XM ? A.row_str : A.ga_str;
    const int64_t r = A.item_first[item] + warp;            // this warp's member
    const bool valid = r < (XM ? (int64_t)A.item_end[item] : g_len);
    const int64_t i = valid ? rdet[g_beg + r] : 0;
    const Str<W> Ai = load_str<W>(A.astr, a);
    const Str<W> Bi = valid ? load_str<W>(rstr, g_beg + r) : Str<W>{};
    RowAcc<MODE, K> R;
    row_begin(R, A, i, valid);
    R.ka = k_active ? k_active : (A.k_active ? A.k_active : K);
    if (XM && A.n_old > 0) {
        // old rows: the new members of the own group (same-spin beta
        // excitations) and of the groups of the alpha singles of a
        // (opposite-spin doubles), by this warp alone
        if (valid) {
            const int64_t n_beg = A.ga_new[a];
            old_row_suffix<W, MODE, K>(R, A, I, Q, Bi, Ai, A.ga_str, A.ga_det, n_beg, g_beg + g_len, cand_local);
            const int64_t s_beg = A.as_off[a], s_end = A.as_off[a + 1];
            for (int64_t s0 = s_beg; s0 < s_end; s0 += 32) {
                // one alpha single per lane: its group's new members and pair context
                int64_t kb = 0;
                int len = 0, ctxl = 1;
                if (s0 + lane < s_end) {
                    const int k = A.as_idx[s0 + lane];
                    kb = A.ga_new[k];
                    len = (int)(A.ga_off[k + 1] - kb);
                    if (!ModeOf<MODE>::count && len > 0) {
                        int pq_a, neg_a;
                        move_info<W>(Ai, load_str<W>(A.astr, k), pq_a, neg_a);
                        ctxl = (pq_a << 2) | ((neg_a & 1) << 1) | 1;
                    }
                }
                int incl = len;                         // inclusive prefix over the lanes
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                cand_local += lane == 0 ? (unsigned long long)total : 0ull;
                for (int t0 = 0; t0 < total; t0 += 32) {
                    const int t = t0 + lane;
                    // the lane q whose range holds candidate t: the first with incl > t
                    int q = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int v = __shfl_sync(0xffffffffu, incl, q + step - 1);
                        if (v <= t) q += step;
                    }
                    q = min(q, 31);
                    const int64_t kq = __shfl_sync(0xffffffffu, kb, q);
                    const int before = __shfl_sync(0xffffffffu, incl - len, q);
                    const int cq = __shfl_sync(0xffffffffu, ctxl, q);
                    bool match = false;
                    int32_t j = 0;
                    Str<W> Bj{};
                    if (t < total) {
                        const int64_t m = kq + (t - before);
                        Bj = load_str<W>(A.ga_str, m);
                        match = xor_popc<W>(Bi, Bj) == 2;
                        if (match) j = __ldg(&A.ga_det[m]);
                    }
                    emit<W, MODE, K>(R, A, I, Q, Bi, Ai, match, j, Bj, cq);
                }
            }
        }
        row_end<W, MODE, K>(R, A, I, Q, Bi, Ai, i, valid);
        return;
    }
    // same-spin beta: candidates with the same alpha string
    for (int64_t t0 = 0; t0 < g_len; t0 += ENUM_TILE) {
        const int cnt = (int)min((int64_t)ENUM_TILE, g_len - t0);
        stage<W>(T, A.ga_str, A.ga_det, g_beg + t0, cnt, need_det);
        __syncthreads();
        if (valid) {
            cand_local += lane == 0 ? cnt : 0;
            for (int b0 = 0; b0 < cnt; b0 += 32) {
                const int e = b0 + lane;
                bool match = false;
                Str<W> Bj{};
                if (e < cnt) {
                    Bj = tile_str<W>(T, e);
                    const int d = xor_popc<W>(Bi, Bj);
                    match = (d == 2) | (d == 4);
                }
                emit<W, MODE, K>(R, A, I, Q, Bi, Ai, match, match && need_det ? T.det[e] : 0, Bj, 0);
            }
        }
        __syncthreads();
    }
    // opposite-spin doubles: candidates in the groups of the alpha singles of a,
    // found by scanning each group k (tiles shared by the CTA's warps) or by
    // looking up every (alpha single k of a, beta single kb of the row's beta
    // string) in the occupancy bitmap; a hit's rank within row k is its member
    // offset in alpha group k (members sorted by beta index)
    const int64_t s_beg = A.as_off[a], s_end = A.as_off[a + 1];
    int sb_len = 0;
    int64_t sb_beg = 0;
    __shared__ int sb_max_sh;
    int sb_max = 0;
    if (A.opp_lookup) {
        if (valid) {
            const int b = A.ib[i];
            sb_beg = A.bs_off[b];
            sb_len = (int)(A.bs_off[b + 1] - sb_beg);
        }
        if (A.opp_hybrid) {
            // the CTA's longest beta-single list: the cost of a lookup pass for its slowest warp
            if (threadIdx.x == 0) sb_max_sh = 0;
            __syncthreads();
            if (lane == 0) atomicMax(&sb_max_sh, sb_len);
            __syncthreads();
            sb_max = sb_max_sh;
            __syncthreads();
        }
    }
    for (int64_t s = s_beg; s < s_end; s++) {
        const int k = A.as_idx[s];
        const int64_t k_beg = A.ga_off[k], k_len = A.ga_off[k + 1] - k_beg;
        int ctx = 1;
        if (!ModeOf<MODE>::count) {
            int pq_a, neg_a;
            move_info<W>(Ai, load_str<W>(A.astr, k), pq_a, neg_a);
            ctx = (pq_a << 2) | ((neg_a & 1) << 1) | 1;
        }
        const bool lookup = A.opp_lookup && (!A.opp_hybrid || (float)k_len > A.opp_factor * (float)sb_max);
        if (lookup) {
            if (!valid) continue;
            const unsigned long long *row = A.occ + (int64_t)k * A.occ_words;
            cand_local += lane == 0 ? sb_len : 0;
            // LU lookups per lane per step, each stage's loads issued together
            // (independent L2 gathers in flight instead of one dependent chain)
            constexpr int LU = W == 1 ? 4 : 2;
            for (int y0 = 0; y0 < sb_len; y0 += 32 * LU) {
                int kb[LU];
                unsigned long long word[LU];
                bool match[LU];
                int32_t j[LU];
                Str<W> Bj[LU];
#pragma unroll
                for (int u = 0; u < LU; u++) {
                    const int y = y0 + 32 * u + lane;
                    kb[u] = y < sb_len ? __ldg(&A.bs_idx[sb_beg + y]) : -1;
                }
#pragma unroll
                for (int u = 0; u < LU; u++) word[u] = kb[u] >= 0 ? __ldg(&row[kb[u] >> 6]) : 0ull;
#pragma unroll
                for (int u = 0; u < LU; u++) {
                    match[u] = kb[u] >= 0 && ((word[u] >> (kb[u] & 63)) & 1ull);
                    j[u] = 0;
                    Bj[u] = Str<W>{};
                }
                if (need_det) {
                    int64_t m[LU];
#pragma unroll
                    for (int u = 0; u < LU; u++)
                        m[u] = match[u] ? __ldg(&A.occ_pref[(int64_t)k * A.occ_words + (kb[u] >> 6)]) : 0;
#pragma unroll
                    for (int u = 0; u < LU; u++) {
                        if (match[u]) {
                            m[u] += k_beg + __popcll(word[u] & ((1ull << (kb[u] & 63)) - 1ull));
                            j[u] = __ldg(&A.ga_det[m[u]]);
                            Bj[u] = load_str<W>(A.ga_str, m[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < LU; u++) emit<W, MODE, K>(R, A, I, Q, Bi, Ai, match[u], j[u], Bj[u], ctx);
            }
            continue;
        }
        for (int64_t t0 = 0; t0 < k_len; t0 += ENUM_TILE) {
            const int cnt = (int)min((int64_t)ENUM_TILE, k_len - t0);
            stage<W>(T, A.ga_str, A.ga_det, k_beg + t0, cnt, need_det);
            __syncthreads();
            if (valid) {
                cand_local += lane == 0 ? cnt : 0;
                for (int b0 = 0; b0 < cnt; b0 += 32) {
                    const int e = b0 + lane;
                    bool match = false;
                    Str<W> Bj{};
                    if (e < cnt) {
                        Bj = tile_str<W>(T, e);
                        match = xor_popc<W>(Bi, Bj) == 2;
                    }
                    emit<W, MODE, K>(R, A, I, Q, Bi, Ai, match, match && need_det ? T.det[e] : 0, Bj, ctx);
                }
            }
            __syncthreads();
        }
    }
    row_end<W, MODE, K>(R, A, I, Q, Bi, Ai, i, valid);
}

// Rows grouped by beta string: same-spin alpha excitations (candidates with
// the same beta string).  One work item, called by the whole CTA.
template <int W, int MODE, int K>
__device__ __forceinline__ void enum_beta_item(const EnumArgs &A, const DevInts &I, int64_t item, Tile<W> &T,
                                               WarpQueue<W> &Q, unsigned long long &cand_local, int k_active = 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool need_det = !ModeOf<MODE>::count || upper_only<MODE>(A);
    constexpr bool XM = ModeOf<MODE>::inc;
    const int b = A.item_group[item];
    const int64_t g_beg = A.gb_off[b], g_len = A.gb_off[b + 1] - g_beg;
    const int32_t *rdet = XM ? A.row_det : A.gb_det;
    const uint64_t *rstr = XM ? A.row_str : A.gb_str;
    const int64_t r = A.item_first[item] + warp;
    const bool valid = r < (XM ? (int64_t)A.item_end[item] : g_len);
    const int64_t i = valid ? rdet[g_beg + r] : 0;
    const Str<W> Bi = load_str<W>(A.bstr, b);
    const Str<W> Ai = valid ? load_str<W>(rstr, g_beg + r) : Str<W>{};
    RowAcc<MODE, K> R;
    row_begin(R, A, i, valid);
    R.ka = k_active ? k_active : (A.k_active ? A.k_active : K);
    if (XM && A.n_old > 0) {
        // old rows: the new members of the own beta group (same-spin alpha excitations)
        if (valid)
            old_row_suffix<W, MODE, K>(R, A, I, Q, Ai, Bi, A.gb_str, A.gb_det, A.gb_new[b], g_beg + g_len,
                                       cand_local);
        row_end<W, MODE, K>(R, A, I, Q, Ai, Bi, i, valid);
        return;
    }
    for (int64_t t0 = 0; t0 < g_len; t0 += ENUM_TILE) {
        const int cnt = (int)min((int64_t)ENUM_TILE, g_len - t0);
        stage<W>(T, A.gb_str, A.gb_det, g_beg + t0, cnt, need_det);
        __syncthreads();
        if (valid) {
            cand_local += lane == 0 ? cnt : 0;
            for (int b0 = 0; b0 < cnt; b0 += 32) {
                const int e = b0 + lane;
                bool match = false;
                Str<W> Aj{};
                if (e < cnt) {
                    Aj = tile_str<W>(T, e);
                    const int d = xor_popc<W>(Ai, Aj);
                    match = (d == 2) | (d == 4);
                }
                emit<W, MODE, K>(R, A, I, Q, Ai, Bi, match, match && need_det ? T.det[e] : 0, Aj, 0);
            }
        }
        __syncthreads();
    }
    row_end<W, MODE, K>(R, A, I, Q, Ai, Bi, i, valid);
}

template <int W>
struct EnumSmem {
    Tile<W> T;
    WarpQueue<W> Q[ENUM_NW];
};

// CTAs per SM the on-the-fly sigma kernels are compiled for (a register cap
// of 65536 / (256 * SHCI_OTF_MINB) per thread); the other modes leave the
// register count to the compiler
#ifndef SHCI_OTF_MINB
#define SHCI_OTF_MINB 5
#endif
template <int MODE>
struct EnumMinBlocks {
    static constexpr int value = MODE == ENUM_SIGMA ? SHCI_OTF_MINB : 1;
};

// persistent grids: CTAs take work items from an atomic counter
template <int W, int MODE, int K>
__global__ void __launch_bounds__(ENUM_THREADS, EnumMinBlocks<MODE>::value) k_enum_alpha(EnumArgs A, DevInts I) {
    __shared__ EnumSmem<W> S;
    __shared__ int item_sh;
    unsigned long long cand_local = 0;
    while (true) {
        if (threadIdx.x == 0) item_sh = atomicAdd(A.work_counter, 1);
        __syncthreads();
        const int64_t item = item_sh;
        __syncthreads();
        if (item >= A.n_items) break;
        enum_alpha_item<W, MODE, K>(A, I, item, S.T, S.Q[threadIdx.x >> 5], cand_local);
    }
    if (ModeOf<MODE>::count && (threadIdx.x & 31) == 0 && cand_local) atomicAdd(A.cand, cand_local);
}

template <int W, int MODE, int K>
__global__ void __launch_bounds__(ENUM_THREADS, EnumMinBlocks<MODE>::value) k_enum_beta(EnumArgs A, DevInts I) {
    __shared__ EnumSmem<W> S;
    __shared__ int item_sh;
    unsigned long long cand_local = 0;
    while (true) {
        if (threadIdx.x == 0) item_sh = atomicAdd(A.work_counter, 1);
        __syncthreads();
        const int64_t item = item_sh;
        __syncthreads();
        if (item >= A.n_items) break;
        enum_beta_item<W, MODE, K>(A, I, item, S.T, S.Q[threadIdx.x >> 5], cand_local);
    }
    if (ModeOf<MODE>::count && (threadIdx.x & 31) == 0 && cand_local) atomicAdd(A.cand, cand_local);
}

// work items: one per chunk of ENUM_NW members of each group
static __global__ void k_items_count(const int64_t *__restrict__ off, int64_t n_groups, int64_t *__restrict__ cnt) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_groups; g += (int64_t)gridDim.x * blockDim.x)
        cnt[g] = (off[g + 1] - off[g] + ENUM_NW - 1) / ENUM_NW;
}

static __global__ void k_items_fill(const int64_t *__restrict__ off, const int64_t *__restrict__ start, int64_t n_groups,
                                    int32_t *__restrict__ item_group, int32_t *__restrict__ item_first) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_groups; g += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = (off[g + 1] - off[g] + ENUM_NW - 1) / ENUM_NW;
        for (int64_t t = 0; t < c; t++) {
            item_group[start[g] + t] = (int32_t)g;
            item_first[start[g] + t] = (int32_t)(t * ENUM_NW);
        }
    }
}

// incremental update: items over one part of each determinant-ordered group,
// the old members [0, g_new - off) (part 0) or the new ones (part 1)
static __global__ void k_items_count_part(const int64_t *__restrict__ off, const int64_t *__restrict__ g_new,
                                          int64_t n_groups, int part, int64_t *__restrict__ cnt) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_groups; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = part ? off[g + 1] - g_new[g] : g_new[g] - off[g];
        cnt[g] = (m + ENUM_NW - 1) / ENUM_NW;
    }
}

static __global__ void k_items_fill_part(const int64_t *__restrict__ off, const int64_t *__restrict__ g_new,
                                         const int64_t *__restrict__ start, int64_t n_groups, int part,
                                         int32_t *__restrict__ item_group, int32_t *__restrict__ item_first,
                                         int32_t *__restrict__ item_end) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_groups; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = part ? g_new[g] - off[g] : 0, hi = part ? off[g + 1] - off[g] : g_new[g] - off[g];
        const int64_t c = (hi - lo + ENUM_NW - 1) / ENUM_NW;
        for (int64_t t = 0; t < c; t++) {
            item_group[start[g] + t] = (int32_t)g;
            item_first[start[g] + t] = (int32_t)(lo + t * ENUM_NW);
            item_end[start[g] + t] = (int32_t)hi;
        }
    }
}

}  // namespace shci
