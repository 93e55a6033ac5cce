// The library context and the internal entry points shared by the .cu files.
#pragma once
#include "common.cuh"
#include "prims.cuh"

struct DavidsonWork {
    int n_alloc = 0, m_alloc = 0, k_alloc = 0;
    DevBuf<double> V, AV;        // [m_max][n]
    DevBuf<double> X, Y;         // interleaved block [n][k] (sigma input / output)
    DevBuf<double> T;            // [k][n] corrections / Ritz scratch
    DevBuf<double> RV, RAV;      // [keep][n] thick-restart rotation targets
    DevBuf<double> G;            // [m_max][m_max] projected matrix
    DevBuf<double> evec;         // [m_max][m_max] subspace eigenvectors (column-major)
    DevBuf<double> eval;         // [m_max]
    DevBuf<double> partial;      // block partial sums for dot products
    DevBuf<double> small;        // small device scalars (norms, coefficients)
    DevBuf<unsigned> ctr;        // last-block reduction counters
    DevBuf<double> host_pinned_dummy;
    DevBuf<double> guess_G, guess_vec, guess_val;   // start vectors: the small subspace problem
    double *h_status = nullptr;  // pinned host mirror of the status block
};

// Double excitations from one orbital pair, sorted by decreasing |H| (CSR
// over the pair slot p * n + q): target pair (r | s << 16), |H|, and |H|
// rounded toward zero to FP32 (the sort key).
struct HBList {
    DevBuf<int64_t> off;
    DevBuf<uint32_t> rs;
    DevBuf<double> val;
    DevBuf<float> kf;
    int64_t entries = 0;
};

struct shci_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    int n_sm = 0;

    // integrals
    bool have_ints = false;
    int n_orb = 0;
    double e_core = 0.0;
    DevBuf<double> h, eri, jk1, j1, jdiag, kdiag;
    // heat-bath lists for the selection (built on first use per set of integrals)
    bool hb_valid = false;
    HBList hb_same, hb_opp;

    // variational space and helper lists (Table I)
    bool built = false;
    int mode = SHCI_STORED;
    int mode_req = SHCI_AUTO;              // the mode the last build was asked for
    bool rows_upper = false;               // rowptr / cnt_b count the pairs j > i only
    int W = 1, n_alpha = 0, n_beta = 0;
    int64_t n_det = 0;
    DevBuf<uint64_t> dets;                 // [n][2W]
    int64_t Ua = 0, Ub = 0;                // unique alpha / beta strings
    DevBuf<uint64_t> astr, bstr;           // [U][W]
    DevBuf<int32_t> ia, ib;                // string index of each determinant
    DevBuf<int64_t> ga_off, gb_off;        // determinants grouped by alpha / beta string
    DevBuf<int32_t> ga_det, gb_det;        // member determinant indices
    DevBuf<uint64_t> ga_str, gb_str;       // member beta / alpha strings [m][W]
    DevBuf<int64_t> as_off;                // alpha-single lists over unique alpha strings
    DevBuf<int32_t> as_idx;
    DevBuf<double> diag;                   // H_ii
    // beta-single lists and the (alpha, beta) occupancy bitmap for opposite-spin lookups
    DevBuf<int64_t> bs_off;
    DevBuf<int32_t> bs_idx;
    DevBuf<unsigned long long> occ;
    DevBuf<int32_t> occ_pref;
    int64_t occ_words = 0, n_beta_singles = 0;
    bool opp_lookup = false;               // the occupancy bitmap is built
    bool opp_hybrid = false;               // scan or look up per alpha single
    float opp_factor = 0.5f;               // scan a group of up to this many x the beta singles
    // enumeration work items: chunks of rows of one alpha (beta) group
    DevBuf<int32_t> item_a_group, item_a_first, item_b_group, item_b_first;
    int64_t n_items_a = 0, n_items_b = 0;
    DevBuf<int64_t> cnt_b;                 // entries of the beta-grouped part of each row (build scratch)

    // stored H, both triangles, diagonal separate; after an incremental
    // update a row holds its old elements first, then the new ones
    DevBuf<int64_t> rowptr;
    DevBuf<int32_t> col;
    DevBuf<double> val;
    int64_t nnz_full = 0, nnz_upper = 0;

    // scratch
    shci::SortWork sw;
    DevBuf<uint64_t> sort_keys;
    DevBuf<uint32_t> sort_vals;
    DevBuf<int64_t> i64a, i64b, i64c;
    DevBuf<int32_t> i32a;
    DevBuf<int> counter;                   // dynamic work counters / flags
    DevBuf<double> vec_a, vec_b;           // layout conversion for the ABI sigma

    DavidsonWork dw;

    // SHCI_AUTO stores H only if it fits this many bytes (negative: no limit
    // beyond the device's free memory)
    double stored_budget = -1.0;

    // measurements
    bool timing = false;                   // sigma launches
    bool timing_dav = false;               // parts of shci_davidson
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    shci_stats_t stats{};
    std::vector<double> hist_theta, hist_rn, hist_t;   // last Davidson: per iteration
    int hist_k = 0;
    int64_t candidates = 0;
    int64_t n_alpha_singles = 0;
};

namespace shci {

// integrals.cu / build.cu
void load_integrals(shci_ctx *c, int n_orb, double e_core, const double *h, const double *eri, int mem);
void build(shci_ctx *c, int n_alpha, int n_beta, int64_t n_det, const uint64_t *dets, int mem, int mode);
void extend(shci_ctx *c, int64_t n_new, const uint64_t *new_dets, int mem, double full_fraction);
// store a context built in any mode as SHCI_STORED or SHCI_STORED_UPPER
// (the lists are kept; the rows are recounted when their form differs)
void store(shci_ctx *c, int mode);
void export_pairs(shci_ctx *c, int64_t cap, int64_t *i_out, int64_t *j_out, double *v_out, int64_t *n_out);

// sigma.cu: y = H x for k vectors; `inter` selects the interleaved [n][k]
// layout (otherwise vector-major [k][n]).
void sigma(shci_ctx *c, int k, const double *x, double *y, bool inter);
void sigma_stored_preload();

// noalloc.cu: the allocation-free sigma's per-device set-up (at shci_create)
void noalloc_prepare(int device);

// select.cu: heat-bath selection of new determinants (Sec. II)
void select_dets(shci_ctx *c, int k, const double *coef, double eps1, int64_t cap, uint64_t *out, int64_t *n_out,
                 int mem);
void pt2(shci_ctx *c, const double *coef, double e_var, double eps2, int nbatch, double *e2, int64_t *n_pert,
         int mem);
void alias_draw(shci_ctx *c, const double *coef, int64_t n_draws, uint64_t seed, int64_t *out, int mem);
void pt2_samples(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_d, int64_t n_d,
                 int n_samples, const int64_t *draws, double *out, int mem, int nbatch, const int *batch_of_sample);
void pt2_3step(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_psto, double eps2_dtm,
               double target, int nbatch_psto, int nbatch_sto, int64_t n_d, int n_samples, uint64_t seed,
               shci_pt2_3step_t *out, int mem);
void pt2_semistochastic(shci_ctx *c, const double *coef, double e_var, double eps2, double eps2_d, int64_t n_d,
                        int n_samples, uint64_t seed, double *e2, double *e2_err, int mem);

// davidson.cu
int davidson(shci_ctx *c, int k, double tol, int max_iter, const double *guess, double *energies,
             double *vecs, int mem, int *iters_out);

DevInts dev_ints(const shci_ctx *c);

inline void count_launch(shci_ctx *c, int n = 1) { c->stats.kernel_launches += n; }

}  // namespace shci
