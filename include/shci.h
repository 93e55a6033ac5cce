/*
 * shci.h -- C ABI of the GB300 library for the variational hot path of fast
 * semistochastic heat-bath configuration interaction (Li, Otten, Holmes,
 * Sharma, Umrigar, arXiv:1809.04600).
 *
 * The library holds one Hamiltonian (integrals) and one variational space V
 * (a list of determinants) per context.  It finds every connected determinant
 * pair of V, evaluates the Slater-Condon element H_ij with its fermionic sign,
 * applies sigma = H c (from a stored sparse H or recomputed on the fly) and
 * runs a diagonally preconditioned Davidson solver for the lowest roots.  All
 * arithmetic on matrix elements and vectors is IEEE binary64.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Determinants: uint64 rows of 2*W words, W = ceil(n_orb / 64): the alpha
 *   string's W words, then the beta string's W words.  Spatial orbital n of a
 *   string is bit (n & 63) of word (n >> 6) (Sec. V.A).  n_orb <= 128.
 * - Fermionic sign convention: |D> = prod_{alpha occupied, ascending} a+ *
 *   prod_{beta occupied, ascending} a+ |0>.  Eigenvalues and |H_ij| do not
 *   depend on this choice; signed results are self-consistent under it.
 * - Hamiltonian: H = E_core + sum h_pq a+_ps a_qs
 *                  + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs  (real orbitals).
 * - Integrals: h is n_orb*n_orb row-major (symmetric); eri_packed holds the
 *   chemists' (pq|rs) with 8-fold symmetry: pq = p(p+1)/2 + q (p >= q),
 *   slot = PQ(PQ+1)/2 + RS (PQ >= RS); length npair(npair+1)/2 with
 *   npair = n_orb(n_orb+1)/2.
 * - Vectors are float64 [k][n_det] (vector-major).
 * - mem_space: SHCI_MEM_HOST for host pointers (pageable or pinned; the call
 *   copies through the context's stream and synchronises before returning),
 *   SHCI_MEM_DEVICE for pointers on the context's device.
 * - Ownership: the library never frees a caller pointer.  It owns copies of
 *   the integrals and determinants, the helper lists, the stored H and its
 *   workspaces until the next build or shci_destroy.
 * - Errors: every int-returning call returns an shci_status; on failure
 *   shci_last_error() describes it.  The library never exits or aborts.
 *   Device-side waits are bounded, so a failing call leaves no sticky CUDA
 *   error behind (a genuine device fault still would: SHCI_ERR_CUDA).
 * - Streams: all device work runs on the context's stream (the one passed to
 *   shci_create, or a stream the context creates).  Calls return after the
 *   work they enqueue has completed unless stated otherwise.
 */
#ifndef SHCI_H
#define SHCI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shci_ctx shci_ctx;

enum shci_status {
    SHCI_OK = 0,
    SHCI_ERR_INVALID = 1,        /* bad argument or input (sizes, popcounts, duplicates) */
    SHCI_ERR_OOM = 2,            /* device allocation failed */
    SHCI_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    SHCI_ERR_NOT_CONVERGED = 4,  /* Davidson hit max_iter; best estimates returned */
    SHCI_ERR_TIMEOUT = 5,        /* a bounded device wait ran out */
    SHCI_ERR_STATE = 6           /* call out of order (e.g. sigma before build) */
};

enum shci_mem_space { SHCI_MEM_HOST = 0, SHCI_MEM_DEVICE = 1 };

/* How H is applied (Sec. III; Sec. VIII for the on-the-fly product):
 * SHCI_STORED      both triangles as sparse rows, 12 bytes per nonzero (the
 *                  product is a pure gather, the fastest form);
 * SHCI_STORED_UPPER the upper triangle alone, as the paper stores H: half the
 *                  memory, the transposed half added with atomic adds
 *                  (summation order then varies between runs);
 * SHCI_ON_THE_FLY  recomputed each product, nothing stored;
 * SHCI_AUTO        the first of the three whose storage fits 80 % of the
 *                  device's free memory (and the batch budget, in a batch). */
enum shci_mode { SHCI_STORED = 0, SHCI_ON_THE_FLY = 1, SHCI_AUTO = 2, SHCI_STORED_UPPER = 3 };

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * on that device (NULL: the context creates and owns a non-blocking stream).
 * Returns SHCI_ERR_INVALID for a bad device, SHCI_ERR_CUDA otherwise. */
int shci_create(shci_ctx **out, int device, void *cuda_stream);

/* Free every device buffer the context owns.  NULL is ignored. */
void shci_destroy(shci_ctx *ctx);

/* Message for the last failing call on this context ("" if none).  Valid
 * until the next call on the context.  ctx == NULL gives the message of the
 * last failed shci_create in this thread. */
const char *shci_last_error(const shci_ctx *ctx);

/* Load the Hamiltonian's integrals (the one- and two-electron integrals the
 * method takes as input, Sec. II; real orbitals, chemists' notation).
 * n_orb in [1, 128].  Invalidates any previous build.  Returns
 * SHCI_ERR_INVALID if h is not symmetric to 1e-12. */
int shci_load_integrals(shci_ctx *ctx, int n_orb, double e_core, const double *h,
                        const double *eri_packed, int mem_space);

/* Build the connectivity of V = dets[0 .. n_det) (Sec. III): helper lists
 * (unique alpha/beta strings, per-string determinant lists, alpha-single
 * lists; Table I), the cached diagonal H_ii (Sec. V.B) and, in SHCI_STORED
 * mode, every off-diagonal H_ij != structural zero in both triangles (in
 * SHCI_STORED_UPPER mode those with i < j).
 * dets: [n_det][2W] uint64 as above, every alpha string with n_alpha bits and
 * every beta string with n_beta bits below n_orb; determinants must be
 * distinct (SHCI_ERR_INVALID otherwise).  n_det in [1, 2^31 - 1].
 * *nnz_upper_out (may be NULL) receives the number of connected pairs i < j,
 * i.e. the upper-triangle nonzeros.  In SHCI_ON_THE_FLY mode the count pass
 * still runs, so the count is exact.  Determinant order is the caller's. */
int shci_build_connectivity(shci_ctx *ctx, int n_alpha, int n_beta, int64_t n_det,
                            const uint64_t *dets, int mem_space, int mode,
                            int64_t *nnz_upper_out);

/* Grow V by n_new determinants (Sec. III): V becomes dets[0 .. n_old) followed
 * by new_dets[0 .. n_new) (same layout and rules as shci_build_connectivity;
 * they must differ from V's and from one another), new determinant j taking
 * index n_old + j.  The helper lists and the diagonal are rebuilt for the
 * whole of V.  When n_new < full_fraction * (n_old + n_new) the update is
 * incremental: only the old-new and new-new elements are evaluated (each old
 * row screens only the new members of its candidate lists, held in
 * determinant order for this pass), and the stored rows of old determinants
 * are copied with their new elements appended, so row i of the stored matrix
 * holds its old elements first.  Otherwise V is rebuilt from scratch
 * (per-string lists in beta order, occupancy-bitmap lookups).  The paper's
 * switch between the two list orders sits at 20 %; full_fraction <= 0 takes
 * 0.2.  The mode of the last build is kept (SHCI_AUTO re-decides against the
 * memory left: a stored matrix whose grown form no longer fits goes to the
 * next form of SHCI_AUTO's order, V being rebuilt when both triangles give
 * way to the upper one); SHCI_ON_THE_FLY contexts get the count only.  n_new = 0 is a
 * no-op.  *nnz_upper_out (may be NULL) as for shci_build_connectivity.
 * SHCI_ERR_STATE without a completed build; SHCI_ERR_INVALID, with the
 * context unchanged, for an unknown mem_space, n_new < 0, a NULL pointer with
 * n_new > 0 or n_old + n_new > 2^31 - 1.  Any later error (SHCI_ERR_INVALID
 * for a determinant with the wrong electron count or already in V, out of
 * memory, a CUDA error) leaves the context unbuilt: SHCI_ERR_STATE from the
 * calls that need a build until the next shci_build_connectivity. */
int shci_extend_connectivity(shci_ctx *ctx, int64_t n_new, const uint64_t *new_dets, int mem_space,
                             double full_fraction, int64_t *nnz_upper_out);

/* The cached diagonal H_ii, [n_det]. */
int shci_get_diag(shci_ctx *ctx, double *diag, int mem_space);

/* Export the stored upper triangle as (i, j, H_ij), i < j, rows ascending and
 * each row in ascending j.  Host buffers of capacity `cap`; *n_out receives
 * the pair count (nothing is written when cap < count).  For parity checks
 * and debugging; SHCI_ERR_STATE unless built in SHCI_STORED or
 * SHCI_STORED_UPPER mode. */
int shci_get_pairs(shci_ctx *ctx, int64_t cap, int64_t *i_out, int64_t *j_out,
                   double *hij_out, int64_t *n_out);

/* One stored row of the full symmetric H without its diagonal: the connected
 * columns j != row in ascending order and their H_ij (host buffers of
 * capacity `cap`; *n_out receives the row length, nothing is written when
 * cap is smaller).  For sampled-row parity checks on large spaces;
 * SHCI_ERR_STATE unless built in SHCI_STORED mode (an upper-triangle matrix
 * does not hold a row's lower part as a row). */
int shci_get_row(shci_ctx *ctx, int64_t row, int64_t cap, int64_t *cols, double *vals, int64_t *n_out);

/* sigma = H c for k vectors (k in [1, 8]), c and sigma [k][n_det] (Sec. V.B:
 * the matrix-vector product of the Davidson step).  Uses the stored H, or the
 * on-the-fly product in SHCI_ON_THE_FLY mode.  c and sigma must not overlap.
 * Repeated calls give bitwise-identical results except in SHCI_STORED_UPPER
 * mode, whose atomic adds change the summation order (a few ulp). */
int shci_sigma(shci_ctx *ctx, int k, const double *c, double *sigma, int mem_space);

/* sigma = H c like shci_sigma, for device pointers only, with no device
 * allocation of any kind.  The paper has no counterpart: this entry point is
 * for callers that cannot let a library call cudaMalloc -- a process whose
 * device memory is already handed to another allocator (a framework's caching
 * pool that reserved nearly all of HBM, where a cudaMalloc fails), or a
 * latency-critical loop that must not pay the device-wide synchronisation of
 * cudaMalloc / cudaFree.
 * Its layout scratch is one file-scope __device__ array of 2 x 524,288
 * doubles (8 MiB), held on every GPU that loads the library until exit.
 * Set-up: shci_create, with the context's device current, looks up the
 * array's device address and loads the kernels this call launches, so that
 * with lazy module loading the array's memory is taken there and no call of
 * this entry point allocates.  Should that look-up fail in shci_create, the
 * first call on the device retries it (and reports a failure as
 * SHCI_ERR_CUDA), and that call then loads the module and takes the array's
 * memory itself.
 * Requirements: built in SHCI_STORED mode (SHCI_ERR_STATE otherwise), k in
 * [1, 8], k * n_det <= 524,288 (SHCI_ERR_INVALID otherwise, before any
 * launch), c and sigma device [k][n_det], not overlapping.  All calls share
 * the array, which keeps the last call's contents, so calls that overlap on
 * the GPU (other streams, contexts or threads) race; nothing in it needs to
 * start at zero, since every element a call reads was written earlier in that
 * call.  The caller's current device is restored before returning.
 * Synchronises the context's stream before returning. */
int shci_sigma_noalloc(shci_ctx *ctx, int k, const double *c, double *sigma);

/* Lowest k_roots (in [1, 8]) eigenpairs of H on V by diagonally
 * preconditioned Davidson (Sec. II.A).  Converged when, for every root, the
 * Ritz value moved by less than `tol` since the previous iteration and the
 * residual norm ||H x - theta x|| is below 0.1 * sqrt(tol), or the residual
 * norm is below 1e-3 of that bound (the Ritz value is then exact to rounding).  A root that meets
 * both conditions adds no further correction vector while the others
 * converge (its Ritz value and residual are still checked every iteration).
 * guess: NULL (start from the k_roots lowest eigenvectors of H restricted to
 * the min(64, n_det) determinants of lowest H_ii, ties by index) or
 * [k_roots][n_det] starting vectors (orthonormalised by the call), in
 * mem_space.  Like any Davidson iteration it can settle on an excited root
 * when the start overlaps the lowest ones poorly, and it keeps every symmetry
 * of H that the start has: a guess steers it.  energies: host [k_roots], ascending.  vecs: [k_roots][n_det]
 * orthonormal Ritz vectors in mem_space, or NULL.  iters_out may be NULL.
 * Returns SHCI_ERR_NOT_CONVERGED (with the last estimates written) after
 * max_iter iterations. */
int shci_davidson(shci_ctx *ctx, int k_roots, double tol, int max_iter, const double *guess,
                  double *energies, double *vecs, int mem_space, int *iters_out);

/* Convergence history of the last shci_davidson on this context (no paper
 * counterpart; for reports such as the time to reach a given accuracy).
 * Iteration it (0-based, < the returned count) has Ritz values
 * theta[it * k_roots + l], residual norms rnorm[it * k_roots + l] and t_s[it],
 * the host wall time in seconds from the call's entry to the moment those
 * values were known on the host.  Host arrays of at least cap iterations; any
 * may be NULL.  Writes min(cap, iterations) rows and *n_out = the number of
 * iterations recorded (0 before any Davidson run).  SHCI_ERR_INVALID if
 * cap < 0 or n_out is NULL. */
int shci_davidson_history(shci_ctx *ctx, int cap, double *theta, double *rnorm, double *t_s, int *n_out);

/* Heat-bath selection (Sec. II.A, Eq. 2): the determinants D_a outside V for
 * which some D_i in V has |H_ai| * |c_i| >= eps1, |c_i| being the largest
 * |coefficient| of D_i over the k_roots vectors c[k_roots][n_det] (mem_space).
 * Double excitations come from per-orbital-pair lists of |H| sorted in
 * decreasing order (built on the first call after shci_load_integrals), each
 * walked until its elements fall below eps1 / |c_i|; single excitations are
 * evaluated exactly.  The comparison is |H_ai| * |c_i| >= eps1 in FP64.
 * new_dets (mem_space) receives min(cap, count) rows of 2W words in the
 * layout of shci_build_connectivity, ascending as 128W-bit integers whose
 * most significant word is the last (beta word W-1), without repeats; *n_new
 * (host) = count.  cap = 0 with new_dets = NULL queries the count.  Needs a
 * completed shci_build_connectivity (either mode), k_roots in [1, 8], eps1
 * positive and finite, n_orb <= 128; at most 2^32 - 1 candidates before
 * removing repeats (SHCI_ERR_INVALID otherwise: raise eps1). */
int shci_select(shci_ctx *ctx, int k_roots, const double *c, double eps1, int64_t cap, uint64_t *new_dets,
                int64_t *n_new, int mem_space);

/* Screened second-order Epstein-Nesbet energy (Sec. II.B, Eq. 7):
 *   dE2 = sum_{a not in V} (sum_i^{(eps2)} H_ai c_i)^2 / (E_V - H_aa),
 * the inner sum keeping the terms with |H_ai c_i| >= eps2 (FP64), found with
 * the same sorted double-excitation lists as shci_select and exact singles.
 * c: [n_det] coefficients of V (mem_space), e_var: the variational energy
 * E_V (with e_core).  The determinants a are processed in n_batches hash
 * batches (each batch repeats the screen and keeps its own a), so that one
 * batch's terms fit device memory; n_batches = 0 picks the number from the
 * free memory.  *e2 (host) receives dE2, *n_pert (host, may be NULL) the
 * number of determinants a with at least one kept term.  Batches are summed
 * in order and each batch in a fixed order: the result does not depend on
 * timing.  Needs a completed shci_build_connectivity (either mode); eps2
 * positive and finite; n_orb <= 128. */
int shci_pt2(shci_ctx *ctx, const double *c, double e_var, double eps2, int n_batches, double *e2, int64_t *n_pert,
             int mem_space);

/* Draws for the stochastic second-order energy: n_draws indices of V drawn
 * independently with p_i = |c_i| / sum_j |c_j| (Sec. II.B, Eq. 10) by Walker's
 * alias method (table by Vose's two-list construction).  Draw d uses the
 * SplitMix64 output for the counter seed + (d + 1) * 0x9E3779B97F4A7C15: the
 * high 32 bits pick a column, the low 32 bits a uniform in [0, 1).  c:
 * [n_det], draws: [n_draws] int64, both in mem_space. */
int shci_alias_draw(shci_ctx *ctx, const double *c, int64_t n_draws, uint64_t seed, int64_t *draws, int mem_space);

/* The stochastic second-order energy of Sec. II.B (Eq. 9) for n_samples
 * samples of n_d draws each (draws: [n_samples][n_d] indices of V with
 * repeats, in mem_space; c: [n_det] in mem_space, p_i as in shci_alias_draw):
 * for every a outside V, S1 = sum_i w_i c_i H_ai / p_i and
 * S2 = sum_i (w_i (n_d - 1) / p_i - w_i^2 / p_i^2) c_i^2 H_ai^2 over the
 * distinct sampled i (w_i copies) with |H_ai c_i| >= eps, and the sample's
 * value is sum_a (S1^2 + S2) / (E_V - H_aa) / (n_d (n_d - 1)).  out (host,
 * [n_samples][2]) receives the value at eps = eps2 and at eps = eps2_d
 * (0 < eps2 <= eps2_d).  Every draw must index a determinant with c_i != 0;
 * n_d >= 2.  With n_batches > 1 the sum over a is restricted to the hash
 * batch batches[s] (host [n_samples], each in [0, n_batches)) of sample s,
 * the partition of shci_pt2: the batches' values add up to the unrestricted
 * value. */
int shci_pt2_samples(shci_ctx *ctx, const double *c, double e_var, double eps2, double eps2_d, int64_t n_d,
                     int n_samples, const int64_t *draws, double *out, int mem_space, int n_batches,
                     const int *batches);

/* The 3-step perturbation scheme (Sec. IV, Eq. 11):
 *   dE2(eps2) = [dE2^sto(eps2) - dE2^sto(eps2_psto)]
 *             + [dE2^psto(eps2_psto) - dE2^psto(eps2_dtm)] + dE2^dtm(eps2_dtm).
 * dtm: shci_pt2 at eps2_dtm.  psto: all of V at eps2_psto, the perturbative
 * determinants in n_batches_psto (>= 16) hash batches taken in order; per
 * determinant the correction (num_psto^2 - num_dtm^2) / (E_V - H_aa); after
 * each batch the mean and variance of the corrections seen estimate the sum
 * over all determinants (their number extrapolated from the batches done) and
 * the standard deviation of the part not yet evaluated; the loop stops when
 * that is below 0.4 target_error (target 0: every batch, exact).  sto:
 * n_samples samples of n_d alias draws (shci_alias_draw with seed), each with
 * one hash batch out of n_batches_sto drawn from the same counter stream
 * (counters after the determinant draws), value times n_batches_sto; the mean
 * and standard error of the differences eps2 - eps2_psto.  Needs
 * 0 < eps2 <= eps2_psto <= eps2_dtm (equal thresholds skip a step). */
typedef struct {
    double e2, e2_err;         /* total and its standard error */
    double dtm;                /* deterministic part */
    double psto, psto_err;     /* pseudo-stochastic difference and its deviation */
    double sto, sto_err;       /* stochastic difference and its standard error */
    int psto_batches;          /* pseudo-stochastic batches evaluated */
} shci_pt2_3step_t;

int shci_pt2_3step(shci_ctx *ctx, const double *c, double e_var, double eps2, double eps2_psto, double eps2_dtm,
                   double target_error, int n_batches_psto, int n_batches_sto, int64_t n_d, int n_samples,
                   uint64_t seed, shci_pt2_3step_t *out, int mem_space);

/* Semistochastic second-order energy (Sec. II.B, Eq. 8): the deterministic
 * energy at eps2_d (shci_pt2) plus the mean over n_samples samples of n_d
 * alias draws (shci_alias_draw with `seed`) of the difference of the
 * stochastic values at eps2 and at eps2_d (shci_pt2_samples; the same
 * samples, so their noise largely cancels).  *e2 receives the estimate and
 * *e2_err (may be NULL) its standard error over the samples (0 for one
 * sample).  eps2_d = eps2 gives the deterministic energy exactly. */
int shci_pt2_semistochastic(shci_ctx *ctx, const double *c, double e_var, double eps2, double eps2_d, int64_t n_d,
                            int n_samples, uint64_t seed, double *e2, double *e2_err, int mem_space);

/* Adjoint of a variational eigenvalue (no counterpart in the paper, which
 * has no derivatives): for a normalised real eigenvector c of H on V,
 * E = c^T H c and, by Hellmann-Feynman, dE/dX = c^T (dH/dX) c.  Writes
 *   dE_dh[p * n_orb + q]   = grad_out_scale * gamma_pq
 *                            (gamma_pq = sum_s <a+_ps a_qs>; every entry of h
 *                            is treated as an independent variable), and
 *   dE_deri_packed[slot]   = grad_out_scale * 1/2 * sum of Gamma_pqrs over the
 *                            (p,q,r,s) that the packed slot stores
 *                            (Gamma_pqrs = sum_{s,t} <a+_ps a+_rt a_st a_qs>).
 * The pairs of V are enumerated again and H_ij recomputed, never stored.
 * c: [n_det]; outputs n_orb^2 and npair(npair+1)/2 doubles; all in mem_space.
 * Needs a completed shci_build_connectivity (either mode).  The determinant
 * set V is held fixed (no reselection). */
int shci_energy_backward(shci_ctx *ctx, const double *c, double grad_out_scale, double *dE_dh,
                         double *dE_deri_packed, int mem_space);

/* ---------------------------------------------------------------- batches
 * Many independent systems (each with its own integrals and determinant
 * list) solved together (no counterpart in the paper, which treats one
 * system at a time).  shci_batch_create builds every system's helper lists,
 * diagonal and, while the total fits `stored_budget_bytes` (negative: no
 * limit beyond free memory), its stored H -- the rest use the on-the-fly
 * product.  shci_batch_davidson then runs the Davidson iterations of all
 * systems (up to 4 roots each; same stopping rule as shci_davidson) inside
 * one persistent cooperative kernel launch captured in a CUDA graph: each
 * phase of an iteration covers every active system, with grid-wide barriers
 * between phases.  The first call also runs the library's autotuner on a few
 * iterations of the real kernel: rows per stored-sigma work item, the
 * kernel variant (CTAs per SM and register budget) and the stored-row
 * schedule (a warp per determinant, or 8 lanes per determinant).  Systems are limited to n_orb <= 64.  The batch keeps using the
 * creating context's stream; destroy the batch before the context. */
typedef struct shci_batch shci_batch;

typedef struct {
    int n_orb, n_alpha, n_beta;
    int64_t n_det;
    double e_core;
    const double *h;           /* n_orb * n_orb */
    const double *eri_packed;  /* packed as for shci_load_integrals */
    const uint64_t *dets;      /* [n_det][2] (W = 1) */
} shci_system_desc;

typedef struct {
    int n_sys, n_stored, n_on_the_fly;
    int64_t total_det, total_nnz_upper;
    int tuned_rows_per_item, tuned_ctas_per_sm;
    int tuned_lanes_per_row;   /* stored sigma: 32 (a warp per determinant) or 8 */
    double tune_ms;            /* best time of the tuning trials (3 iterations) */
    double solve_ms;           /* last shci_batch_davidson, device time */
    int max_iters;             /* iterations of the slowest system */
    int graph;                 /* 1 if the solve ran as a captured CUDA graph */
    int grid_ctas;
    /* last shci_batch_davidson: device time between consecutive grid barriers,
     * summed over iterations, per phase: 0 start, 1 sigma (stored rows and
     * alpha-grouped items), 2 sigma (beta-grouped items), 3 Gram columns,
     * 4 eigensolver, 5 Ritz vectors and residuals, 6 convergence and restart
     * decision, 7 basis rotation, 8 second-pass coefficients, 9 second
     * projection, 10-12 Cholesky-QR, 13 next block, 14 bookkeeping */
    double phase_ms[16];
    int n_stored_upper;        /* systems stored as their upper triangle (not in n_stored) */
    int tuned_vslice;          /* vector elements per work item of the phases over vectors (8192 or 2048) */
} shci_batch_stats_t;

/* Build every system's connectivity (Sec. III) and decide how each H is held
 * within stored_budget_bytes of device memory (< 0: no budget beyond 80 % of
 * the free memory), 12 bytes per stored nonzero: when the upper triangles of
 * all systems fit, every system is stored, as both triangles for the systems
 * taken in ascending order of pair count while the budget allows and as its
 * upper triangle for the rest; otherwise upper triangles are stored in that
 * order while they fit and the remaining systems are applied on the fly.
 * Systems need n_orb <= 64.  The contexts belong to the batch. */
int shci_batch_create(shci_ctx *ctx, int n_sys, const shci_system_desc *systems, int mem_space,
                      double stored_budget_bytes, shci_batch **out);
/* The mode each system was given (SHCI_STORED, SHCI_STORED_UPPER or
 * SHCI_ON_THE_FLY), host [n_sys]; SHCI_ERR_INVALID if cap < n_sys. */
int shci_batch_get_modes(const shci_batch *b, int cap, int *modes);
/* energies: host [n_sys][k_roots]; iters, converged: host [n_sys] or NULL.
 * SHCI_ERR_NOT_CONVERGED if a system hit max_iter (its estimates are still
 * written); SHCI_ERR_TIMEOUT if the grid barrier gave up. */
int shci_batch_davidson(shci_batch *b, int k_roots, double tol, int max_iter, double *energies, int *iters,
                        int *converged);
int shci_batch_get_stats(shci_batch *b, shci_batch_stats_t *out);
/* Bound of the grid barrier's wait in shci_batch_davidson (no counterpart in
 * the paper): a block that has waited `naps` naps of about 100 ns for the
 * others gives up, every block then leaves the kernel, and the call returns
 * SHCI_ERR_TIMEOUT with the context still usable.  naps < 0 restores the
 * default (2^27 naps, at least ~13 s); 0 gives up at the first wait, which
 * failure-handling tests use to make the bound run out. */
int shci_batch_set_wait_limit(shci_batch *b, long long naps);
void shci_batch_destroy(shci_batch *b);

/* Library-side measurements of the last build / Davidson run (for reports). */
typedef struct {
    int64_t n_det;
    int64_t nnz_upper;          /* connected pairs i < j */
    int64_t n_alpha_strings;    /* unique alpha strings in V */
    int64_t n_beta_strings;
    int64_t n_alpha_singles;    /* entries of the alpha-single lists */
    int64_t candidates;         /* candidate pairs screened per build pass */
    double build_ms;            /* last shci_build_connectivity, device time */
    double sigma_ms_total;      /* sum of sigma-kernel times since reset */
    int64_t sigma_launches;     /* sigma-kernel launches since reset */
    int64_t sigma_vectors;      /* vectors multiplied since reset */
    int64_t kernel_launches;    /* all kernels this context launched since reset */
    int davidson_iters;
    int mode;                   /* SHCI_STORED, SHCI_STORED_UPPER or SHCI_ON_THE_FLY after a build */
    int n_words;                /* W */
    /* last shci_davidson with phase timing on: device-timeline time per part
     * (gaps while the host decides included in the part that follows):
     * 0 start (guess, first product), 1 eigensolver, 2 Ritz vectors and
     * residuals (with the read of the Ritz values), 3 restarts,
     * 4 orthonormalisation, 5 sigma (with layout changes), 6 new Gram columns */
    double davidson_phase_ms[8];
    double select_ms;           /* last shci_select, device time (lists included when built) */
    int64_t select_candidates;  /* last shci_select: candidates before removing repeats and V */
    double pt2_ms;              /* last shci_pt2, device time (lists included when built) */
    int pt2_batches;            /* last shci_pt2: hash batches used */
    int64_t pt2_terms;          /* last shci_pt2: terms H_ai c_i kept by the eps2 screen */
    double extend_ms;           /* last shci_extend_connectivity, device time */
    int extend_incremental;     /* last shci_extend_connectivity: 1 incremental, 0 rebuilt */
    int64_t extend_n_old;       /* last shci_extend_connectivity: determinants before it */
    /* last incremental shci_extend_connectivity, device-timeline time per part:
     * 0 lists (helper lists of the grown V, determinant-ordered groups, work
     * items), 1 count (new elements per row, row offsets), 2 copy (the grown
     * matrix's allocation and the old rows' copy), 3 fill (new elements and
     * the release of the old matrix); zeros after a rebuild */
    double extend_phase_ms[4];
} shci_stats_t;

/* Fill *out.  Kernel times are recorded only while timing is enabled. */
int shci_get_stats(shci_ctx *ctx, shci_stats_t *out);

/* Timing switches (bit mask), and reset of the accumulated counters:
 * bit 0: CUDA-event timing of every sigma launch (synchronises after each);
 * bit 1: per-part timing of shci_davidson (events only, no extra
 * synchronisation).  0 turns both off. */
int shci_set_timing(shci_ctx *ctx, int enable);

#ifdef __cplusplus
}
#endif

#endif /* SHCI_H */
