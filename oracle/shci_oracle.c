/*
 * CPU oracle for the SHCI variational hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs may load this library.  It shares no code with the CUDA library: it is
 * a plain, slow, obviously correct restatement of what the method computes,
 * written in the spin-orbital operator language rather than the alpha/beta
 * string language the GPU kernels use.
 *
 * Conventions (readings of the paper, which does not print them):
 *   - Determinants are bit-packed uint64 words, orbital n at bit (n & 63) of
 *     word (n >> 6) (Sec. V.A); a determinant row is W alpha words then W
 *     beta words.
 *   - Spin-orbital so in [0, 2n): so < n is alpha orbital so, so >= n is beta
 *     orbital so - n.  |D> = prod_{so ascending, occupied} a+_so |0>, i.e. all
 *     alpha creators (ascending) to the left of all beta creators (ascending).
 *   - H = E_core + sum_{PQ} h_PQ a+_P a_Q + 1/2 sum_{PQRS} (PQ|RS) a+_P a+_R a_S a_Q
 *     over spin-orbitals, (PQ|RS) = (pq|rs) delta(s_P,s_Q) delta(s_R,s_S),
 *     chemists' notation, real orbitals, 8-fold packed storage.
 *   - Matrix elements are nonzero only for the diagonal and for single and
 *     double excitations (Sec. III): the Slater-Condon rules below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n;              /* spatial orbitals */
    int W;              /* 64-bit words per spin string */
    double e_core;
    const double *h;    /* n*n row-major */
    const double *eri;  /* packed */
} oints;

/* ------------------------------------------------------------ integrals */

static int64_t pair_of(int p, int q)
{
    if (p < q) { int t = p; p = q; q = t; }
    return (int64_t)p * (p + 1) / 2 + q;
}

/* (pq|rs), chemists' notation, from the 8-fold packed array. */
static double eri_at(const oints *I, int p, int q, int r, int s)
{
    int64_t a = pair_of(p, q), b = pair_of(r, s);
    if (a < b) { int64_t t = a; a = b; b = t; }
    return I->eri[a * (a + 1) / 2 + b];
}

/* spin-orbital helpers */
static int so_spin(const oints *I, int so) { return so >= I->n; }
static int so_orb(const oints *I, int so) { return so >= I->n ? so - I->n : so; }

/* (PQ|RS) over spin-orbitals: zero unless spin(P)=spin(Q) and spin(R)=spin(S). */
static double eri_so(const oints *I, int P, int Q, int R, int S)
{
    if (so_spin(I, P) != so_spin(I, Q) || so_spin(I, R) != so_spin(I, S)) return 0.0;
    return eri_at(I, so_orb(I, P), so_orb(I, Q), so_orb(I, R), so_orb(I, S));
}

static double h_so(const oints *I, int P, int Q)
{
    if (so_spin(I, P) != so_spin(I, Q)) return 0.0;
    return I->h[so_orb(I, P) * I->n + so_orb(I, Q)];
}

/* ------------------------------------------------------------ operators */

static int occ(const oints *I, const uint64_t *d, int so)
{
    int spin = so_spin(I, so), p = so_orb(I, so);
    return (int)((d[spin * I->W + (p >> 6)] >> (p & 63)) & 1u);
}

static void put(const oints *I, uint64_t *d, int so, int v)
{
    int spin = so_spin(I, so), p = so_orb(I, so);
    uint64_t bit = (uint64_t)1 << (p & 63);
    if (v) d[spin * I->W + (p >> 6)] |= bit;
    else d[spin * I->W + (p >> 6)] &= ~bit;
}

/* number of occupied spin-orbitals that precede so in the creator ordering */
static int n_before(const oints *I, const uint64_t *d, int so)
{
    int c = 0;
    for (int t = 0; t < so; t++) c += occ(I, d, t);
    return c;
}

/* a_so |d>: returns the phase (+1/-1) and updates d, or 0 if so is empty. */
static int annihilate(const oints *I, uint64_t *d, int so)
{
    if (!occ(I, d, so)) return 0;
    int ph = (n_before(I, d, so) & 1) ? -1 : 1;
    put(I, d, so, 0);
    return ph;
}

/* a+_so |d>: returns the phase and updates d, or 0 if so is occupied. */
static int create(const oints *I, uint64_t *d, int so)
{
    if (occ(I, d, so)) return 0;
    int ph = (n_before(I, d, so) & 1) ? -1 : 1;
    put(I, d, so, 1);
    return ph;
}

/* ------------------------------------------------------------ Slater-Condon */

static double diag_element(const oints *I, const uint64_t *d)
{
    int nso = 2 * I->n;
    double e = I->e_core;
    for (int k = 0; k < nso; k++) {
        if (!occ(I, d, k)) continue;
        e += h_so(I, k, k);
        for (int l = 0; l < nso; l++) {
            if (!occ(I, d, l)) continue;
            e += 0.5 * (eri_so(I, k, k, l, l) - eri_so(I, k, l, l, k));
        }
    }
    return e;
}

/* <D_i| H |D_j> */
static double matrix_element(const oints *I, const uint64_t *di, const uint64_t *dj)
{
    int nso = 2 * I->n;
    int holes[3], parts[3], nh = 0, np = 0;   /* holes: in j only; particles: in i only */
    for (int so = 0; so < nso; so++) {
        int a = occ(I, di, so), b = occ(I, dj, so);
        if (b && !a) { if (nh < 3) holes[nh] = so; nh++; }
        if (a && !b) { if (np < 3) parts[np] = so; np++; }
    }
    if (nh != np || nh > 2) return 0.0;
    if (nh == 0) return diag_element(I, di);
    uint64_t t[8];
    memcpy(t, dj, sizeof(uint64_t) * 2 * I->W);
    if (nh == 1) {
        int q = holes[0], p = parts[0];
        int ph = annihilate(I, t, q);
        ph *= create(I, t, p);                 /* a+_p a_q |D_j> = ph |D_i> */
        double v = h_so(I, p, q);
        for (int k = 0; k < nso; k++) {
            if (!(occ(I, di, k) && occ(I, dj, k))) continue;   /* common occupied */
            v += eri_so(I, p, q, k, k) - eri_so(I, p, k, k, q);
        }
        return ph * v;
    }
    {
        int q = holes[0], s = holes[1], p = parts[0], r = parts[1];
        int ph = annihilate(I, t, q);
        ph *= annihilate(I, t, s);
        ph *= create(I, t, r);
        ph *= create(I, t, p);                 /* a+_p a+_r a_s a_q |D_j> = ph |D_i> */
        double v = eri_so(I, p, q, r, s) - eri_so(I, p, s, r, q);
        return ph * v;
    }
}

static int exc_degree2(int W, const uint64_t *a, const uint64_t *b)
{
    int c = 0;
    for (int w = 0; w < 2 * W; w++) c += __builtin_popcountll(a[w] ^ b[w]);
    return c;   /* twice the excitation degree */
}

/* ------------------------------------------------------------ exported API */

double oracle_hij(int n, int W, double e_core, const double *h, const double *eri,
                  const uint64_t *di, const uint64_t *dj)
{
    oints I = {n, W, e_core, h, eri};
    return matrix_element(&I, di, dj);
}

void oracle_hdiag(int n, int W, double e_core, const double *h, const double *eri,
                  int64_t n_det, const uint64_t *dets, double *out)
{
    oints I = {n, W, e_core, h, eri};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_det; i++) out[i] = diag_element(&I, dets + i * 2 * W);
}

/*
 * Brute force (a) of Sec. III: loop over all pairs i < j and keep those whose
 * determinants differ by one or two excitations.  Writes up to cap pairs in
 * (i, j) lexicographic order and returns the total count.
 */
int64_t oracle_pairs_allpairs(int64_t n_det, int W, const uint64_t *dets, int64_t cap,
                              int64_t *i_out, int64_t *j_out)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n_det + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_det; i++) {
        int64_t c = 0;
        for (int64_t j = i + 1; j < n_det; j++) {
            int d = exc_degree2(W, dets + i * 2 * W, dets + j * 2 * W);
            if (d == 2 || d == 4) c++;
        }
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n_det; i++) cnt[i + 1] += cnt[i];
    int64_t total = cnt[n_det];
    if (total <= cap) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n_det; i++) {
            int64_t o = cnt[i];
            for (int64_t j = i + 1; j < n_det; j++) {
                int d = exc_degree2(W, dets + i * 2 * W, dets + j * 2 * W);
                if (d == 2 || d == 4) { i_out[o] = i; j_out[o] = j; o++; }
            }
        }
    }
    free(cnt);
    return total;
}

/* ---- open-addressing table from determinant words to index (brute force b) */

typedef struct { int64_t cap; int64_t *slot; const uint64_t *dets; int W; } dtable;

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t det_hash(int W, const uint64_t *d)
{
    uint64_t hsh = 0x9E3779B97F4A7C15ull;
    for (int w = 0; w < 2 * W; w++) hsh = mix64(hsh ^ d[w]);
    return hsh;
}

static int dtable_init(dtable *t, int64_t n_det, int W, const uint64_t *dets)
{
    t->cap = 16;
    while (t->cap < 2 * n_det + 16) t->cap <<= 1;
    t->slot = (int64_t *)malloc(sizeof(int64_t) * t->cap);
    if (!t->slot) return -1;
    for (int64_t s = 0; s < t->cap; s++) t->slot[s] = -1;
    t->dets = dets; t->W = W;
    for (int64_t i = 0; i < n_det; i++) {
        uint64_t s = det_hash(W, dets + i * 2 * W) & (uint64_t)(t->cap - 1);
        while (t->slot[s] >= 0) {
            if (memcmp(dets + t->slot[s] * 2 * W, dets + i * 2 * W, 16 * W) == 0) return -2;
            s = (s + 1) & (uint64_t)(t->cap - 1);
        }
        t->slot[s] = i;
    }
    return 0;
}

static int64_t dtable_find(const dtable *t, const uint64_t *d)
{
    uint64_t s = det_hash(t->W, d) & (uint64_t)(t->cap - 1);
    while (t->slot[s] >= 0) {
        if (memcmp(t->dets + t->slot[s] * 2 * t->W, d, 16 * t->W) == 0) return t->slot[s];
        s = (s + 1) & (uint64_t)(t->cap - 1);
    }
    return -1;
}

/* 0: ok; -2: duplicate determinants */
int oracle_check_unique(int64_t n_det, int W, const uint64_t *dets)
{
    dtable t;
    int rc = dtable_init(&t, n_det, W, dets);
    free(t.slot);
    return rc;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* all determinants of V that one or two excitations of d reach (indices, unsorted) */
static int64_t generate_connections(const oints *I, const dtable *t, const uint64_t *d,
                                    int64_t *out, int64_t cap)
{
    int nso = 2 * I->n;
    int64_t m = 0;
    uint64_t x[8];
    int W2 = 2 * I->W;
    for (int q = 0; q < nso; q++) {
        if (!occ(I, d, q)) continue;
        for (int p = 0; p < nso; p++) {            /* singles q -> p, same spin */
            if (occ(I, d, p) || so_spin(I, p) != so_spin(I, q)) continue;
            memcpy(x, d, 8 * W2); put(I, x, q, 0); put(I, x, p, 1);
            int64_t j = dtable_find(t, x);
            if (j >= 0) { if (m < cap) out[m] = j; m++; }
        }
        for (int s = q + 1; s < nso; s++) {        /* doubles {q,s} -> {p,r} */
            if (!occ(I, d, s)) continue;
            for (int p = 0; p < nso; p++) {
                if (occ(I, d, p)) continue;
                for (int r = p + 1; r < nso; r++) {
                    if (occ(I, d, r)) continue;
                    int nq = so_spin(I, q) + so_spin(I, s), npr = so_spin(I, p) + so_spin(I, r);
                    if (nq != npr) continue;        /* conserve the number of beta electrons */
                    memcpy(x, d, 8 * W2);
                    put(I, x, q, 0); put(I, x, s, 0); put(I, x, p, 1); put(I, x, r, 1);
                    int64_t j = dtable_find(t, x);
                    if (j >= 0) { if (m < cap) out[m] = j; m++; }
                }
            }
        }
    }
    return m;
}

/*
 * Brute force (b) of Sec. III: generate every single and double excitation of
 * each determinant and look it up in V.  Same output contract as
 * oracle_pairs_allpairs.  Returns -2 on duplicate determinants, -1 on OOM.
 */
int64_t oracle_pairs_generate(int n, int64_t n_det, int W, const uint64_t *dets, int64_t cap,
                              int64_t *i_out, int64_t *j_out)
{
    oints I = {n, W, 0.0, NULL, NULL};
    dtable t;
    int rc = dtable_init(&t, n_det, W, dets);
    if (rc) { free(t.slot); return rc; }
    int64_t *cnt = (int64_t *)calloc((size_t)n_det + 1, sizeof(int64_t));
    int64_t max_conn = 0;
    {
        /* bound: singles ne*(2n-ne) plus doubles C(ne,2)*C(2n-ne,2) */
        int64_t ne = 0;
        for (int w = 0; w < 2 * W; w++) ne += __builtin_popcountll(dets[w]);
        int64_t nv = 2 * (int64_t)n - ne;
        max_conn = ne * nv + (ne * (ne - 1) / 2) * (nv * (nv - 1) / 2) + 16;
    }
    int64_t total = 0;
#pragma omp parallel
    {
        int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * max_conn);
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n_det; i++) {
            int64_t m = generate_connections(&I, &t, dets + i * 2 * W, buf, max_conn);
            int64_t c = 0;
            for (int64_t k = 0; k < m; k++) c += buf[k] > i;
            cnt[i + 1] = c;
        }
#pragma omp single
        {
            for (int64_t i = 0; i < n_det; i++) cnt[i + 1] += cnt[i];
            total = cnt[n_det];
        }
        if (total <= cap) {
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < n_det; i++) {
                int64_t m = generate_connections(&I, &t, dets + i * 2 * W, buf, max_conn);
                int64_t o = cnt[i];
                qsort(buf, (size_t)m, sizeof(int64_t), cmp_i64);
                for (int64_t k = 0; k < m; k++)
                    if (buf[k] > i) { i_out[o] = i; j_out[o] = buf[k]; o++; }
            }
        }
        free(buf);
    }
    free(cnt);
    free(t.slot);
    return total;
}

/* H_ij for a list of pairs */
void oracle_hij_list(int n, int W, double e_core, const double *h, const double *eri,
                     const uint64_t *dets, int64_t m, const int64_t *ii, const int64_t *jj,
                     double *out)
{
    oints I = {n, W, e_core, h, eri};
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; k++)
        out[k] = matrix_element(&I, dets + ii[k] * 2 * W, dets + jj[k] * 2 * W);
}

/*
 * Row i of the full Hamiltonian by brute force over all j: the connected
 * columns (j != i, ascending) and their values.  Returns the number of
 * connected columns (writes at most cap).
 */
int64_t oracle_row(int n, int W, double e_core, const double *h, const double *eri,
                   int64_t n_det, const uint64_t *dets, int64_t i, int64_t cap,
                   int64_t *cols, double *vals)
{
    oints I = {n, W, e_core, h, eri};
    int64_t m = 0;
    const uint64_t *di = dets + i * 2 * W;
    for (int64_t j = 0; j < n_det; j++) {
        if (j == i) continue;
        int d = exc_degree2(W, di, dets + j * 2 * W);
        if (d == 2 || d == 4) {
            if (m < cap) { cols[m] = j; vals[m] = matrix_element(&I, di, dets + j * 2 * W); }
            m++;
        }
    }
    return m;
}

/*
 * sigma = H c for the listed rows, by brute force over all columns, with
 * long-double accumulation.  c is [k][n_det]; out is [k][n_rows].
 */
void oracle_sigma_rows(int n, int W, double e_core, const double *h, const double *eri,
                       int64_t n_det, const uint64_t *dets, int k, const double *c,
                       int64_t n_rows, const int64_t *rows, double *out)
{
    oints I = {n, W, e_core, h, eri};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < n_rows; r++) {
        int64_t i = rows[r];
        const uint64_t *di = dets + i * 2 * W;
        long double acc[16];
        for (int v = 0; v < k; v++) acc[v] = 0.0L;
        for (int64_t j = 0; j < n_det; j++) {
            int d = exc_degree2(W, di, dets + j * 2 * W);
            if (d > 4) continue;
            double hij = matrix_element(&I, di, dets + j * 2 * W);
            for (int v = 0; v < k; v++) acc[v] += (long double)hij * c[v * n_det + j];
        }
        for (int v = 0; v < k; v++) out[v * n_rows + r] = (double)acc[v];
    }
}

/*
 * sigma = H c from an upper-triangle pair list (i < j) plus the diagonal, with
 * long-double accumulation (sequential, deterministic).
 */
void oracle_sigma_pairs(int64_t n_det, int64_t m, const int64_t *ii, const int64_t *jj,
                        const double *hij, const double *diag, int k, const double *c,
                        double *out)
{
    long double *acc = (long double *)calloc((size_t)n_det * k, sizeof(long double));
    for (int v = 0; v < k; v++)
        for (int64_t i = 0; i < n_det; i++)
            acc[v * n_det + i] = (long double)diag[i] * c[v * n_det + i];
    for (int64_t p = 0; p < m; p++) {
        int64_t i = ii[p], j = jj[p];
        for (int v = 0; v < k; v++) {
            acc[v * n_det + i] += (long double)hij[p] * c[v * n_det + j];
            acc[v * n_det + j] += (long double)hij[p] * c[v * n_det + i];
        }
    }
    for (int64_t x = 0; x < n_det * k; x++) out[x] = (double)acc[x];
    free(acc);
}

/*
 * The upper triangle of H (Sec. III: elements nonzero only within a double
 * excitation) as compressed rows: row i holds the connected j > i in
 * ascending order, found by brute force (a) over all pairs, with H_ij from the
 * Slater-Condon rules.  With col == NULL, rowptr[0 .. n_det] receives the row
 * offsets (rowptr[0] = 0) and the call returns the total; otherwise rowptr
 * must hold those offsets and col (int32) / val are filled.  Needs
 * n_det < 2^31.
 */
int64_t oracle_upper_csr(int n, int W, double e_core, const double *h, const double *eri, int64_t n_det,
                         const uint64_t *dets, int64_t *rowptr, int32_t *col, double *val)
{
    oints I = {n, W, e_core, h, eri};
    if (!col) {
        rowptr[0] = 0;
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n_det; i++) {
            int64_t cnt = 0;
            for (int64_t j = i + 1; j < n_det; j++) {
                int d = exc_degree2(W, dets + i * 2 * W, dets + j * 2 * W);
                if (d == 2 || d == 4) cnt++;
            }
            rowptr[i + 1] = cnt;
        }
        for (int64_t i = 0; i < n_det; i++) rowptr[i + 1] += rowptr[i];
        return rowptr[n_det];
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_det; i++) {
        int64_t o = rowptr[i];
        const uint64_t *di = dets + i * 2 * W;
        for (int64_t j = i + 1; j < n_det; j++) {
            int d = exc_degree2(W, di, dets + j * 2 * W);
            if (d == 2 || d == 4) {
                col[o] = (int32_t)j;
                val[o] = matrix_element(&I, di, dets + j * 2 * W);
                o++;
            }
        }
    }
    return rowptr[n_det];
}

/*
 * sigma = H c from the upper-triangle rows of oracle_upper_csr plus the
 * diagonal: sigma_i = H_ii c_i + sum_{j>i} H_ij c_j + sum_{j<i} H_ji c_j
 * (H symmetric).  c and out are [k][n_det].  Rows are shared out over threads
 * in fixed contiguous blocks, each thread accumulating into its own copy of
 * sigma; the copies are then added in thread order, so the result depends
 * only on the number of threads.
 */
void oracle_sigma_upper(int64_t n_det, const int64_t *rowptr, const int32_t *col, const double *val,
                        const double *diag, int k, const double *c, double *out)
{
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *part = (double *)calloc((size_t)nthr * n_det * k, sizeof(double));
#pragma omp parallel num_threads(nthr)
    {
        int me = 0, nt = 1;
#ifdef _OPENMP
        me = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        double *acc = part + (size_t)me * n_det * k;
        /* blocks of equal pair counts */
        const int64_t total = rowptr[n_det];
        int64_t lo = 0, hi = n_det;
        {
            const int64_t want_lo = total * me / nt, want_hi = total * (me + 1) / nt;
            int64_t a = 0, b = n_det;
            while (a < b) { int64_t mid = (a + b) / 2; if (rowptr[mid] < want_lo) a = mid + 1; else b = mid; }
            lo = a;
            a = 0; b = n_det;
            while (a < b) { int64_t mid = (a + b) / 2; if (rowptr[mid] < want_hi) a = mid + 1; else b = mid; }
            hi = (me == nt - 1) ? n_det : a;
        }
        for (int64_t i = lo; i < hi; i++) {
            for (int v = 0; v < k; v++) {
                const double *cv = c + (int64_t)v * n_det;
                double *av = acc + (int64_t)v * n_det;
                double si = 0.0;
                for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
                    const int64_t j = col[e];
                    si += val[e] * cv[j];
                    av[j] += val[e] * cv[i];
                }
                av[i] += si;
            }
        }
    }
    for (int v = 0; v < k; v++)
        for (int64_t i = 0; i < n_det; i++) {
            double s = diag[i] * c[(int64_t)v * n_det + i];
            for (int t = 0; t < nthr; t++) s += part[((size_t)t * k + v) * n_det + i];
            out[(int64_t)v * n_det + i] = s;
        }
    free(part);
}

/* ------------------------------------------------------------ density matrices */

/*
 * One- and two-body reduced density matrices of Psi = sum_i c_i |D_i> within V:
 *   gamma_pq    = sum_s <Psi| a+_ps a_qs |Psi>
 *   Gamma_pqrs  = sum_{s,t} <Psi| a+_ps a+_rt a_st a_qs |Psi>
 * by applying the operator string to every |D_i> and projecting on V.  The
 * requested entries are given as index lists (spatial orbitals).
 */
static double rdm1_entry(const oints *I, const dtable *t, int64_t n_det, const uint64_t *dets,
                         const double *c, int p, int q)
{
    long double acc = 0.0L;
    uint64_t x[8];
    int W2 = 2 * I->W;
    for (int spin = 0; spin < 2; spin++) {
        int P = p + spin * I->n, Q = q + spin * I->n;
        for (int64_t i = 0; i < n_det; i++) {
            if (c[i] == 0.0) continue;
            memcpy(x, dets + i * W2, 8 * W2);
            int ph = annihilate(I, x, Q);
            if (!ph) continue;
            ph *= create(I, x, P);
            if (!ph) continue;
            int64_t j = dtable_find(t, x);
            if (j >= 0) acc += (long double)ph * c[j] * c[i];
        }
    }
    return (double)acc;
}

static double rdm2_entry(const oints *I, const dtable *t, int64_t n_det, const uint64_t *dets,
                         const double *c, int p, int q, int r, int s)
{
    long double acc = 0.0L;
    uint64_t x[8];
    int W2 = 2 * I->W;
    for (int s1 = 0; s1 < 2; s1++)
        for (int s2 = 0; s2 < 2; s2++) {
            int P = p + s1 * I->n, Q = q + s1 * I->n, R = r + s2 * I->n, S = s + s2 * I->n;
            for (int64_t i = 0; i < n_det; i++) {
                if (c[i] == 0.0) continue;
                memcpy(x, dets + i * W2, 8 * W2);
                int ph = annihilate(I, x, Q);
                if (!ph) continue;
                ph *= annihilate(I, x, S);
                if (!ph) continue;
                ph *= create(I, x, R);
                if (!ph) continue;
                ph *= create(I, x, P);
                if (!ph) continue;
                int64_t j = dtable_find(t, x);
                if (j >= 0) acc += (long double)ph * c[j] * c[i];
            }
        }
    return (double)acc;
}

/* entries of gamma: idx = [m][2] (p, q); returns 0, or -2 on duplicates */
int oracle_rdm1(int n, int W, int64_t n_det, const uint64_t *dets, const double *c,
                int64_t m, const int32_t *idx, double *out)
{
    oints I = {n, W, 0.0, NULL, NULL};
    dtable t;
    int rc = dtable_init(&t, n_det, W, dets);
    if (rc) { free(t.slot); return rc; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < m; e++)
        out[e] = rdm1_entry(&I, &t, n_det, dets, c, idx[2 * e], idx[2 * e + 1]);
    free(t.slot);
    return 0;
}

/* entries of Gamma: idx = [m][4] (p, q, r, s) */
int oracle_rdm2(int n, int W, int64_t n_det, const uint64_t *dets, const double *c,
                int64_t m, const int32_t *idx, double *out)
{
    oints I = {n, W, 0.0, NULL, NULL};
    dtable t;
    int rc = dtable_init(&t, n_det, W, dets);
    if (rc) { free(t.slot); return rc; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < m; e++)
        out[e] = rdm2_entry(&I, &t, n_det, dets, c, idx[4 * e], idx[4 * e + 1],
                            idx[4 * e + 2], idx[4 * e + 3]);
    free(t.slot);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ heat-bath selection */

/* records of 2W determinant words followed by the bits of the best product;
 * ascending order of the words read as one 128W-bit integer whose most
 * significant word is the last stored word (beta word W-1) */
static int g_sel_words = 2;
static int cmp_det_desc_words(const void *a, const void *b)
{
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    for (int w = g_sel_words - 1; w >= 0; w--) {
        if (x[w] != y[w]) return x[w] < y[w] ? -1 : 1;
    }
    return 0;
}

/*
 * The selection criterion of Sec. II.A (Eq. 2): a determinant D_a outside V is
 * selected when some D_i in V has |H_ai c_i| >= eps1, c_i taken as the largest
 * |coefficient| of D_i over the k given vectors c[k][n_det].  Brute force:
 * every single and double excitation of every D_i is generated, its H_ai
 * evaluated exactly (Slater-Condon, operator form) and the product compared in
 * FP64 as |H_ai| * |c_i| >= eps1.  The selected determinants are written to
 * out (cap rows of 2W words) sorted ascending (last stored word most
 * significant) without repeats, and, when best is not NULL, the largest
 * product |H_ai| |c_i| over V of each; returns their number (which may exceed
 * cap: only cap rows are written), -1 on OOM, -2 on duplicate determinants.
 */
/* Append to buf (records of R = 2W + 1 words, grown by doubling) every
 * determinant outside V that one single or double excitation of d reaches
 * with |H_ad| * ci >= eps1, followed by the bits of that product.  Returns 0,
 * or -1 on OOM. */
static int select_from(const oints *I, const dtable *t, const uint64_t *d, double ci, double eps1,
                       uint64_t **buf, int64_t *m, int64_t *mcap)
{
    const int W2 = 2 * I->W, nso = 2 * I->n, R = 2 * I->W + 1;
    uint64_t x[8];
    for (int q = 0; q < nso; q++) {
        if (!occ(I, d, q)) continue;
        for (int pass = 0; pass < 2; pass++) {
            /* pass 0: singles q -> p; pass 1: doubles {q, s} -> {p, r} */
            for (int s = (pass ? q + 1 : nso); s < (pass ? nso : nso + 1); s++) {
                if (pass && !occ(I, d, s)) continue;
                for (int p = 0; p < nso; p++) {
                    if (occ(I, d, p)) continue;
                    for (int r = (pass ? p + 1 : nso); r < (pass ? nso : nso + 1); r++) {
                        if (pass && occ(I, d, r)) continue;
                        if (!pass && so_spin(I, p) != so_spin(I, q)) continue;
                        if (pass && so_spin(I, q) + so_spin(I, s) != so_spin(I, p) + so_spin(I, r))
                            continue;
                        memcpy(x, d, 8 * W2);
                        put(I, x, q, 0);
                        put(I, x, p, 1);
                        if (pass) { put(I, x, s, 0); put(I, x, r, 1); }
                        if (dtable_find(t, x) >= 0) continue;          /* already in V */
                        const double prod = fabs(matrix_element(I, x, d)) * ci;
                        if (!(prod >= eps1)) continue;
                        if (*m == *mcap) {
                            int64_t nc = 2 * *mcap;
                            uint64_t *nb = (uint64_t *)realloc(*buf, sizeof(uint64_t) * R * nc);
                            if (!nb) return -1;
                            *buf = nb;
                            *mcap = nc;
                        }
                        memcpy(*buf + *m * R, x, 8 * W2);
                        memcpy(*buf + *m * R + W2, &prod, 8);
                        (*m)++;
                    }
                }
            }
        }
    }
    return 0;
}

/*
 * The selection criterion of Sec. II.A (Eq. 2): a determinant D_a outside V is
 * selected when some D_i in V has |H_ai c_i| >= eps1, c_i taken as the largest
 * |coefficient| of D_i over the k given vectors c[k][n_det].  Brute force:
 * every single and double excitation of every D_i is generated, its H_ai
 * evaluated exactly (Slater-Condon, operator form) and the product compared in
 * FP64 as |H_ai| * |c_i| >= eps1.  The selected determinants are written to
 * out (cap rows of 2W words) sorted ascending (last stored word most
 * significant) without repeats, and, when best is not NULL, the largest
 * product |H_ai| |c_i| over V of each; returns their number (which may exceed
 * cap: only cap rows are written), -1 on OOM, -2 on duplicate determinants.
 * The determinants of V are shared out over threads, each collecting its own
 * records; the records are then concatenated and sorted, so the result does
 * not depend on the number of threads.
 */
int64_t oracle_select(int n, int W, double e_core, const double *h, const double *eri, int64_t n_det,
                      const uint64_t *dets, int k, const double *c, double eps1, int64_t cap, uint64_t *out,
                      double *best)
{
    oints I = {n, W, e_core, h, eri};
    dtable t;
    int rc = dtable_init(&t, n_det, W, dets);
    if (rc) { free(t.slot); return rc; }
    const int W2 = 2 * W, R = 2 * W + 1;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    uint64_t **tbuf = (uint64_t **)calloc((size_t)nthr, sizeof(uint64_t *));
    int64_t *tm = (int64_t *)calloc((size_t)nthr, sizeof(int64_t));
    int64_t *tcap = (int64_t *)calloc((size_t)nthr, sizeof(int64_t));
    int failed = 0;
#pragma omp parallel num_threads(nthr)
    {
        int me = 0;
#ifdef _OPENMP
        me = omp_get_thread_num();
#endif
        tcap[me] = 1024;
        tbuf[me] = (uint64_t *)malloc(sizeof(uint64_t) * R * tcap[me]);
        if (!tbuf[me]) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < n_det; i++) {
            if (failed || !tbuf[me]) continue;
            double ci = 0.0;
            for (int l = 0; l < k; l++) ci = fmax(ci, fabs(c[(int64_t)l * n_det + i]));
            if (ci == 0.0) continue;
            if (select_from(&I, &t, dets + i * W2, ci, eps1, &tbuf[me], &tm[me], &tcap[me])) {
#pragma omp atomic write
                failed = 1;
            }
        }
    }
    free(t.slot);
    int64_t m = 0;
    for (int e = 0; e < nthr; e++) m += tm[e];
    uint64_t *buf = failed ? NULL : (uint64_t *)malloc(sizeof(uint64_t) * R * (m > 0 ? m : 1));
    if (buf) {
        int64_t o = 0;
        for (int e = 0; e < nthr; e++) {
            memcpy(buf + o * R, tbuf[e], sizeof(uint64_t) * R * tm[e]);
            o += tm[e];
        }
    }
    for (int e = 0; e < nthr; e++) free(tbuf[e]);
    free(tbuf); free(tm); free(tcap);
    if (!buf) return -1;
    g_sel_words = W2;
    qsort(buf, (size_t)m, sizeof(uint64_t) * R, cmp_det_desc_words);
    int64_t u = 0;
    for (int64_t e = 0; e < m; e++) {
        if (u > 0 && memcmp(buf + (u - 1) * R, buf + e * R, 8 * W2) == 0) {
            double a, b;
            memcpy(&a, buf + (u - 1) * R + W2, 8);
            memcpy(&b, buf + e * R + W2, 8);
            if (b > a) memcpy(buf + (u - 1) * R + W2, &b, 8);
            continue;
        }
        if (u != e) memmove(buf + u * R, buf + e * R, 8 * R);
        u++;
    }
    for (int64_t e = 0; e < u && e < cap; e++) {
        memcpy(out + e * W2, buf + e * R, 8 * W2);
        if (best) memcpy(best + e, buf + e * R + W2, 8);
    }
    free(buf);
    return u;
}

/* ------------------------------------------------------------ Epstein-Nesbet PT2 */

/* records: 2W determinant words, the term H_ai c_i (bits), generation index */
static int cmp_pt_records(const void *a, const void *b)
{
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    for (int w = g_sel_words - 1; w >= 0; w--) {
        if (x[w] != y[w]) return x[w] < y[w] ? -1 : 1;
    }
    return (x[g_sel_words + 1] > y[g_sel_words + 1]) - (x[g_sel_words + 1] < y[g_sel_words + 1]);
}

/*
 * The screened second-order Epstein-Nesbet energy of Sec. II.B (Eq. 7):
 *   dE2 = sum_{a not in V} (sum_i^{(eps2)} H_ai c_i)^2 / (E_V - H_aa),
 * where the inner sum keeps only the terms with |H_ai c_i| >= eps2 (FP64).
 * Brute force: every single and double excitation a of every D_i, the term
 * H_ai c_i by Slater-Condon (operator form), terms gathered per a (sorted by
 * determinant, then by generation order), H_aa from the diagonal rule.
 * *n_pert receives the number of determinants a with at least one term.
 * Returns 0, -1 on OOM, -2 on duplicate determinants.
 */
int oracle_pt2(int n, int W, double e_core, const double *h, const double *eri, int64_t n_det,
               const uint64_t *dets, const double *c, double e_var, double eps2, double *e2, int64_t *n_pert)
{
    oints I = {n, W, e_core, h, eri};
    dtable t;
    int rc = dtable_init(&t, n_det, W, dets);
    if (rc) { free(t.slot); return rc; }
    const int W2 = 2 * W, nso = 2 * n, R = 2 * W + 2;
    int64_t m = 0, mcap = 1024;
    uint64_t *buf = (uint64_t *)malloc(sizeof(uint64_t) * R * mcap);
    if (!buf) { free(t.slot); return -1; }
    uint64_t x[8];
    for (int64_t i = 0; i < n_det; i++) {
        const uint64_t *d = dets + i * W2;
        if (c[i] == 0.0) continue;
        for (int q = 0; q < nso; q++) {
            if (!occ(&I, d, q)) continue;
            for (int pass = 0; pass < 2; pass++) {
                for (int s = (pass ? q + 1 : nso); s < (pass ? nso : nso + 1); s++) {
                    if (pass && !occ(&I, d, s)) continue;
                    for (int p = 0; p < nso; p++) {
                        if (occ(&I, d, p)) continue;
                        for (int r = (pass ? p + 1 : nso); r < (pass ? nso : nso + 1); r++) {
                            if (pass && occ(&I, d, r)) continue;
                            if (!pass && so_spin(&I, p) != so_spin(&I, q)) continue;
                            if (pass && so_spin(&I, q) + so_spin(&I, s) != so_spin(&I, p) + so_spin(&I, r))
                                continue;
                            memcpy(x, d, 8 * W2);
                            put(&I, x, q, 0);
                            put(&I, x, p, 1);
                            if (pass) { put(&I, x, s, 0); put(&I, x, r, 1); }
                            if (dtable_find(&t, x) >= 0) continue;
                            const double term = matrix_element(&I, x, d) * c[i];
                            if (!(fabs(term) >= eps2)) continue;
                            if (m == mcap) {
                                mcap *= 2;
                                uint64_t *nb = (uint64_t *)realloc(buf, sizeof(uint64_t) * R * mcap);
                                if (!nb) { free(buf); free(t.slot); return -1; }
                                buf = nb;
                            }
                            memcpy(buf + m * R, x, 8 * W2);
                            memcpy(buf + m * R + W2, &term, 8);
                            buf[m * R + W2 + 1] = (uint64_t)m;
                            m++;
                        }
                    }
                }
            }
        }
    }
    free(t.slot);
    g_sel_words = W2;
    qsort(buf, (size_t)m, sizeof(uint64_t) * R, cmp_pt_records);
    double sum = 0.0;
    int64_t runs = 0;
    for (int64_t e = 0; e < m;) {
        int64_t f = e;
        double num = 0.0;
        while (f < m && memcmp(buf + f * R, buf + e * R, 8 * W2) == 0) {
            double v;
            memcpy(&v, buf + f * R + W2, 8);
            num += v;
            f++;
        }
        const double haa = diag_element(&I, buf + e * R);
        sum += num * num / (e_var - haa);
        runs++;
        e = f;
    }
    free(buf);
    *e2 = sum;
    *n_pert = runs;
    return 0;
}

/* ------------------------------------------------------------ stochastic PT2 estimator */

/* records: 2W determinant words, then t1, t2, |H_ai c_i| (bits), generation index */
static int cmp_st_records(const void *a, const void *b)
{
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    for (int w = g_sel_words - 1; w >= 0; w--) {
        if (x[w] != y[w]) return x[w] < y[w] ? -1 : 1;
    }
    return (x[g_sel_words + 3] > y[g_sel_words + 3]) - (x[g_sel_words + 3] < y[g_sel_words + 3]);
}

/*
 * One sample of the stochastic second-order energy of Sec. II.B (Eq. 9): the
 * sample holds n_dist distinct determinants sidx[] of V with copy counts sw[]
 * (sum n_d), drawn with p_i = |c_i| / sum_j |c_j| (Eq. 10).  For every a
 * outside V:
 *   S1 = sum_i w_i c_i H_ai / p_i,
 *   S2 = sum_i (w_i (n_d - 1) / p_i - w_i^2 / p_i^2) c_i^2 H_ai^2,
 * both over the sampled i with |H_ai c_i| >= eps, and the sample's value is
 *   sum_a (S1^2 + S2) / (E_V - H_aa) / (n_d (n_d - 1)).
 * out[0]: eps = eps2; out[1]: eps = eps2_d (the same sample, Eq. 8).
 * Returns 0, -1 on OOM, -2 on duplicates in V, -3 on a bad sample.
 */
int oracle_pt2_sample(int n, int W, double e_core, const double *h, const double *eri, int64_t n_det,
                      const uint64_t *dets, const double *c, double e_var, double eps2, double eps2_d, int64_t n_d,
                      int64_t n_dist, const int64_t *sidx, const int64_t *sw, double *out)
{
    if (n_d < 2) return -3;
    oints I = {n, W, e_core, h, eri};
    dtable t;
    int rc = dtable_init(&t, n_det, W, dets);
    if (rc) { free(t.slot); return rc; }
    double csum = 0.0;
    for (int64_t i = 0; i < n_det; i++) csum += fabs(c[i]);
    const int W2 = 2 * W, nso = 2 * n, R = 2 * W + 4;
    int64_t m = 0, mcap = 1024;
    uint64_t *buf = (uint64_t *)malloc(sizeof(uint64_t) * R * mcap);
    if (!buf) { free(t.slot); return -1; }
    uint64_t x[8];
    for (int64_t u = 0; u < n_dist; u++) {
        const int64_t i = sidx[u];
        if (i < 0 || i >= n_det || sw[u] < 1) { free(buf); free(t.slot); return -3; }
        const double pi = fabs(c[i]) / csum, wi = (double)sw[u];
        if (!(pi > 0.0)) { free(buf); free(t.slot); return -3; }
        const double f1 = wi / pi, f2 = wi * (double)(n_d - 1) / pi - wi * wi / (pi * pi);
        const uint64_t *d = dets + i * W2;
        for (int q = 0; q < nso; q++) {
            if (!occ(&I, d, q)) continue;
            for (int pass = 0; pass < 2; pass++) {
                for (int s = (pass ? q + 1 : nso); s < (pass ? nso : nso + 1); s++) {
                    if (pass && !occ(&I, d, s)) continue;
                    for (int p = 0; p < nso; p++) {
                        if (occ(&I, d, p)) continue;
                        for (int r = (pass ? p + 1 : nso); r < (pass ? nso : nso + 1); r++) {
                            if (pass && occ(&I, d, r)) continue;
                            if (!pass && so_spin(&I, p) != so_spin(&I, q)) continue;
                            if (pass && so_spin(&I, q) + so_spin(&I, s) != so_spin(&I, p) + so_spin(&I, r))
                                continue;
                            memcpy(x, d, 8 * W2);
                            put(&I, x, q, 0);
                            put(&I, x, p, 1);
                            if (pass) { put(&I, x, s, 0); put(&I, x, r, 1); }
                            if (dtable_find(&t, x) >= 0) continue;
                            const double hv = matrix_element(&I, x, d);
                            const double mag = fabs(hv) * fabs(c[i]);
                            if (!(mag >= eps2)) continue;
                            const double t1 = f1 * c[i] * hv, t2 = f2 * c[i] * c[i] * hv * hv;
                            if (m == mcap) {
                                mcap *= 2;
                                uint64_t *nb = (uint64_t *)realloc(buf, sizeof(uint64_t) * R * mcap);
                                if (!nb) { free(buf); free(t.slot); return -1; }
                                buf = nb;
                            }
                            memcpy(buf + m * R, x, 8 * W2);
                            memcpy(buf + m * R + W2, &t1, 8);
                            memcpy(buf + m * R + W2 + 1, &t2, 8);
                            memcpy(buf + m * R + W2 + 2, &mag, 8);
                            buf[m * R + W2 + 3] = (uint64_t)m;
                            m++;
                        }
                    }
                }
            }
        }
    }
    free(t.slot);
    g_sel_words = W2;
    qsort(buf, (size_t)m, sizeof(uint64_t) * R, cmp_st_records);
    double sum = 0.0, sum_d = 0.0;
    for (int64_t e = 0; e < m;) {
        int64_t f = e;
        double s1 = 0.0, s2 = 0.0, s1d = 0.0, s2d = 0.0;
        while (f < m && memcmp(buf + f * R, buf + e * R, 8 * W2) == 0) {
            double t1, t2, mag;
            memcpy(&t1, buf + f * R + W2, 8);
            memcpy(&t2, buf + f * R + W2 + 1, 8);
            memcpy(&mag, buf + f * R + W2 + 2, 8);
            s1 += t1;
            s2 += t2;
            if (mag >= eps2_d) { s1d += t1; s2d += t2; }
            f++;
        }
        const double den = e_var - diag_element(&I, buf + e * R);
        sum += (s1 * s1 + s2) / den;
        sum_d += (s1d * s1d + s2d) / den;
        e = f;
    }
    free(buf);
    const double norm = 1.0 / ((double)n_d * (double)(n_d - 1));
    out[0] = sum * norm;
    out[1] = sum_d * norm;
    return 0;
}
