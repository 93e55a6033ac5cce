// Subspace eigen-solver of the Davidson iteration (one CTA per matrix).
#pragma once
#include "common.cuh"

namespace shci {

// Cholesky-QR coefficients for kb (<= SHCI_MAX_K) vectors with Gram matrix S
// (kb x kb, row-major).  Column l is dropped when its component outside the
// span of the accepted earlier columns has squared norm below rel * ref[l]
// (ref: S's diagonal when null).  Writes M (kb x kb) such that the accepted
// columns q_l' = sum_j M[j * kb + l'] t_j are orthonormal (columns l' >=
// count are zero) and returns the number accepted.  Single thread.
__device__ __forceinline__ int cholqr_coef(const double *S, int kb, const double *ref, double rel, double *M) {
    double R[SHCI_MAX_K][SHCI_MAX_K];
    double Mi[SHCI_MAX_K][SHCI_MAX_K];   // Mi[j][l]: coefficient of t_j in q_l
    int acc[SHCI_MAX_K];
    int na = 0;
    for (int l = 0; l < kb; l++)
        for (int j = 0; j < kb; j++) { R[j][l] = 0.0; Mi[j][l] = 0.0; }
    for (int l = 0; l < kb; l++) {
        // R[j][l] for accepted j < l
        for (int x = 0; x < na; x++) {
            int j = acc[x];
            double s = S[j * kb + l];
            for (int y = 0; y < x; y++) s -= R[acc[y]][j] * R[acc[y]][l];
            R[j][l] = s / R[j][j];
        }
        double d = S[l * kb + l];
        for (int x = 0; x < na; x++) d -= R[acc[x]][l] * R[acc[x]][l];
        double r0 = ref ? ref[l] : S[l * kb + l];
        if (!(d > rel * r0) || !(d > 1e-300)) continue;      // numerically dependent: drop
        R[l][l] = sqrt(d);
        // q_l = (t_l - sum_{j acc} R[j][l] q_j) / R[l][l]
        for (int j = 0; j < kb; j++) {
            double v = (j == l) ? 1.0 : 0.0;
            for (int x = 0; x < na; x++) v -= R[acc[x]][l] * Mi[j][acc[x]];
            Mi[j][l] = v / R[l][l];
        }
        acc[na++] = l;
    }
    for (int j = 0; j < kb; j++)
        for (int x = 0; x < kb; x++) M[j * kb + x] = x < na ? Mi[j][acc[x]] : 0.0;
    return na;
}

// Eigen-decomposition of the symmetric m x m matrix G (row-major, leading
// dimension ld) by cyclic Jacobi with Brent-Luk parallel ordering (m/2
// disjoint rotations per round).
//
// Warm start: when m_prev > 0, evec holds the eigenvectors of G's leading
// m_prev x m_prev block from the previous call (G only grew since), so in
// the basis blockdiag(evec, I) the leading block is diag(eval) and only the
// new border has to be transformed.  Rotations whose off-diagonal element is
// below 1e-14 (|a_pp| + |a_qq|) become the identity, a round with none active
// is skipped, and sweeps stop when one applies no rotation.  A round applies
// its active rotations in one pass over the 2 x 2 blocks they touch (two
// barriers per round).  One SM issues few FP64 instructions (a warp-wide FP64
// instruction occupies its FP64 pipe for many cycles), so no FP64 work is
// spent on identity blocks and the work is packed into few warps.  Output:
// eigenvalues (the converged diagonal) ascending and eigenvectors as columns,
// evec[l * ld + a] = component a of vector l.
//
// The working matrix A lives in shared memory (jsm).  The accumulated
// rotation Q lives there too (QSHARED, JACOBI_SMEM bytes in all), or in the
// global scratch qg of JACOBI_Q_DOUBLES doubles owned by the calling CTA
// (JACOBI_SMEM_A bytes of shared memory), accessed through L2.
template <bool QSHARED = true>
__device__ __forceinline__ void jacobi_solve(const double *G, int ld, int m, int m_prev,
                                             double *__restrict__ eval, double *__restrict__ evec, double *jsm,
                                             double *qg = nullptr) {
    constexpr int QL = SHCI_MAX_SUB + 1;
    double (*A)[QL] = reinterpret_cast<double (*)[QL]>(jsm);
    double *Qp = QSHARED ? jsm + SHCI_MAX_SUB * QL : qg;
    auto qget = [&](int r, int c) { return QSHARED ? Qp[r * QL + c] : __ldcg(&Qp[r * QL + c]); };
    auto qset = [&](int r, int c, double v) {
        if (QSHARED) Qp[r * QL + c] = v;
        else __stcg(&Qp[r * QL + c], v);
    };
    __shared__ double cs[SHCI_MAX_SUB / 2], sn[SHCI_MAX_SUB / 2];
    __shared__ int pp[SHCI_MAX_SUB / 2], qq[SHCI_MAX_SUB / 2];
    __shared__ double lam[SHCI_MAX_SUB];
    const int mm = (m + 1) & ~1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mp = (m_prev > 0 && m_prev <= m) ? m_prev : 0;
    // G is read symmetrised, (G + G^T) / 2, from L2 (ld.global.cg: the caller may
    // have written it earlier in the same kernel)
    auto gs = [&](int r, int c) { return 0.5 * (__ldcg(&G[r * ld + c]) + __ldcg(&G[c * ld + r])); };
    // Q = blockdiag(previous eigenvectors, I)
    for (int e = tid; e < mm * mm; e += nt) {
        int r = e / mm, c = e % mm;
        double q = (r == c) ? 1.0 : 0.0;
        if (r < mp && c < mp) q = __ldcg(&evec[c * ld + r]);
        qset(r, c, q);
    }
    __syncthreads();
    // A = Q^T G Q: leading block diag(previous eigenvalues), border transformed, trailing block copied
    for (int e = tid; e < mm * mm; e += nt) {
        int r = e / mm, c = e % mm;
        double v = 0.0;
        if (r < m && c < m) {
            if (r < mp && c < mp) {
                v = (r == c) ? __ldcg(&eval[r]) : 0.0;
            } else if (r < mp) {          // (Q^T G)[r][c] for border column c
                for (int s = 0; s < mp; s++) v = fma(qget(s, r), gs(s, c), v);
            } else if (c < mp) {
                for (int s = 0; s < mp; s++) v = fma(qget(s, c), gs(r, s), v);
            } else {
                v = gs(r, c);
            }
        }
        A[r][c] = v;
    }
    __syncthreads();
    if (mm != m && tid == 0) {
        // padding index: decoupled, with a diagonal value above every Gershgorin bound
        double bound = 0.0;
        for (int r = 0; r < m; r++) {
            double s = 0.0;
            for (int c = 0; c < m; c++) s += fabs(A[r][c]);
            bound = fmax(bound, s);
        }
        A[m][m] = 2.0 * bound + 1.0;
    }
    __syncthreads();
    const int half = mm / 2;                 // <= 32: the rotations of a round fit one warp
    __shared__ int act_idx[SHCI_MAX_SUB / 2];
    __shared__ int act_pos[SHCI_MAX_SUB / 2];
    __shared__ int n_act[2];
    for (int sweep = 0; sweep < 30; sweep++) {
        int swept = 0;
        for (int round = 0; round < mm - 1; round++) {
            // warp 0: the round's mm/2 disjoint pairs, their rotations and the list of
            // active ones (an inactive pair is the identity)
            if (tid < 32) {
                int active = 0;
                if (tid < half) {
                    int x = tid, y = mm - 1 - tid;
                    int p = x == 0 ? 0 : ((x - 1 + round) % (mm - 1)) + 1;
                    int q = y == 0 ? 0 : ((y - 1 + round) % (mm - 1)) + 1;
                    if (p > q) { int t = p; p = q; q = t; }
                    const double apq = A[p][q];
                    double c = 1.0, s = 0.0;
                    if (fabs(apq) > 1e-14 * (fabs(A[p][p]) + fabs(A[q][q])) + 1e-300) {
                        active = 1;
                        const double diff = A[q][q] - A[p][p];
                        const float tauf = (float)diff / (2.0f * (float)apq);
                        if (fabs(apq) > 1e-30 && isfinite(tauf)) {
                            // rotation angle in FP32 (an FP64 divide or square root is a long
                            // chain of FP64 instructions, and one SM issues few of those),
                            // then (c, s) renormalised in FP64 so that c^2 + s^2 = 1 to FP64
                            // precision: the rotation stays exactly orthogonal and zeroes
                            // a_pq to ~1e-7 relative, which the next sweep finishes
                            const float tf = copysignf(1.0f, tauf) / (fabsf(tauf) + sqrtf(1.0f + tauf * tauf));
                            const float cf = rsqrtf(1.0f + tf * tf);
                            c = (double)cf;
                            s = (double)(tf * cf);
                            double f = 1.5 - 0.5 * (c * c + s * s);
                            c *= f;
                            s *= f;
                            f = 1.5 - 0.5 * (c * c + s * s);
                            c *= f;
                            s *= f;
                        } else {
                            const double tau = diff / (2.0 * apq);
                            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                            c = 1.0 / sqrt(1.0 + t * t);
                            s = t * c;
                        }
                    }
                    cs[tid] = c;
                    sn[tid] = s;
                    pp[tid] = p;
                    qq[tid] = q;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, active);
                const int pos = __popc(mask & ((1u << tid) - 1u));
                if (active) act_idx[pos] = tid;
                if (tid < half) act_pos[tid] = active ? pos : -1;
                if (tid == 0) n_act[round & 1] = __popc(mask);
            }
            __syncthreads();
            const int na = n_act[round & 1];       // double-buffered: warp 0 may run ahead
            if (na == 0) continue;                 // uniform
            swept = 1;
            // A <- J^T A J in one pass over 2 x 2 blocks (rows of pair t, columns of
            // pair u): a block depends only on itself and on rotations t and u.  Only
            // blocks touched by an active rotation are computed, enumerated densely
            // (active t, any u; the block of two active pairs once) so that the FP64
            // work sits in as few warps as possible; the block u, t is written as
            // the transpose, which keeps A exactly symmetric.
            for (int e = tid; e < na * half; e += nt) {
                const int x = e / half, u = e - x * half;
                const int t = act_idx[x];
                const int pu = act_pos[u];
                if (pu >= 0 && pu < x) continue;
                const int p = pp[t], q = qq[t], r = pp[u], v = qq[u];
                const double ct = cs[t], st = sn[t], cu = cs[u], su = sn[u];
                const double apr = A[p][r], apv = A[p][v], aqr = A[q][r], aqv = A[q][v];
                const double bpr = ct * apr - st * aqr, bpv = ct * apv - st * aqv;   // rows
                const double bqr = st * apr + ct * aqr, bqv = st * apv + ct * aqv;
                const double npr = cu * bpr - su * bpv, npv = su * bpr + cu * bpv;  // columns
                const double nqr = cu * bqr - su * bqv, nqv = su * bqr + cu * bqv;
                if (t == u) {                      // r = p, v = q
                    A[p][p] = npr;
                    A[q][q] = nqv;
                    A[p][q] = npv;
                    A[q][p] = npv;
                } else {
                    A[p][r] = npr;
                    A[p][v] = npv;
                    A[q][r] = nqr;
                    A[q][v] = nqv;
                    A[r][p] = npr;
                    A[v][p] = npv;
                    A[r][q] = nqr;
                    A[v][q] = nqv;
                }
            }
            // Q <- Q J over the active rotations
            for (int e = tid; e < mm * na; e += nt) {
                const int i = e / na, t = act_idx[e - i * na];
                const int p = pp[t], q = qq[t];
                const double c = cs[t], s = sn[t];
                const double qp = qget(i, p), qv = qget(i, q);
                qset(i, p, c * qp - s * qv);
                qset(i, q, s * qp + c * qv);
            }
            __syncthreads();
        }
        if (!swept) break;               // uniform
    }
    for (int a = tid; a < mm; a += nt) lam[a] = A[a][a];
    __syncthreads();
    // sort ascending (rank by value, ties by index) and write out the first m
    for (int a = tid; a < mm; a += nt) {
        double va = lam[a];
        int rank = 0;
        for (int b = 0; b < mm; b++) {
            double vb = lam[b];
            rank += (vb < va) || (vb == va && b < a);
        }
        if (rank < m) {
            eval[rank] = va;
            for (int r = 0; r < m; r++) evec[rank * ld + r] = qget(r, a);
        }
    }
}

constexpr size_t JACOBI_SMEM_A = sizeof(double) * SHCI_MAX_SUB * (SHCI_MAX_SUB + 1);
constexpr size_t JACOBI_SMEM = 2 * JACOBI_SMEM_A;
constexpr int JACOBI_Q_DOUBLES = SHCI_MAX_SUB * (SHCI_MAX_SUB + 1);

}  // namespace shci
