"""CPU oracle for the SHCI variational hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline /
reference legs may import this package.  The product (the CUDA library and its
binding) never imports it, and it never imports the product: the two share only
the seeded input generators of ``shci_synth``.

What it computes, and where the paper defines it:

* ``hij``, ``hdiag``, ``hij_list``, ``row`` -- Hamiltonian matrix elements
  between determinants, nonzero only for the diagonal, single and double
  excitations (Sec. III, the paragraph after Algorithm 2), evaluated with the
  Slater-Condon rules in spin-orbital operator form (``shci_oracle.c``).
* ``pairs_allpairs`` -- brute force (a) of Sec. III: all pairs i < j tested
  for one or two excitations.
* ``pairs_generate`` -- brute force (b) of Sec. III: every single and double
  excitation of each determinant looked up in V.
* ``sigma_rows`` / ``sigma_pairs`` -- sigma = H c (the matrix-vector product of
  the Davidson step, Sec. V.B), long-double accumulation.
* ``lowest_eigenpairs`` -- the lowest roots of H on V (Sec. II.A): a dense
  symmetric eigensolver for small spaces, else a plain diagonally
  preconditioned Davidson iteration (Sec. II.A) on a sparse matrix the oracle
  assembles itself.
* ``rdm1`` / ``rdm2`` / ``energy_gradient`` -- dE/dh_pq = gamma_pq and the
  packed dE/d(pq|rs) from the 1- and 2-body density matrices of the root
  (Hellmann-Feynman for a variational eigenvalue; the paper has no adjoint).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shci_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle's C code into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_hij.restype = ctypes.c_double
        lib.oracle_hij.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p, _u64p, _u64p]
        lib.oracle_hdiag.restype = None
        lib.oracle_hdiag.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p,
                                     ctypes.c_int64, _u64p, _f64p]
        lib.oracle_pairs_allpairs.restype = ctypes.c_int64
        lib.oracle_pairs_allpairs.argtypes = [ctypes.c_int64, ctypes.c_int, _u64p, ctypes.c_int64, _i64p, _i64p]
        lib.oracle_pairs_generate.restype = ctypes.c_int64
        lib.oracle_pairs_generate.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _u64p,
                                              ctypes.c_int64, _i64p, _i64p]
        lib.oracle_check_unique.restype = ctypes.c_int
        lib.oracle_check_unique.argtypes = [ctypes.c_int64, ctypes.c_int, _u64p]
        lib.oracle_hij_list.restype = None
        lib.oracle_hij_list.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p, _u64p,
                                        ctypes.c_int64, _i64p, _i64p, _f64p]
        lib.oracle_row.restype = ctypes.c_int64
        lib.oracle_row.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p, ctypes.c_int64,
                                   _u64p, ctypes.c_int64, ctypes.c_int64, _i64p, _f64p]
        lib.oracle_sigma_rows.restype = None
        lib.oracle_sigma_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p,
                                          ctypes.c_int64, _u64p, ctypes.c_int, _f64p, ctypes.c_int64,
                                          _i64p, _f64p]
        lib.oracle_sigma_pairs.restype = None
        lib.oracle_sigma_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p, _f64p,
                                           ctypes.c_int, _f64p, _f64p]
        lib.oracle_rdm1.restype = ctypes.c_int
        lib.oracle_rdm1.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _u64p, _f64p,
                                    ctypes.c_int64, _i32p, _f64p]
        lib.oracle_rdm2.restype = ctypes.c_int
        lib.oracle_rdm2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _u64p, _f64p,
                                    ctypes.c_int64, _i32p, _f64p]
        lib.oracle_select.restype = ctypes.c_int64
        lib.oracle_select.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p,
                                      ctypes.c_int64, _u64p, ctypes.c_int, _f64p, ctypes.c_double,
                                      ctypes.c_int64, _u64p, _f64p]
        lib.oracle_pt2.restype = ctypes.c_int
        lib.oracle_pt2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p, ctypes.c_int64,
                                   _u64p, _f64p, ctypes.c_double, ctypes.c_double, _f64p, _i64p]
        lib.oracle_pt2_sample.restype = ctypes.c_int
        lib.oracle_pt2_sample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p,
                                          ctypes.c_int64, _u64p, _f64p, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _f64p]
        lib.oracle_upper_csr.restype = ctypes.c_int64
        lib.oracle_upper_csr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, _f64p, ctypes.c_int64,
                                         _u64p, _i64p, _i32p, _f64p]
        lib.oracle_sigma_upper.restype = None
        lib.oracle_sigma_upper.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int, _f64p,
                                           _f64p]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def n_words(dets) -> int:
    return dets.shape[1] // 2


def num_threads() -> int:
    return int(_load().oracle_num_threads())


class System:
    """Integrals of one Hamiltonian, as the oracle sees them."""

    def __init__(self, h, eri_packed, e_core=0.0):
        self.h = _f64(h)
        self.eri = _f64(eri_packed)
        self.e_core = float(e_core)
        self.n = self.h.shape[0]

    # ---------------------------------------------------------- elements
    def hij(self, di, dj) -> float:
        di, dj = _u64(di), _u64(dj)
        W = di.size // 2
        return float(_load().oracle_hij(self.n, W, self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                                        _p(di, _u64p), _p(dj, _u64p)))

    def hdiag(self, dets) -> np.ndarray:
        dets = _u64(dets)
        out = np.empty(dets.shape[0])
        _load().oracle_hdiag(self.n, n_words(dets), self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                             dets.shape[0], _p(dets, _u64p), _p(out, _f64p))
        return out

    def hij_list(self, dets, ii, jj) -> np.ndarray:
        dets, ii, jj = _u64(dets), _i64(ii), _i64(jj)
        out = np.empty(ii.size)
        _load().oracle_hij_list(self.n, n_words(dets), self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                                _p(dets, _u64p), ii.size, _p(ii, _i64p), _p(jj, _i64p), _p(out, _f64p))
        return out

    def row(self, dets, i):
        """(cols, vals) of the off-diagonal row i, ascending columns, brute force."""
        dets = _u64(dets)
        lib = _load()
        cap = 4096
        while True:
            cols = np.empty(cap, np.int64)
            vals = np.empty(cap)
            m = lib.oracle_row(self.n, n_words(dets), self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                               dets.shape[0], _p(dets, _u64p), int(i), cap, _p(cols, _i64p), _p(vals, _f64p))
            if m <= cap:
                return cols[:m].copy(), vals[:m].copy()
            cap = int(m)

    # ---------------------------------------------------------- selection
    def select(self, dets, c, eps1, with_best=False):
        """Determinants outside V selected by the criterion of Sec. II.A (Eq. 2):
        some D_i in V has |H_ai| * max_l |c_l[i]| >= eps1.  Brute force over
        every single and double excitation; rows sorted ascending with the
        last stored word most significant, no repeats.  with_best: also the
        largest product of each over V."""
        dets = _u64(dets)
        c = _f64(np.atleast_2d(c))
        W = n_words(dets)
        lib = _load()
        cap = 1 << 16
        while True:
            out = np.empty((cap, 2 * W), np.uint64)
            best = np.empty(cap)
            m = lib.oracle_select(self.n, W, self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                                  dets.shape[0], _p(dets, _u64p), c.shape[0], _p(c, _f64p), float(eps1),
                                  cap, _p(out, _u64p), _p(best, _f64p))
            if m < 0:
                raise RuntimeError("oracle_select failed (%d)" % m)
            if m <= cap:
                return (out[:m].copy(), best[:m].copy()) if with_best else out[:m].copy()
            cap = int(m)

    def pt2(self, dets, c, e_var, eps2):
        """(dE2, number of perturbative determinants): the screened second-order
        Epstein-Nesbet energy of Sec. II.B (Eq. 7) by brute force."""
        dets = _u64(dets)
        c = _f64(np.ravel(c))
        e2 = np.zeros(1)
        npert = np.zeros(1, np.int64)
        rc = _load().oracle_pt2(self.n, n_words(dets), self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                                dets.shape[0], _p(dets, _u64p), _p(c, _f64p), float(e_var), float(eps2),
                                _p(e2, _f64p), _p(npert, _i64p))
        if rc != 0:
            raise RuntimeError("oracle_pt2 failed (%d)" % rc)
        return float(e2[0]), int(npert[0])

    def pt2_sample(self, dets, c, e_var, eps2, eps2_d, draws):
        """One sample of the stochastic second-order energy of Sec. II.B (Eq. 9)
        at eps2 and at eps2_d, for the drawn indices `draws` (n_d of them, with
        repeats) of V sampled with p_i proportional to |c_i| (Eq. 10)."""
        dets = _u64(dets)
        c = _f64(np.ravel(c))
        draws = np.asarray(draws, np.int64)
        sidx, sw = np.unique(draws, return_counts=True)
        sidx, sw = _i64(sidx), _i64(sw)
        out = np.zeros(2)
        rc = _load().oracle_pt2_sample(self.n, n_words(dets), self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                                       dets.shape[0], _p(dets, _u64p), _p(c, _f64p), float(e_var), float(eps2),
                                       float(eps2_d), draws.size, sidx.size, _p(sidx, _i64p), _p(sw, _i64p),
                                       _p(out, _f64p))
        if rc != 0:
            raise RuntimeError("oracle_pt2_sample failed (%d)" % rc)
        return float(out[0]), float(out[1])

    # ---------------------------------------------------------- sigma
    def sigma_rows(self, dets, c, rows) -> np.ndarray:
        """sigma[k, rows] by brute force over all columns (c is [k, n_det])."""
        dets = _u64(dets)
        c = _f64(np.atleast_2d(c))
        rows = _i64(rows)
        out = np.empty((c.shape[0], rows.size))
        _load().oracle_sigma_rows(self.n, n_words(dets), self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p),
                                  dets.shape[0], _p(dets, _u64p), c.shape[0], _p(c, _f64p), rows.size,
                                  _p(rows, _i64p), _p(out, _f64p))
        return out

    # ---------------------------------------------------------- matrices
    def upper_pairs(self, dets):
        """(i, j, H_ij) for all connected i < j, lexicographic, by brute force (a)."""
        ii, jj = pairs_allpairs(dets)
        return ii, jj, self.hij_list(dets, ii, jj)

    def upper_csr(self, dets):
        """The upper triangle of H on V as compressed rows (rowptr int64 [n+1],
        col int32, val f64; row i holds its connected j > i ascending), by brute
        force (a) -- 12 bytes per connected pair, for spaces of ~1e6."""
        dets = _u64(dets)
        n = dets.shape[0]
        if n >= 2 ** 31:
            raise ValueError("upper_csr: n_det must be below 2^31")
        lib = _load()
        rowptr = np.empty(n + 1, np.int64)
        args = (self.n, n_words(dets), self.e_core, _p(self.h, _f64p), _p(self.eri, _f64p), n, _p(dets, _u64p))
        total = lib.oracle_upper_csr(*args, _p(rowptr, _i64p), None, None)
        col = np.empty(max(total, 1), np.int32)
        val = np.empty(max(total, 1))
        lib.oracle_upper_csr(*args, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p))
        return rowptr, col[:total], val[:total]

    def sparse_h(self, dets):
        """scipy CSR of the full symmetric H on V (assembled from the oracle's pairs)."""
        import scipy.sparse as sp
        n = dets.shape[0]
        ii, jj, v = self.upper_pairs(dets)
        d = self.hdiag(dets)
        rows = np.concatenate([ii, jj, np.arange(n)])
        cols = np.concatenate([jj, ii, np.arange(n)])
        vals = np.concatenate([v, v, d])
        return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

    def dense_h(self, dets) -> np.ndarray:
        n = dets.shape[0]
        H = np.zeros((n, n))
        ii, jj, v = self.upper_pairs(dets)
        H[ii, jj] = v
        H[jj, ii] = v
        H[np.arange(n), np.arange(n)] = self.hdiag(dets)
        return H

    # ---------------------------------------------------------- eigenpairs
    def lowest_eigenpairs(self, dets, k=1, tol=1e-10, dense_max=6000, res_tol=1e-7, guess=None):
        """(E[k], C[k, n]) lowest roots of H on V: a dense eigensolver up to
        dense_max determinants, else Davidson on the upper-triangle rows."""
        n = dets.shape[0]
        if n <= dense_max:
            w, v = np.linalg.eigh(self.dense_h(dets))
            return w[:k].copy(), np.ascontiguousarray(v[:, :k].T)
        op = UpperMatrix(*self.upper_csr(dets), self.hdiag(dets))
        return davidson(op.matvec, op.diag, k, tol=tol, res_tol=res_tol, guess=guess)

    # ---------------------------------------------------------- gradients
    def energy_gradient(self, dets, c):
        """(dE/dh [n, n], dE/d eri_packed) for the normalised real root c: gamma and the
        packed, symmetry-summed Gamma / 2.  Full RDMs: small spaces only."""
        n = self.n
        g1 = rdm1_full(dets, c, n)
        g2 = rdm2_full(dets, c, n)
        return g1, fold_rdm2_to_packed(g2, n)


# ------------------------------------------------------------ pair sets

def pairs_allpairs(dets):
    """Brute force (a): all connected pairs i < j, lexicographic."""
    dets = _u64(dets)
    lib = _load()
    total = lib.oracle_pairs_allpairs(dets.shape[0], n_words(dets), _p(dets, _u64p), 0, None, None)
    ii = np.empty(total, np.int64)
    jj = np.empty(total, np.int64)
    lib.oracle_pairs_allpairs(dets.shape[0], n_words(dets), _p(dets, _u64p), total, _p(ii, _i64p), _p(jj, _i64p))
    return ii, jj


def pairs_generate(dets, n_orb):
    """Brute force (b): excitations of each determinant looked up in V (i < j, lexicographic)."""
    dets = _u64(dets)
    lib = _load()
    total = lib.oracle_pairs_generate(n_orb, dets.shape[0], n_words(dets), _p(dets, _u64p), 0, None, None)
    if total < 0:
        raise ValueError("duplicate determinants" if total == -2 else "out of memory")
    ii = np.empty(total, np.int64)
    jj = np.empty(total, np.int64)
    lib.oracle_pairs_generate(n_orb, dets.shape[0], n_words(dets), _p(dets, _u64p), total,
                              _p(ii, _i64p), _p(jj, _i64p))
    return ii, jj


def has_duplicates(dets) -> bool:
    dets = _u64(dets)
    return _load().oracle_check_unique(dets.shape[0], n_words(dets), _p(dets, _u64p)) == -2


def sigma_pairs(n_det, ii, jj, hij, diag, c):
    """sigma = H c from an upper pair list plus diagonal (long double, sequential)."""
    c = _f64(np.atleast_2d(c))
    ii, jj, hij, diag = _i64(ii), _i64(jj), _f64(hij), _f64(diag)
    out = np.empty_like(c)
    _load().oracle_sigma_pairs(n_det, ii.size, _p(ii, _i64p), _p(jj, _i64p), _p(hij, _f64p), _p(diag, _f64p),
                               c.shape[0], _p(c, _f64p), _p(out, _f64p))
    return out


class UpperMatrix:
    """H from its upper-triangle rows (System.upper_csr) and its diagonal."""

    def __init__(self, rowptr, col, val, diag):
        self.rowptr, self.col, self.val = _i64(rowptr), np.ascontiguousarray(col, np.int32), _f64(val)
        self.diag = _f64(diag)
        self.n = self.diag.size

    @property
    def nnz_upper(self) -> int:
        return int(self.rowptr[-1])

    def matvec(self, x):
        """H x for x [n] or [k, n] (vectors as rows)."""
        x = _f64(x)
        one = x.ndim == 1
        c = np.atleast_2d(x)
        out = np.empty_like(c)
        _load().oracle_sigma_upper(self.n, _p(self.rowptr, _i64p), _p(self.col, _i32p), _p(self.val, _f64p),
                                   _p(self.diag, _f64p), c.shape[0], _p(c, _f64p), _p(out, _f64p))
        return out[0] if one else out


# ------------------------------------------------------------ Davidson

def davidson(matvec, diag, k=1, tol=1e-10, res_tol=1e-7, max_iter=400, max_sub=None, guess=None):
    """Diagonally preconditioned Davidson for the k lowest roots (Sec. II.A).

    Start from the unit vectors of the k lowest diagonal entries (or from the
    rows of ``guess`` [k, n], orthonormalised); each step
    projects H on the subspace, takes the lowest k Ritz pairs, forms residuals
    r = H x - theta x, preconditions them by (theta - H_ii)^-1 and adds the
    orthonormalised corrections.  Stops when every root moved by less than
    ``tol`` and has ||r|| < ``res_tol``.  Plain numpy; slow by design.
    """
    n = diag.size
    max_sub = max_sub or max(8 * k, 24)
    if guess is not None:
        V, _ = np.linalg.qr(np.asarray(guess, dtype=np.float64).reshape(k, n).T)
    else:
        V = np.zeros((n, 0))
        for idx in np.argsort(diag, kind="stable")[:k]:
            e = np.zeros(n)
            e[idx] = 1.0
            V = np.column_stack([V, e])
    AV = np.column_stack([matvec(V[:, a]) for a in range(V.shape[1])])
    theta_old = np.full(k, np.inf)
    for _ in range(max_iter):
        G = V.T @ AV
        G = 0.5 * (G + G.T)
        w, Y = np.linalg.eigh(G)
        theta, Y = w[:k], Y[:, :k]
        X = V @ Y
        R = AV @ Y - X * theta
        rn = np.linalg.norm(R, axis=0)
        if np.all(np.abs(theta - theta_old) < tol) and np.all(rn < res_tol):
            return theta, np.ascontiguousarray(X.T)
        theta_old = theta
        if V.shape[1] + k > max_sub:
            V, AV = X, AV @ Y          # restart on the current Ritz vectors
        new = []
        for a in range(k):
            if rn[a] < 1e-14:
                continue
            den = theta[a] - diag
            den = np.where(np.abs(den) < 1e-8, np.copysign(1e-8, den), den)
            t = R[:, a] / den
            for _rep in range(2):
                t -= V @ (V.T @ t)
                for u in new:
                    t -= u * (u @ t)
            nt = np.linalg.norm(t)
            if nt > 1e-12:
                new.append(t / nt)
        if not new:
            return theta, np.ascontiguousarray(X.T)
        N = np.column_stack(new)
        V = np.column_stack([V, N])
        AV = np.column_stack([AV] + [matvec(N[:, a]) for a in range(N.shape[1])])
    raise RuntimeError("oracle Davidson did not converge")


# ------------------------------------------------------------ density matrices

def rdm1_entries(dets, c, n_orb, idx):
    """gamma_pq for idx [m, 2] (spin-summed, real c)."""
    dets, c = _u64(dets), _f64(c)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(idx.shape[0])
    rc = _load().oracle_rdm1(n_orb, n_words(dets), dets.shape[0], _p(dets, _u64p), _p(c, _f64p),
                             idx.shape[0], _p(idx, _i32p), _p(out, _f64p))
    if rc:
        raise ValueError("duplicate determinants")
    return out


def rdm2_entries(dets, c, n_orb, idx):
    """Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs> for idx [m, 4]."""
    dets, c = _u64(dets), _f64(c)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(idx.shape[0])
    rc = _load().oracle_rdm2(n_orb, n_words(dets), dets.shape[0], _p(dets, _u64p), _p(c, _f64p),
                             idx.shape[0], _p(idx, _i32p), _p(out, _f64p))
    if rc:
        raise ValueError("duplicate determinants")
    return out


def rdm1_full(dets, c, n):
    idx = np.array([(p, q) for p in range(n) for q in range(n)], dtype=np.int32)
    return rdm1_entries(dets, c, n, idx).reshape(n, n)


def rdm2_full(dets, c, n):
    idx = np.array([(p, q, r, s) for p in range(n) for q in range(n) for r in range(n) for s in range(n)],
                   dtype=np.int32)
    return rdm2_entries(dets, c, n, idx).reshape(n, n, n, n)


def slot_members(n):
    """For every packed slot, the list of (p, q, r, s) index tuples that map to it."""
    members = {}
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    a = max(p, q) * (max(p, q) + 1) // 2 + min(p, q)
                    b = max(r, s) * (max(r, s) + 1) // 2 + min(r, s)
                    slot = max(a, b) * (max(a, b) + 1) // 2 + min(a, b)
                    members.setdefault(slot, []).append((p, q, r, s))
    return members


def packed_gradient_entries(dets, c, n_orb, slots, members=None):
    """dE/d(packed slot) = 1/2 sum_{(p,q,r,s) -> slot} Gamma_pqrs for the listed slots."""
    members = members or slot_members(n_orb)
    idx, owner = [], []
    for t, slot in enumerate(slots):
        for tup in members[int(slot)]:
            idx.append(tup)
            owner.append(t)
    vals = rdm2_entries(dets, c, n_orb, np.array(idx, dtype=np.int32))
    out = np.zeros(len(slots))
    np.add.at(out, np.array(owner), 0.5 * vals)
    return out


def fold_rdm2_to_packed(G, n):
    """dE/d(packed slot) = 1/2 * sum of Gamma_pqrs over every distinct (p,q,r,s) that the
    slot stores (its 8-fold symmetry orbit)."""
    npair = n * (n + 1) // 2
    out = np.zeros(npair * (npair + 1) // 2)
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    a = max(p, q) * (max(p, q) + 1) // 2 + min(p, q)
                    b = max(r, s) * (max(r, s) + 1) // 2 + min(r, s)
                    slot = max(a, b) * (max(a, b) + 1) // 2 + min(a, b)
                    out[slot] += 0.5 * G[p, q, r, s]
    return out
