"""Independent second-quantised Hamiltonian for pinning the oracle.

Builds H = E_core + sum_PQ h_PQ a+_P a_Q + 1/2 sum_PQRS (PQ|RS) a+_P a+_R a_S a_Q
as an explicit sparse matrix on the 2^(2n) Fock space (Jordan-Wigner
representation: mode j's annihilator carries the parity of the occupied modes
below j), by multiplying operator matrices term by term.  No excitation
analysis and no Slater-Condon rule is involved, so agreement with the oracle's
matrix elements pins their values *and* signs.

Mode order: alpha orbitals 0..n-1, then beta orbitals 0..n-1; a Fock basis
state's index has bit j set when mode j is occupied, and the state equals
prod_{j ascending, occupied} a+_j |0> with a + sign.
"""
import numpy as np
import scipy.sparse as sp


def annihilators(n_modes):
    dim = 1 << n_modes
    ops = []
    states = np.arange(dim)
    for j in range(n_modes):
        occ = (states >> j) & 1
        src = states[occ == 1]
        dst = src - (1 << j)
        below = src & ((1 << j) - 1)
        parity = np.array([bin(int(b)).count("1") & 1 for b in below])
        vals = np.where(parity == 1, -1.0, 1.0)
        ops.append(sp.csr_matrix((vals, (dst, src)), shape=(dim, dim)))
    return ops


def eri_full(eri_packed, n):
    out = np.empty((n, n, n, n))
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    a = max(p, q) * (max(p, q) + 1) // 2 + min(p, q)
                    b = max(r, s) * (max(r, s) + 1) // 2 + min(r, s)
                    out[p, q, r, s] = eri_packed[max(a, b) * (max(a, b) + 1) // 2 + min(a, b)]
    return out


def fock_hamiltonian(h, eri_packed, e_core=0.0):
    n = h.shape[0]
    M = 2 * n
    a = annihilators(M)
    ad = [x.T.tocsr() for x in a]
    g = eri_full(eri_packed, n)
    dim = 1 << M
    H = sp.identity(dim, format="csr") * e_core
    spin = lambda P: P // n
    orb = lambda P: P % n
    for P in range(M):
        for Q in range(M):
            if spin(P) == spin(Q) and h[orb(P), orb(Q)] != 0.0:
                H = H + h[orb(P), orb(Q)] * (ad[P] @ a[Q])
    for P in range(M):
        for Q in range(M):
            if spin(P) != spin(Q):
                continue
            for R in range(M):
                for S in range(M):
                    if spin(R) != spin(S):
                        continue
                    v = g[orb(P), orb(Q), orb(R), orb(S)]
                    if v == 0.0:
                        continue
                    H = H + 0.5 * v * (ad[P] @ (ad[R] @ (a[S] @ a[Q])))
    return H.tocsr()


def det_to_fock_index(det, n):
    """uint64 [2] (W = 1) determinant -> Fock basis index."""
    return int(det[0]) | (int(det[1]) << n)


def projected(h, eri_packed, dets, e_core=0.0):
    """<D_i| H |D_j> for determinants dets (W = 1), from the Fock-space matrix."""
    n = h.shape[0]
    H = fock_hamiltonian(h, eri_packed, e_core)
    idx = np.array([det_to_fock_index(d, n) for d in dets])
    return np.asarray(H[idx][:, idx].todense())
