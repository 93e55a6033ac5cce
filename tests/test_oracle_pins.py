"""Pins for the CPU oracle: checks against things other than the oracle itself.

* the second-quantised Hamiltonian built from operator matrices (tests/jw.py),
* hand-worked excitation signs (tests/golden/slater_condon_signs.json),
* closed forms (one electron; no two-body term; one alpha + one beta electron),
* invariants (Hermiticity, orbital-rotation invariance of the full-CI spectrum),
* the two brute-force pair definitions of Sec. III agreeing with each other,
* the Davidson iteration against a dense eigensolver and ARPACK,
* density-matrix identities and central finite differences of the energy,
* planted mistakes in a copy of the oracle's C source being caught.
"""
import itertools
import json
import os
import shutil
import subprocess
import ctypes

import numpy as np
import pytest

import shci_synth as S
from tests import jw

HERE = os.path.dirname(os.path.abspath(__file__))


def small_system(n, rank, seed):
    h, eri, ec = S.integrals(n, rank, seed)
    return h, eri, ec


def rotate(h, eri, U):
    n = h.shape[0]
    g = jw.eri_full(eri, n)
    h2 = U.T @ h @ U
    g2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", g, U, U, U, U, optimize=True)
    packed = np.empty(S.eri_len(n))
    for p in range(n):
        for q in range(p + 1):
            for r in range(n):
                for s in range(r + 1):
                    a = p * (p + 1) // 2 + q
                    b = r * (r + 1) // 2 + s
                    if a >= b:
                        packed[a * (a + 1) // 2 + b] = g2[p, q, r, s]
    return 0.5 * (h2 + h2.T), packed


# ------------------------------------------------------------------ JW pin

@pytest.mark.parametrize("n,na,nb", [(3, 1, 1), (3, 2, 1), (4, 2, 2), (4, 3, 1), (4, 2, 1)])
def test_matrix_elements_match_second_quantised_h(oracle_mod, n, na, nb):
    h, eri, _ = small_system(n, 5, 100 + 10 * n + na)
    e_core = 0.37
    dets = S.fci_dets(n, na, nb)
    ref = jw.projected(h, eri, dets, e_core)
    got = oracle_mod.System(h, eri, e_core).dense_h(dets)
    np.testing.assert_allclose(got, ref, atol=1e-12, rtol=0)
    # the pair set of brute force (a) is exactly the structurally connected set
    nz = np.abs(np.triu(ref, 1)) > 1e-14
    ii, jj = oracle_mod.pairs_allpairs(dets)
    mask = np.zeros_like(nz)
    mask[ii, jj] = True
    assert not np.any(nz & ~mask)          # every nonzero element is a listed pair


# ------------------------------------------------------------------ two-word strings (n_orb > 64)

EMBED_AT = 62          # the small system's orbitals 0..3 become orbitals 62..65: both words of a string


def embedded_two_word_system(n_big=76, n=4, na=2, nb=2, e_core=0.37, seed=151):
    """A 4-orbital system placed at orbitals 62..65 of a 76-orbital space (all
    other integrals zero, electrons only in those orbitals) and the small
    system's Jordan-Wigner Hamiltonian on the same determinants.  The relative
    order of the occupied orbitals is unchanged, so the signed elements must
    be identical; strings straddle the word boundary at orbital 64."""
    h4, eri4, _ = small_system(n, 5, seed)
    g4 = jw.eri_full(eri4, n)
    h = np.zeros((n_big, n_big))
    h[EMBED_AT:EMBED_AT + n, EMBED_AT:EMBED_AT + n] = h4
    eri = np.zeros(S.eri_len(n_big))
    for p, q, r, s_ in itertools.product(range(n), repeat=4):
        P, Q, R, Sx = (EMBED_AT + x for x in (p, q, r, s_))
        a = max(P, Q) * (max(P, Q) + 1) // 2 + min(P, Q)
        b = max(R, Sx) * (max(R, Sx) + 1) // 2 + min(R, Sx)
        eri[max(a, b) * (max(a, b) + 1) // 2 + min(a, b)] = g4[p, q, r, s_]
    small = S.fci_dets(n, na, nb)
    occ = lambda w: [k for k in range(n) if (int(w) >> k) & 1]
    big = np.concatenate([
        S.strings_from_occ(np.array([[EMBED_AT + k for k in occ(d[0])] for d in small]), n_big),
        S.strings_from_occ(np.array([[EMBED_AT + k for k in occ(d[1])] for d in small]), n_big)], axis=1)
    straddle = lambda w0, w1: np.any((w0 != 0) & (w1 != 0))
    assert big.shape[1] == 4 and straddle(big[:, 0], big[:, 1]) and straddle(big[:, 2], big[:, 3])
    return h, eri, e_core, big, jw.projected(h4, eri4, small, e_core)


def test_two_word_strings_match_embedded_small_system(oracle_mod):
    """Orbitals >= 64 (the second word of a string, Sec. V.A's bit layout): the
    oracle's signed H on the embedded determinants equals the small system's
    Jordan-Wigner Hamiltonian entry by entry."""
    h, eri, ec, dets, ref = embedded_two_word_system()
    got = oracle_mod.System(h, eri, ec).dense_h(dets)
    np.testing.assert_allclose(got, ref, atol=1e-12, rtol=0)
    assert np.count_nonzero(np.abs(ref) > 1e-12) > dets.shape[0]


# ------------------------------------------------------------------ hand signs

def test_hand_worked_signs(oracle_mod):
    spec = json.load(open(os.path.join(HERE, "golden", "slater_condon_signs.json")))
    n = spec["integrals"]["n_orb"]
    h, eri, _ = S.integrals(n, spec["integrals"]["rank"], spec["integrals"]["seed"])
    g = jw.eri_full(eri, n)
    O = oracle_mod.System(h, eri, 0.0)
    for case in spec["cases"]:
        def det(occ):
            a = S.strings_from_occ(np.array([occ[0]], dtype=np.int64).reshape(1, -1), n)
            b = S.strings_from_occ(np.array([occ[1]], dtype=np.int64).reshape(1, -1), n)
            return np.concatenate([a, b], axis=1)[0]
        val = 0.0
        for coef, kind, idx in case["terms"]:
            val += coef * (h[idx[0], idx[1]] if kind == "h" else g[tuple(idx)])
        want = case["sign"] * val
        got = O.hij(det(case["i"]), det(case["j"]))
        assert abs(got - want) < 1e-14, case["name"]
        # Hermiticity: the reverse element through the other hole/particle assignment
        assert abs(O.hij(det(case["j"]), det(case["i"])) - want) < 1e-14, case["name"]


# ------------------------------------------------------------------ closed forms

def test_one_electron_is_h(oracle_mod):
    n = 7
    h, eri, _ = small_system(n, 4, 5)
    dets = S.fci_dets(n, 1, 0)
    H = oracle_mod.System(h, eri, 0.0).dense_h(dets)
    np.testing.assert_allclose(H, h, atol=1e-15, rtol=0)


def test_no_two_body_term_gives_orbital_sums(oracle_mod):
    n, na, nb = 6, 2, 3
    h, eri, _ = small_system(n, 4, 6)
    eri = np.zeros_like(eri)
    dets = S.fci_dets(n, na, nb)
    w = np.linalg.eigvalsh(oracle_mod.System(h, eri, 0.0).dense_h(dets))
    eps = np.linalg.eigvalsh(h)
    sums = sorted(sum(eps[list(a)]) + sum(eps[list(b)])
                  for a in itertools.combinations(range(n), na)
                  for b in itertools.combinations(range(n), nb))
    np.testing.assert_allclose(w, sums, atol=1e-12)


def test_one_alpha_one_beta_is_kronecker_form(oracle_mod):
    n = 6
    h, eri, _ = small_system(n, 5, 9)
    g = jw.eri_full(eri, n)
    dets = S.fci_dets(n, 1, 1)               # alpha index major, beta minor
    H = oracle_mod.System(h, eri, 0.0).dense_h(dets)
    V = np.einsum("prqs->pqrs", g).reshape(n * n, n * n)   # V[(p,q),(r,s)] = (pr|qs)
    ref = np.kron(h, np.eye(n)) + np.kron(np.eye(n), h) + V
    np.testing.assert_allclose(H, ref, atol=1e-13, rtol=0)


# ------------------------------------------------------------------ invariants

def test_hermitian_random_pairs(oracle_mod):
    cfg = S.config("sel_24o_6a6b_1m")
    h, eri, ec, dets = S.make_system(cfg, n_det=3000)
    O = oracle_mod.System(h, eri, ec)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    rng = np.random.default_rng(0)
    sel = rng.choice(ii.size, size=min(4000, ii.size), replace=False)
    a = O.hij_list(dets, ii[sel], jj[sel])
    b = O.hij_list(dets, jj[sel], ii[sel])
    np.testing.assert_allclose(a, b, atol=1e-14, rtol=0)


def test_fci_spectrum_invariant_under_orbital_rotation(oracle_mod):
    n, na, nb = 6, 3, 2
    h, eri, _ = small_system(n, 6, 11)
    dets = S.fci_dets(n, na, nb)
    w0 = np.linalg.eigvalsh(oracle_mod.System(h, eri, 0.0).dense_h(dets))
    U, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(n, n)))
    h2, eri2 = rotate(h, eri, U)
    w1 = np.linalg.eigvalsh(oracle_mod.System(h2, eri2, 0.0).dense_h(dets))
    np.testing.assert_allclose(w0, w1, atol=1e-10)


# ------------------------------------------------------------------ pair sets

@pytest.mark.parametrize("cfgname,n_det", [("fci_10o_4a4b", None), ("sel_24o_6a6b_1m", 20000),
                                           ("sel_20o_5a5b_1m", 20000)])
def test_two_brute_force_pair_definitions_agree(oracle_mod, cfgname, n_det):
    cfg = S.config(cfgname)
    h, eri, ec, dets = S.make_system(cfg, n_det=n_det)
    a = oracle_mod.pairs_allpairs(dets)
    b = oracle_mod.pairs_generate(dets, cfg.n_orb)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    if cfgname == "fci_10o_4a4b":
        # full-CI: every determinant has (24+24+90+90+576) = 804 connections
        assert a[0].size == 44100 * 804 // 2


def test_duplicates_detected(oracle_mod):
    dets = S.fci_dets(5, 2, 2)
    assert not oracle_mod.has_duplicates(dets)
    bad = np.concatenate([dets, dets[3:4]])
    assert oracle_mod.has_duplicates(bad)


# ------------------------------------------------------------------ sigma

def test_sigma_rows_and_pairs_match_dense(oracle_mod):
    cfg = S.config("sel_24o_6a6b_1m")
    h, eri, ec, dets = S.make_system(cfg, n_det=1500)
    O = oracle_mod.System(h, eri, ec)
    H = O.dense_h(dets)
    c = S.random_vectors(dets.shape[0], 2, 5)
    ref = c @ H.T
    rows = np.arange(dets.shape[0])
    np.testing.assert_allclose(O.sigma_rows(dets, c, rows), ref, atol=1e-11)
    ii, jj, v = O.upper_pairs(dets)
    np.testing.assert_allclose(oracle_mod.sigma_pairs(dets.shape[0], ii, jj, v, O.hdiag(dets), c), ref,
                               atol=1e-11)
    cols, vals = O.row(dets, 17)
    dense_row = H[17].copy()
    dense_row[17] = 0.0
    nzc = np.nonzero(np.abs(dense_row) > 0)[0]
    assert set(nzc.tolist()) <= set(cols.tolist())
    np.testing.assert_allclose(vals, H[17, cols], atol=1e-15)


def test_upper_rows_sigma_matches_dense(oracle_mod):
    """The upper-triangle rows hold exactly the pairs of brute force (a), and
    H x from them (with the diagonal) equals the dense matrix, whose entries
    the Jordan-Wigner pin checks, for one and several vectors, one- and
    two-word strings."""
    cfg = S.config("sel_24o_6a6b_1m")
    h, eri, ec, dets = S.make_system(cfg, n_det=2500)
    cases = [(h, eri, ec, dets)]
    hb, eb, ecb, db, _ = embedded_two_word_system()
    cases.append((hb, eb, ecb, db))
    for hh, ee, cc, dd in cases:
        O = oracle_mod.System(hh, ee, cc)
        rowptr, col, val = O.upper_csr(dd)
        ii, jj = oracle_mod.pairs_allpairs(dd)
        assert rowptr[-1] == ii.size
        assert np.array_equal(np.repeat(np.arange(dd.shape[0]), np.diff(rowptr)), ii)
        assert np.array_equal(col.astype(np.int64), jj)
        op = oracle_mod.UpperMatrix(rowptr, col, val, O.hdiag(dd))
        Hd = O.dense_h(dd)
        x = S.random_vectors(dd.shape[0], 3, 8)
        np.testing.assert_allclose(op.matvec(x), x @ Hd.T, atol=1e-11, rtol=0)
        np.testing.assert_allclose(op.matvec(x[1]), Hd @ x[1], atol=1e-11, rtol=0)


# ------------------------------------------------------------------ eigenpairs

def test_davidson_matches_dense_and_arpack(oracle_mod):
    import scipy.sparse.linalg as sla
    cfg = S.config("sel_24o_6a6b_1m")
    h, eri, ec, dets = S.make_system(cfg, n_det=4000)
    O = oracle_mod.System(h, eri, ec)
    w = np.linalg.eigvalsh(O.dense_h(dets))[:2]
    H = O.sparse_h(dets)
    e, C = oracle_mod.davidson(H.dot, H.diagonal(), k=2, tol=1e-12, res_tol=1e-8)
    np.testing.assert_allclose(e, w, atol=1e-9)
    ea = np.sort(sla.eigsh(H, k=2, which="SA", tol=1e-12)[0])
    np.testing.assert_allclose(e, ea, atol=1e-9)
    # eigenvectors: residual small and orthonormal
    for a in range(2):
        r = H.dot(C[a]) - e[a] * C[a]
        assert np.linalg.norm(r) < 1e-7
    np.testing.assert_allclose(C @ C.T, np.eye(2), atol=1e-10)
    # started from a guess (the route the selection loop takes), through the upper rows
    guess = C + 1e-3 * S.random_vectors(dets.shape[0], 2, 9)
    e2, _ = O.lowest_eigenpairs(dets, 2, tol=1e-12, dense_max=0, res_tol=1e-8, guess=guess)
    np.testing.assert_allclose(e2, w, atol=1e-9)


# ------------------------------------------------------------------ RDMs and gradients

def _ground(oracle_mod, h, eri, ec, dets):
    O = oracle_mod.System(h, eri, ec)
    w, v = np.linalg.eigh(O.dense_h(dets))
    return O, w[0], v[:, 0]


def test_rdm_traces_and_energy_identity(oracle_mod):
    n, na, nb = 5, 2, 2
    h, eri, _ = small_system(n, 5, 21)
    dets = S.fci_dets(n, na, nb)
    O, E, c = _ground(oracle_mod, h, eri, 0.25, dets)
    g1 = oracle_mod.rdm1_full(dets, c, n)
    g2 = oracle_mod.rdm2_full(dets, c, n)
    N = na + nb
    assert abs(np.trace(g1) - N) < 1e-12
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-10
    np.testing.assert_allclose(g1, g1.T, atol=1e-13)
    G = jw.eri_full(eri, n)
    E2 = 0.25 + np.sum(h * g1) + 0.5 * np.sum(G * g2)
    assert abs(E2 - E) < 1e-11
    # packed folding: sum_slot eri[slot] * dE/deri[slot] reproduces the two-body energy
    gh, ge = O.energy_gradient(dets, c)
    assert abs(np.dot(eri, ge) - 0.5 * np.sum(G * g2)) < 1e-11


def test_rdm_no_two_body_closed_form(oracle_mod):
    n, na, nb = 6, 2, 3
    h, eri, _ = small_system(n, 4, 23)
    eri = np.zeros_like(eri)
    dets = S.fci_dets(n, na, nb)
    O, E, c = _ground(oracle_mod, h, eri, 0.0, dets)
    eps, U = np.linalg.eigh(h)
    ref = U[:, :na] @ U[:, :na].T + U[:, :nb] @ U[:, :nb].T
    np.testing.assert_allclose(oracle_mod.rdm1_full(dets, c, n), ref, atol=1e-10)


def test_packed_gradient_entries_equal_folded_rdm2(oracle_mod):
    """Per-slot gradient entries (the symmetry orbit of each packed slot,
    gathered from single Gamma entries) equal the fold of the full 2-RDM, which
    the energy identity and the finite differences pin; every (p,q,r,s) is a
    member of exactly one slot."""
    n, na, nb = 5, 2, 2
    h, eri, _ = small_system(n, 5, 41)
    dets = S.fci_dets(n, na, nb)
    O, E, c = _ground(oracle_mod, h, eri, 0.0, dets)
    members = oracle_mod.slot_members(n)
    assert sorted(members) == list(range(S.eri_len(n)))
    assert sum(len(m) for m in members.values()) == n ** 4
    slots = np.arange(S.eri_len(n))
    got = oracle_mod.packed_gradient_entries(dets, c, n, slots, members)
    want = oracle_mod.fold_rdm2_to_packed(oracle_mod.rdm2_full(dets, c, n), n)
    np.testing.assert_allclose(got, want, atol=1e-13, rtol=0)
    _, ge = O.energy_gradient(dets, c)
    np.testing.assert_allclose(got, ge, atol=1e-13, rtol=0)


def test_gradient_matches_central_differences(oracle_mod):
    n, na, nb = 5, 2, 2
    h, eri, _ = small_system(n, 5, 31)
    dets = S.fci_dets(n, na, nb)
    O, E, c = _ground(oracle_mod, h, eri, 0.0, dets)
    gh, ge = O.energy_gradient(dets, c)
    rng = np.random.default_rng(4004)
    step = 1e-5
    for _ in range(4):
        dh = rng.normal(size=(n, n))
        dh = 0.5 * (dh + dh.T)
        de = rng.normal(size=eri.size)
        ep = np.linalg.eigvalsh(oracle_mod.System(h + step * dh, eri + step * de, 0.0).dense_h(dets))[0]
        em = np.linalg.eigvalsh(oracle_mod.System(h - step * dh, eri - step * de, 0.0).dense_h(dets))[0]
        fd = (ep - em) / (2 * step)
        an = np.sum(gh * dh) + np.dot(ge, de)
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


# ------------------------------------------------------------------ planted mistakes

MUTATIONS = {
    "single exchange sign": ("v += eri_so(I, p, q, k, k) - eri_so(I, p, k, k, q);",
                             "v += eri_so(I, p, q, k, k) + eri_so(I, p, k, k, q);"),
    "double exchange dropped": ("double v = eri_so(I, p, q, r, s) - eri_so(I, p, s, r, q);",
                                "double v = eri_so(I, p, q, r, s);"),
    "double operand transposed": ("double v = eri_so(I, p, q, r, s) - eri_so(I, p, s, r, q);",
                                  "double v = eri_so(I, p, r, q, s) - eri_so(I, p, s, r, q);"),
    "creation phase ignored": ("    int ph = (n_before(I, d, so) & 1) ? -1 : 1;\n    put(I, d, so, 1);",
                               "    int ph = 1;\n    put(I, d, so, 1);"),
    "diagonal exchange dropped": ("e += 0.5 * (eri_so(I, k, k, l, l) - eri_so(I, k, l, l, k));",
                                  "e += 0.5 * (eri_so(I, k, k, l, l));"),
    "two-word index": ("spin * I->W + (p >> 6)", "spin + (p >> 6)"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name):
    """A mistake planted in a copy of the oracle's C source must fail the JW pin
    (one-word strings, or the 4-orbital system embedded across two words)."""
    src = open(os.path.join(os.path.dirname(oracle_mod.__file__), "shci_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert old in src
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-std=c11", "-o", str(so), str(mut), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    f64p = ctypes.POINTER(ctypes.c_double)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.oracle_hij.restype = ctypes.c_double
    lib.oracle_hij.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, f64p, f64p, u64p, u64p]

    def worst(n, h, eri, ec, dets, ref):
        W = dets.shape[1] // 2
        got = np.empty_like(ref)
        for i in range(dets.shape[0]):
            for j in range(dets.shape[0]):
                di = np.ascontiguousarray(dets[i])
                dj = np.ascontiguousarray(dets[j])
                got[i, j] = lib.oracle_hij(n, W, ec, h.ctypes.data_as(f64p), eri.ctypes.data_as(f64p),
                                           di.ctypes.data_as(u64p), dj.ctypes.data_as(u64p))
        return np.max(np.abs(got - ref))

    n, na, nb = 4, 2, 2
    h, eri, _ = small_system(n, 5, 140 + na)
    dets = S.fci_dets(n, na, nb)
    err = worst(n, h, eri, 0.0, dets, jw.projected(h, eri, dets, 0.0))
    hb, eb, ecb, db, refb = embedded_two_word_system()
    err = max(err, worst(hb.shape[0], hb, eb, ecb, db, refb))
    assert err > 1e-6, "planted mistake was not detected"


# ---------------------------------------------------------------- heat-bath selection (Sec. II.A, Eq. 2)

def _excitation_degree(a, b):
    return int(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))) // 2


def test_selection_from_one_determinant_reaches_every_connection(oracle_mod):
    """From V = {HF} with a threshold below every matrix element, the selected
    set is every determinant one or two excitations away: 804 for 10 orbitals
    with 4a4b (24 + 24 singles, 90 + 90 same-spin and 576 opposite-spin
    doubles), each at excitation degree 1 or 2 from HF."""
    h, eri, ec = S.integrals(10, 20, 1000)
    hf = S.fci_dets(10, 4, 4)[:1]
    O = oracle_mod.System(h, eri, ec)
    sel = O.select(hf, np.ones((1, 1)), 1e-14)
    assert sel.shape[0] == 804
    deg = [_excitation_degree(hf[0], d) for d in sel]
    assert sorted(set(deg)) == [1, 2]
    assert deg.count(1) == 48


def test_selection_matches_dense_hamiltonian(oracle_mod):
    """V a random subset of the full-CI space (8 orbitals, 3a2b): the selected
    set equals {a outside V : max_i |H_ai| |c_i| >= eps1} read off the dense
    full-CI matrix (whose entries the Jordan-Wigner pin checks), borderline
    products aside; a larger eps1 selects a subset; V = full space selects
    nothing."""
    n, na, nb = 8, 3, 2
    h, eri, ec = S.integrals(n, 10, 4242)
    fci = S.fci_dets(n, na, nb)
    O = oracle_mod.System(h, eri, ec)
    H = O.dense_h(fci)
    rng = np.random.default_rng(3)
    vidx = np.sort(rng.choice(fci.shape[0], 25, replace=False))
    c = rng.standard_normal((2, vidx.size))
    cmax = np.max(np.abs(c), axis=0)
    prod = np.abs(H[:, vidx]) * cmax[None, :]
    prod[vidx, :] = 0.0                              # determinants already in V are never selected
    best = prod.max(axis=1)
    key = lambda d: tuple(int(x) for x in d[::-1])   # last stored word most significant
    prev = None
    for eps1 in (1e-1, 1e-2, 1e-3):
        sel = O.select(fci[vidx], c, eps1)
        got = {key(d) for d in sel}
        want = {key(fci[a]) for a in np.nonzero(best >= eps1)[0]}
        border = {key(fci[a]) for a in np.nonzero(np.abs(best - eps1) <= 1e-12 * eps1)[0]}
        assert got - border == want - border
        assert [key(d) for d in sel] == sorted(got)  # ascending, no repeats
        if prev is not None:
            assert prev <= got                       # smaller eps1: superset
        prev = got
    assert O.select(fci, np.ones((1, fci.shape[0])), 1e-6).shape[0] == 0


# ---------------------------------------------------------------- screened Epstein-Nesbet PT2 (Sec. II.B, Eq. 7)

def test_pt2_matches_dense_hamiltonian(oracle_mod):
    """dE2(eps2) equals the screened sum read off the dense full-CI matrix:
    num_a = sum_i H_ai c_i over the terms with |H_ai c_i| >= eps2, a outside
    V, dE2 = sum_a num_a^2 / (E_V - H_aa); from one determinant with eps2 -> 0
    it is the textbook second-order Epstein-Nesbet energy; the full space has
    none."""
    n, na, nb = 8, 3, 2
    h, eri, ec = S.integrals(n, 10, 4242)
    fci = S.fci_dets(n, na, nb)
    O = oracle_mod.System(h, eri, ec)
    H = O.dense_h(fci)
    rng = np.random.default_rng(11)
    vidx = np.sort(rng.choice(fci.shape[0], 30, replace=False))
    c = rng.standard_normal(vidx.size)
    c /= np.linalg.norm(c)
    e_var = float(c @ H[np.ix_(vidx, vidx)] @ c)
    out = np.setdiff1d(np.arange(fci.shape[0]), vidx)
    for eps2 in (1e-2, 1e-3, 1e-12):
        T = H[np.ix_(out, vidx)] * c[None, :]
        T[np.abs(T) < eps2] = 0.0
        num = T.sum(axis=1)
        keep = np.any(T != 0.0, axis=1)
        want = float(np.sum(num[keep] ** 2 / (e_var - np.diag(H)[out][keep])))
        got, npert = O.pt2(fci[vidx], c, e_var, eps2)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want))
        assert npert == int(keep.sum())
    hf = 0
    e0 = H[hf, hf]
    others = np.arange(1, fci.shape[0])
    want = float(np.sum(H[others, hf] ** 2 / (e0 - np.diag(H)[others])))
    got, _ = O.pt2(fci[:1], np.ones(1), e0, 1e-300)
    assert abs(got - want) <= 1e-12 * abs(want)
    assert O.pt2(fci, np.ones(fci.shape[0]) / np.sqrt(fci.shape[0]), 0.0, 1e-8) == (0.0, 0)


def test_stochastic_pt2_is_unbiased_exactly(oracle_mod):
    """The sample estimator of Sec. II.B (Eq. 9) averaged over every possible
    sample of n_d draws (multinomial weights, p_i = |c_i| / sum |c|, Eq. 10)
    equals the deterministic screened energy (Eq. 7) at both thresholds: the
    exact expectation over all multisets, not a statistical estimate."""
    import math
    n, na, nb = 6, 2, 2
    h, eri, ec = S.integrals(n, 8, 77)
    fci = S.fci_dets(n, na, nb)
    O = oracle_mod.System(h, eri, ec)
    rng = np.random.default_rng(5)
    vidx = np.sort(rng.choice(fci.shape[0], 4, replace=False))
    v = fci[vidx]
    c = rng.standard_normal(4)
    c /= np.linalg.norm(c)
    e_var = float(c @ O.dense_h(v) @ c)
    p = np.abs(c) / np.abs(c).sum()
    eps2, eps2_d = 1e-3, 5e-2
    for n_d in (2, 3, 4):
        exp_all = exp_d = 0.0
        for combo in itertools.combinations_with_replacement(range(4), n_d):
            w = np.bincount(combo, minlength=4)
            prob = math.factorial(n_d) / np.prod([math.factorial(k) for k in w]) * np.prod(p ** w)
            s_all, s_d = O.pt2_sample(v, c, e_var, eps2, eps2_d, np.array(combo))
            exp_all += prob * s_all
            exp_d += prob * s_d
        det_all, _ = O.pt2(v, c, e_var, eps2)
        det_d, _ = O.pt2(v, c, e_var, eps2_d)
        assert abs(exp_all - det_all) <= 1e-12 * abs(det_all)
        assert abs(exp_d - det_d) <= 1e-12 * abs(det_d)
