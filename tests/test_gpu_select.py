"""Heat-bath selection (Sec. II.A, Eq. 2) on the GPU against the oracle's brute
force: the selected sets are compared as sets of determinants, bit-exact.
The GPU tests |H_ai| |c_i| >= eps1 in FP64 with matrix elements summed in
another order than the oracle's.  A matrix element is a sum of at most
m = 2 n_e + 1 terms; two summation orders of the same terms differ by at most
2 gamma_{m-1} sum|t|, gamma_j = j u / (1 - j u), u = 2^-53 (the bound on
recursive summation): about 6e-15 sum|t| for the 28 electrons of the largest
case.  BAND = 1e-12 relative covers term sums up to ~160 times the element, so
products within BAND of eps1 may fall either way: the GPU set at eps1 must
contain the oracle set at eps1 (1 + BAND) and lie inside the oracle set at
eps1 (1 - BAND)."""
import numpy as np
import pytest
import torch

import shci_synth as S
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

BAND = 1e-12

@pytest.fixture(scope="module")
def P():
    return G.lib()


def _rows(a):
    a = np.asarray(a)
    if a.dtype != np.uint64:
        a = a.view(np.uint64)
    return {tuple(int(x) for x in d) for d in a}


def _check(P, O, B, dets, c, eps1, device=True):
    cc = G.dev(c) if device else np.ascontiguousarray(c)
    got = P.shci_select(B.ctx.handle, cc, eps1)
    got = got.cpu().numpy() if device else got
    g = _rows(got)
    assert len(g) == got.shape[0]                              # no repeats
    keys = [tuple(int(x) for x in d[::-1]) for d in got.view(np.uint64)]
    assert keys == sorted(keys)                                # ascending, last word most significant
    ref, best = O.select(dets, c, eps1 * (1 - BAND), with_best=True)
    hi = _rows(ref)
    lo = _rows(ref[best >= eps1 * (1 + BAND)])
    assert lo <= g <= hi
    assert not (g & _rows(dets))                               # nothing already in V
    st = P.shci_get_stats(B.ctx.handle)
    assert st["select_candidates"] >= got.shape[0] and st["select_ms"] > 0.0
    return g


def test_from_one_determinant_every_connection(P, oracle_mod):
    h, eri, ec = S.integrals(10, 20, 1000)
    hf = S.fci_dets(10, 4, 4)[:1]
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, hf, 4, 4)
    g = _check(P, O, B, hf, np.ones((1, 1)), 1e-12)
    assert len(g) == 804
    B.close()


@pytest.mark.parametrize("eps1", [3e-2, 3e-3, 3e-4])
def test_full_ci_subset(P, oracle_mod, eps1):
    cfg, h, eri, ec, dets = G.system("fci_10o_4a4b", None)
    rng = np.random.default_rng(7)
    v = dets[np.sort(rng.choice(dets.shape[0], 400, replace=False))]
    c = rng.standard_normal((2, v.shape[0])) / np.sqrt(v.shape[0])
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, v, 4, 4)
    g = _check(P, O, B, v, c, eps1)
    assert len(g) > 0
    B.close()


def test_selected_space_ground_state_coefficients(P, oracle_mod):
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m", 600)
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, dets, 6, 6)
    e, vecs, it = B.davidson(1, tol=1e-10)
    for eps1 in (1e-3, 1e-4):
        g = _check(P, O, B, dets, vecs, eps1)
        assert len(g) > 0
    # host coefficients give the same set
    assert _check(P, O, B, dets, vecs, 1e-3, device=False) == _check(P, O, B, dets, vecs, 1e-3)
    B.close()


def test_two_word_strings(P, oracle_mod):
    cfg, h, eri, ec, dets = G.system("sel_76o_14a14b_50m", 12)
    rng = np.random.default_rng(5)
    c = rng.standard_normal((1, dets.shape[0]))
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, dets, 14, 14)
    g = _check(P, O, B, dets, c, 2e-2)
    assert len(g) > 0
    B.close()


def test_full_space_selects_nothing_and_bad_arguments(P, oracle_mod):
    h, eri, ec = S.integrals(8, 10, 4242)
    fci = S.fci_dets(8, 3, 2)
    B = G.Built(P, h, eri, ec, fci, 3, 2)
    c = G.dev(np.ones((1, fci.shape[0])))
    assert P.shci_select(B.ctx.handle, c, 1e-8).shape[0] == 0
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(P.ShciError):
            P.shci_select(B.ctx.handle, c, bad)
    with pytest.raises(P.ShciError):
        P.shci_select(B.ctx.handle, G.dev(np.ones((9, fci.shape[0]))), 1e-3)   # k out of range
    B.close()


# ---------------------------------------------------------------- screened Epstein-Nesbet PT2 (Sec. II.B, Eq. 7)

def _pt2_check(P, O, B, dets, c, e_var, eps2, n_batches=0):
    """GPU dE2 against the oracle's.  Terms within BAND of eps2 may be kept on
    one side and dropped on the other: the GPU value must match the oracle
    at eps2 (1 - BAND) or at eps2 (1 + BAND), to 1e-10 relative."""
    got, npert = P.shci_pt2(B.ctx.handle, G.dev(c), e_var, eps2, n_batches)
    lo = O.pt2(dets, c, e_var, eps2 * (1 - BAND))
    hi = O.pt2(dets, c, e_var, eps2 * (1 + BAND))
    ok = [abs(got - r[0]) <= 1e-10 * max(1e-6, abs(r[0])) and npert == r[1] for r in (lo, hi)]
    assert any(ok), (got, npert, lo, hi)
    st = P.shci_get_stats(B.ctx.handle)
    assert st["pt2_ms"] > 0.0 and st["pt2_batches"] >= 1 and st["pt2_terms"] >= npert
    return got, npert


def test_pt2_full_ci_subset_and_batches(P, oracle_mod):
    n, na, nb = 8, 3, 2
    h, eri, ec = S.integrals(n, 10, 4242)
    fci = S.fci_dets(n, na, nb)
    rng = np.random.default_rng(11)
    v = fci[np.sort(rng.choice(fci.shape[0], 30, replace=False))]
    O = oracle_mod.System(h, eri, ec)
    Hv = O.dense_h(v)
    c = rng.standard_normal(v.shape[0])
    c /= np.linalg.norm(c)
    e_var = float(c @ Hv @ c)
    B = G.Built(P, h, eri, ec, v, na, nb)
    for eps2 in (1e-2, 1e-4, 1e-10):
        ref, npert = _pt2_check(P, O, B, v, c, e_var, eps2)
        for nbt in (1, 3, 7):                        # the batching does not change the sum
            got, np2 = P.shci_pt2(B.ctx.handle, G.dev(c), e_var, eps2, nbt)
            assert np2 == npert and abs(got - ref) <= 1e-13 * abs(ref)
        assert P.shci_get_stats(B.ctx.handle)["pt2_batches"] == 7
    B.close()
    Bf = G.Built(P, h, eri, ec, fci, na, nb)
    assert P.shci_pt2(Bf.ctx.handle, G.dev(np.ones(fci.shape[0])), -1.0, 1e-8) == (0.0, 0)
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(P.ShciError):
            P.shci_pt2(Bf.ctx.handle, G.dev(np.ones(fci.shape[0])), -1.0, bad)
    Bf.close()


def test_pt2_selected_space_ground_state(P, oracle_mod):
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m", 600)
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, dets, 6, 6)
    e, vecs, it = B.davidson(1, tol=1e-10)
    got, npert = _pt2_check(P, O, B, dets, vecs[0], float(e[0]), 1e-5)
    assert got < 0.0 and npert > 0
    # host coefficients, same value
    assert P.shci_pt2(B.ctx.handle, np.ascontiguousarray(vecs[0]), float(e[0]), 1e-5)[0] == got
    B.close()


def test_pt2_two_word_strings(P, oracle_mod):
    cfg, h, eri, ec, dets = G.system("sel_76o_14a14b_50m", 12)
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, dets, 14, 14)
    e, vecs, it = B.davidson(1, tol=1e-10)
    _pt2_check(P, O, B, dets, vecs[0], float(e[0]), 3e-3)
    B.close()


# ---------------------------------------------------------------- stochastic and semistochastic PT2 (Eqs. 8-10)

def _draws(c, n_samples, n_d, seed):
    """Samples of V drawn with p_i proportional to |c_i| (Eq. 10) by a seeded
    generator: the random numbers are an input shared by both sides."""
    p = np.abs(c) / np.abs(c).sum()
    return np.random.default_rng(seed).choice(c.size, size=(n_samples, n_d), p=p).astype(np.int64)


def _samples_check(P, O, B, dets, c, e_var, eps2, eps2_d, draws):
    got = P.shci_pt2_samples(B.ctx.handle, G.dev(c), e_var, eps2, eps2_d, G.dev(draws))
    for s in range(draws.shape[0]):
        refs = [O.pt2_sample(dets, c, e_var, eps2 * f, eps2_d * f, draws[s]) for f in (1 - BAND, 1 + BAND)]
        ok = [all(abs(got[s, j] - r[j]) <= 1e-10 * max(1e-8, abs(r[j])) for j in (0, 1)) for r in refs]
        assert any(ok), (s, got[s], refs)
    return got


def test_pt2_samples_match_oracle(P, oracle_mod):
    n, na, nb = 8, 3, 2
    h, eri, ec = S.integrals(n, 10, 4242)
    fci = S.fci_dets(n, na, nb)
    rng = np.random.default_rng(11)
    v = fci[np.sort(rng.choice(fci.shape[0], 30, replace=False))]
    O = oracle_mod.System(h, eri, ec)
    c = rng.standard_normal(v.shape[0])
    c /= np.linalg.norm(c)
    e_var = float(c @ O.dense_h(v) @ c)
    B = G.Built(P, h, eri, ec, v, na, nb)
    _samples_check(P, O, B, v, c, e_var, 1e-4, 1e-2, _draws(c, 4, 12, 1))
    B.close()
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m", 600)
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, dets, 6, 6)
    e, vecs, it = B.davidson(1, tol=1e-10)
    _samples_check(P, O, B, dets, vecs[0], float(e[0]), 1e-5, 1e-4, _draws(vecs[0], 2, 50, 2))
    B.close()


def test_alias_draws_follow_the_coefficients(P):
    """p_i = |c_i| / sum |c| (Eq. 10): frequencies of 4e6 draws pass a chi-square
    test at a 1e-6 false-alarm level; zero coefficients are never drawn; the
    draws depend only on the seed."""
    from scipy import stats
    h, eri, ec = S.integrals(8, 10, 4242)
    fci = S.fci_dets(8, 3, 2)[:50]
    B = G.Built(P, h, eri, ec, fci, 3, 2)
    c = np.random.default_rng(3).standard_normal(50)
    c[[4, 17, 33]] = 0.0
    n_draws = 4_000_000
    d = P.shci_alias_draw(B.ctx.handle, G.dev(c), n_draws, 12345).cpu().numpy()
    counts = np.bincount(d, minlength=50)
    assert counts[[4, 17, 33]].sum() == 0 and d.min() >= 0 and d.max() < 50
    p = np.abs(c) / np.abs(c).sum()
    nz = p > 0
    chi2 = float(np.sum((counts[nz] - n_draws * p[nz]) ** 2 / (n_draws * p[nz])))
    assert chi2 < stats.chi2.ppf(1 - 1e-6, nz.sum() - 1)
    d2 = P.shci_alias_draw(B.ctx.handle, np.ascontiguousarray(c), 1000, 12345)
    np.testing.assert_array_equal(d2, d[:1000])
    B.close()


def test_semistochastic_pt2(P, oracle_mod):
    """eps2_d = eps2 is the deterministic energy exactly; with eps2_d > eps2 the
    estimate lies within 6 standard errors of the deterministic energy at eps2."""
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m", 600)
    B = G.Built(P, h, eri, ec, dets, 6, 6)
    e, vecs, it = B.davidson(1, tol=1e-10)
    c = G.dev(vecs[0])
    det, _ = P.shci_pt2(B.ctx.handle, c, float(e[0]), 1e-5)
    same, err0 = P.shci_pt2_semistochastic(B.ctx.handle, c, float(e[0]), 1e-5, 1e-5, 100, 4, 7)
    assert abs(same - det) <= 1e-13 * abs(det) and err0 == 0.0
    est, err = P.shci_pt2_semistochastic(B.ctx.handle, c, float(e[0]), 1e-5, 1e-3, 200, 64, 7)
    assert err > 0.0 and abs(est - det) <= 6.0 * err + 1e-12
    B.close()


# ---------------------------------------------------------------- 3-step perturbation scheme (Sec. IV, Eq. 11)

def test_pt2_sample_batches_add_up(P, oracle_mod):
    """A sample's value restricted to each hash batch adds up to its
    unrestricted value (the batches partition the perturbative determinants)."""
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m", 600)
    B = G.Built(P, h, eri, ec, dets, 6, 6)
    e, vecs, it = B.davidson(1, tol=1e-10)
    c = G.dev(vecs[0])
    draws = G.dev(_draws(vecs[0], 2, 40, 9))
    full = P.shci_pt2_samples(B.ctx.handle, c, float(e[0]), 1e-5, 1e-4, draws)
    parts = sum(P.shci_pt2_samples(B.ctx.handle, c, float(e[0]), 1e-5, 1e-4, draws, 5, [b, b]) for b in range(5))
    np.testing.assert_allclose(parts, full, rtol=1e-12, atol=0)
    B.close()


def test_pt2_three_step(P, oracle_mod):
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m", 600)
    B = G.Built(P, h, eri, ec, dets, 6, 6)
    e, vecs, it = B.davidson(1, tol=1e-10)
    c, ev = G.dev(vecs[0]), float(e[0])
    ref = {eps: P.shci_pt2(B.ctx.handle, c, ev, eps)[0] for eps in (1e-6, 1e-5, 1e-4)}
    # every pseudo-stochastic batch (target 0) and no stochastic step: deterministic, exact
    r = P.shci_pt2_3step(B.ctx.handle, c, ev, 1e-5, 1e-5, 1e-4, 0.0, 16, 8, 100, 4, 3)
    assert r["psto_batches"] == 16 and r["psto_err"] == 0.0 and r["sto"] == 0.0 and r["sto_err"] == 0.0
    assert abs(r["dtm"] - ref[1e-4]) <= 1e-13 * abs(ref[1e-4])
    assert abs(r["psto"] - (ref[1e-5] - ref[1e-4])) <= 1e-12 * abs(ref[1e-5])
    assert abs(r["e2"] - ref[1e-5]) <= 1e-12 * abs(ref[1e-5])
    # all three steps: within 6 standard errors of the deterministic energy at eps2
    r = P.shci_pt2_3step(B.ctx.handle, c, ev, 1e-6, 1e-5, 1e-4, 2e-4, 16, 8, 200, 48, 5)
    assert 1 <= r["psto_batches"] <= 16 and r["e2_err"] > 0.0
    assert abs(r["e2"] - ref[1e-6]) <= 6.0 * r["e2_err"] + 1e-12
    B.close()
