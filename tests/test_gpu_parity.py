"""GPU path vs the CPU oracle, through the C ABI.

Bars: connected pair sets bit-exact; H_ij (signed, same convention) and H_ii
within 1e-12 Ha; sigma within 1e-12 of the row scale sum_j |H_ij c_j|;
eigenvalues within 1e-9 Ha.
"""
import time

import numpy as np
import pytest
import torch

import shci_synth as S
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

HIJ_TOL = 1e-12
E_TOL = 1e-9
SIGMA_REL = 1e-12


@pytest.fixture(scope="module")
def P():
    return G.lib()


@pytest.fixture(scope="module")
def fci(oracle_mod):
    cfg, h, eri, ec, dets = G.system("fci_10o_4a4b")
    O = oracle_mod.System(h, eri, ec)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    return dict(cfg=cfg, h=h, eri=eri, ec=ec, dets=dets, O=O, ii=ii, jj=jj)


def _check_pairs_and_values(B, O, dets, ii, jj):
    gi, gj, gv = B.pairs()
    assert gi.size == ii.size
    assert np.array_equal(gi, ii) and np.array_equal(gj, jj)
    ov = O.hij_list(dets, ii, jj)
    err = np.max(np.abs(gv - ov)) if ov.size else 0.0
    assert err < HIJ_TOL, err
    d = B.diag()
    assert np.max(np.abs(d - O.hdiag(dets))) < HIJ_TOL


def test_fci_space_pairs_values_diag(P, fci):
    B = G.Built(P, fci["h"], fci["eri"], fci["ec"], fci["dets"], 4, 4)
    assert B.nnz == 44100 * 804 // 2
    _check_pairs_and_values(B, fci["O"], fci["dets"], fci["ii"], fci["jj"])
    B.close()


def test_fci_space_sigma_and_energy(P, fci, oracle_mod):
    dets, O = fci["dets"], fci["O"]
    B = G.Built(P, fci["h"], fci["eri"], fci["ec"], dets, 4, 4)
    c = S.random_vectors(dets.shape[0], 2, 77)
    ref = oracle_mod.sigma_pairs(dets.shape[0], fci["ii"], fci["jj"], O.hij_list(dets, fci["ii"], fci["jj"]),
                                 O.hdiag(dets), c)
    for k in (1, 2):
        got = B.sigma(c[:k])
        rows = np.arange(0, dets.shape[0], 97)
        scale = G.row_scale(O, dets, c[:k], rows)
        assert np.all(np.abs(got[:, rows] - ref[:k, rows]) <= SIGMA_REL * scale + 1e-300)
        assert np.max(np.abs(got - ref[:k])) < 1e-10
    e_ref, _ = O.lowest_eigenpairs(dets, 1, tol=1e-12)
    e, vecs, it = B.davidson(1, tol=1e-10)
    assert abs(e[0] - e_ref[0]) < E_TOL, (e, e_ref)
    # the returned vector is a normalised eigenvector
    hv = B.sigma(vecs)
    assert abs(np.linalg.norm(vecs[0]) - 1.0) < 1e-10
    assert np.linalg.norm(hv[0] - e[0] * vecs[0]) < 1e-5
    B.close()


@pytest.mark.parametrize("name,n_det", [
    ("sel_24o_6a6b_1m", 1), ("sel_24o_6a6b_1m", 2), ("sel_24o_6a6b_1m", 37), ("sel_24o_6a6b_1m", 2053),
    ("sel_24o_6a6b_1m", 20000), ("sel_20o_5a5b_1m", 4099), ("sel_20o_5a5b_1m", 30000),
    ("sel_76o_14a14b_50m", 3001),
])
def test_selected_space_pairs_values(P, oracle_mod, name, n_det):
    cfg, h, eri, ec, dets = G.system(name, n_det)
    O = oracle_mod.System(h, eri, ec)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta)
    assert B.nnz == ii.size
    _check_pairs_and_values(B, O, dets, ii, jj)
    if n_det >= 2:
        c = S.random_vectors(dets.shape[0], 3, 5)
        got = B.sigma(c)
        ref = oracle_mod.sigma_pairs(dets.shape[0], ii, jj, O.hij_list(dets, ii, jj), O.hdiag(dets), c)
        rows = np.unique(np.linspace(0, dets.shape[0] - 1, 64).astype(np.int64))
        scale = G.row_scale(O, dets, c, rows)
        assert np.all(np.abs(got[:, rows] - ref[:, rows]) <= SIGMA_REL * scale + 1e-300)
    B.close()


@pytest.mark.parametrize("name,n_det", [("fci_10o_4a4b", None), ("sel_24o_6a6b_1m", 20000),
                                        ("sel_20o_5a5b_1m", 4099), ("sel_76o_14a14b_50m", 5003)])
def test_on_the_fly_sigma_and_energy(P, oracle_mod, name, n_det):
    """The direct (on-the-fly) product matches the oracle without storing H."""
    cfg, h, eri, ec, dets = G.system(name, n_det)
    O = oracle_mod.System(h, eri, ec)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_ON_THE_FLY)
    assert B.stats()["mode"] == P.SHCI_ON_THE_FLY
    assert B.nnz == ii.size
    with pytest.raises(P.ShciError):
        B.pairs()                                  # nothing stored
    n = dets.shape[0]
    c = S.random_vectors(n, 3, 13)
    ref = oracle_mod.sigma_pairs(n, ii, jj, O.hij_list(dets, ii, jj), O.hdiag(dets), c)
    rows = np.unique(np.linspace(0, n - 1, 64).astype(np.int64))
    scale = G.row_scale(O, dets, c, rows)
    for k in (1, 2, 3):
        got = B.sigma(c[:k])
        assert np.all(np.abs(got[:, rows] - ref[:k, rows]) <= SIGMA_REL * scale[:k] + 1e-300)
        assert np.max(np.abs(got - ref[:k])) < 1e-10
    if n <= 20000:
        e_ref, _ = O.lowest_eigenpairs(dets, 1, tol=1e-12)
        e, vecs, it = B.davidson(1, tol=1e-10)
        assert abs(e[0] - e_ref[0]) < E_TOL
    B.close()


@pytest.mark.parametrize("opp", ["scan", "lookup", "auto"])
@pytest.mark.parametrize("name,n_det", [("sel_24o_6a6b_1m", 20000), ("sel_76o_14a14b_50m", 3001),
                                        ("fci_10o_4a4b", None)])
def test_opposite_spin_strategies(P, oracle_mod, monkeypatch, opp, name, n_det):
    """Every opposite-spin strategy (scanning alpha groups; looking up
    (alpha single, beta single) pairs in the occupancy bitmap; choosing per
    alpha single) gives the same pairs, values and on-the-fly sigma."""
    monkeypatch.setenv("SHCI_OPP_SPIN", opp)
    cfg, h, eri, ec, dets = G.system(name, n_det)
    O = oracle_mod.System(h, eri, ec)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta)
    _check_pairs_and_values(B, O, dets, ii, jj)
    B.close()
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_ON_THE_FLY)
    n = dets.shape[0]
    c = S.random_vectors(n, 2, 17)
    ref = oracle_mod.sigma_pairs(n, ii, jj, O.hij_list(dets, ii, jj), O.hdiag(dets), c)
    got = B.sigma(c)
    assert np.max(np.abs(got - ref)) < 1e-10
    B.close()


def test_selected_space_two_roots(P, oracle_mod):
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m", 20000)
    O = oracle_mod.System(h, eri, ec)
    e_ref, _ = O.lowest_eigenpairs(dets, 2, tol=1e-12)
    B = G.Built(P, h, eri, ec, dets, 6, 6)
    e, vecs, it = B.davidson(2, tol=1e-10)
    np.testing.assert_allclose(e, e_ref, atol=E_TOL, rtol=0)
    np.testing.assert_allclose(vecs @ vecs.T, np.eye(2), atol=1e-10)
    # the convergence history: one row per iteration, ending on the returned energies
    th, rn, ts = P.shci_davidson_history(B.ctx.handle, 2)
    assert th.shape == (it, 2) and rn.shape == (it, 2) and ts.shape == (it,)
    np.testing.assert_array_equal(th[-1], e)
    assert np.all(np.diff(ts) >= 0.0) and ts[0] >= 0.0
    assert np.all(rn[-1] < 0.1 * np.sqrt(1e-10))
    assert np.all(np.diff(th[:, 0]) <= 1e-10)        # Ritz values never rise (thick restart keeps them)
    # the part timer: every part accounted, summing to about the call's device time
    P.shci_set_timing(B.ctx.handle, False, davidson_phases=True)
    t0 = time.perf_counter()
    e3, _, _ = B.davidson(2, tol=1e-10)
    wall_ms = (time.perf_counter() - t0) * 1e3
    parts = B.stats()["davidson_phase_ms"]
    np.testing.assert_array_equal(e3, e)
    assert all(x >= 0.0 for x in parts) and parts[1] > 0.0 and parts[5] > 0.0
    assert 0.3 * wall_ms < sum(parts) <= wall_ms * 1.05 + 1.0
    P.shci_set_timing(B.ctx.handle, False)
    # restarting from the converged vectors converges at once to the same roots
    e2, _, it2 = B.davidson(2, tol=1e-10, guess=vecs)
    np.testing.assert_allclose(e2, e_ref, atol=E_TOL, rtol=0)
    assert it2 <= 3
    B.close()


@pytest.mark.parametrize("name", ["sel_24o_6a6b_1m", "sel_20o_5a5b_1m", "sel_24o_6a6b_1m_standin"])
def test_full_size_selected_space_sampled_rows(P, oracle_mod, name):
    """|V| = 1e6 at the workloads' full size: sampled rows against the
    brute-force oracle (columns bit-exact, values, sigma rows), the
    eigen-residual of the GPU Ritz vectors on sampled rows, and -- for the
    heat-bath-selected spaces -- the eigenvalues against the oracle's energies
    of the whole space (Davidson on its own upper-triangle rows, stored with
    the space by tests/golden/make_selected_spaces.py)."""
    cfg, h, eri, ec, dets = G.system(name)
    O = oracle_mod.System(h, eri, ec)
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta)
    rng = np.random.default_rng(11)
    rows = np.concatenate([[0, 1, dets.shape[0] - 1], rng.choice(dets.shape[0], 60, replace=False)])
    for i in rows:
        cols, vals = O.row(dets, int(i))
        gc, gv = B.row(int(i))
        assert np.array_equal(gc, cols), i
        assert np.max(np.abs(gv - vals)) < HIJ_TOL
    k = cfg.roots
    c = S.random_vectors(dets.shape[0], k, 9)
    got = B.sigma(c)
    ref = O.sigma_rows(dets, c, rows)
    scale = G.row_scale(O, dets, c, rows)
    assert np.all(np.abs(got[:, rows] - ref) <= SIGMA_REL * scale + 1e-300)
    e, vecs, it = B.davidson(k, tol=1e-10)
    hv = O.sigma_rows(dets, vecs, rows)
    r = hv - e[:, None] * vecs[:, rows]
    assert np.max(np.abs(r)) < 1e-5
    assert np.all(np.diff(e) > 0)
    if cfg.space == "heat-bath":
        meta = S.selected_space_meta(name)
        assert B.nnz == meta["oracle"]["nnz_upper"]
        np.testing.assert_allclose(e, meta["oracle"]["energies"][:k], atol=E_TOL, rtol=0)
    B.close()


def test_host_memory_path_matches_device_path(P, oracle_mod):
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m", 5000)
    Bd = G.Built(P, h, eri, ec, dets, 5, 5)
    Bh = G.Built(P, h, eri, ec, dets, 5, 5, host=True)
    assert Bd.nnz == Bh.nnz
    c = S.random_vectors(dets.shape[0], 2, 3)
    yh = np.empty_like(c)
    P.shci_sigma(Bh.ctx.handle, c, yh)
    np.testing.assert_array_equal(yh, Bd.sigma(c))
    e = np.empty(1)
    ev = np.empty((1, dets.shape[0]))
    e1, it1, rc1 = P.shci_davidson(Bh.ctx.handle, 1, 1e-10, 300, vecs=ev)
    e2, _, _ = Bd.davidson(1)
    assert abs(e1[0] - e2[0]) < 1e-10
    Bd.close()
    Bh.close()


def test_invalid_inputs_are_rejected(P):
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m", 500)
    ctx = P.Context(0, torch.cuda.current_stream())
    H = ctx.handle
    with pytest.raises(P.ShciError) as e:
        P.shci_sigma(H, G.dev(np.zeros((1, 500))), torch.zeros((1, 500), dtype=torch.float64, device="cuda"))
    assert e.value.code == 6                      # state: nothing built
    P.shci_load_integrals(H, 20, ec, G.dev(h), G.dev(eri))
    dup = np.concatenate([dets, dets[7:8]])
    with pytest.raises(P.ShciError) as e:
        P.shci_build_connectivity(H, 5, 5, G.dev(dup))
    assert e.value.code == 1
    with pytest.raises(P.ShciError) as e:
        P.shci_build_connectivity(H, 4, 5, G.dev(dets))   # wrong alpha electron count
    assert e.value.code == 1
    bad = dets.copy()
    bad[3, 0] = np.uint64(bad[3, 0]) | np.uint64(1 << 40)   # orbital beyond n_orb (and a 6th electron)
    with pytest.raises(P.ShciError):
        P.shci_build_connectivity(H, 5, 5, G.dev(bad))
    hb = h.copy()
    hb[0, 1] += 1e-6
    with pytest.raises(P.ShciError):
        P.shci_load_integrals(H, 20, ec, G.dev(hb), G.dev(eri))
    P.shci_load_integrals(H, 20, ec, G.dev(h), G.dev(eri))
    P.shci_build_connectivity(H, 5, 5, G.dev(dets))
    with pytest.raises(P.ShciError):
        x = torch.zeros((9, 500), dtype=torch.float64, device="cuda")
        P.shci_sigma(H, x, torch.zeros_like(x))      # k out of range
    e, it, rc = P.shci_davidson(H, 1, 1e-14, 1, check=False)
    assert rc == 4                                # not converged in one iteration
    ctx.close()


def test_no_beta_electrons(P, oracle_mod):
    n = 9
    h, eri, _ = S.integrals(n, 6, 123)
    dets = S.fci_dets(n, 3, 0)
    O = oracle_mod.System(h, eri, 0.0)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    B = G.Built(P, h, eri, 0.0, dets, 3, 0)
    _check_pairs_and_values(B, O, dets, ii, jj)
    w = np.linalg.eigvalsh(O.dense_h(dets))[:2]
    e, _, _ = B.davidson(2, tol=1e-12)
    np.testing.assert_allclose(e, w, atol=E_TOL)
    B.close()
