"""The upper-triangle stored form (SHCI_STORED_UPPER: H_ij with i < j only, the
transposed half added by atomic adds) against the oracle, against the
both-triangle form, under incremental growth of V, when SHCI_AUTO picks it
for lack of memory, and inside the batched solver's storage plan.

Bars: the stored pairs bit-identical to the both-triangle build's upper
triangle (the same pair is evaluated from the same row) and equal to the
oracle's pair set, values within 1e-12 Ha; sigma within 1e-12 of the row
scale sum_j |H_ij c_j| (the atomic adds change only the summation order);
eigenvalues within 1e-9 Ha."""
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


def _sigma_checks(P, B, O, oracle_mod, dets, ii, jj, ks, seed):
    n = dets.shape[0]
    c = S.random_vectors(n, max(ks), seed)
    ref = oracle_mod.sigma_pairs(n, ii, jj, O.hij_list(dets, ii, jj), O.hdiag(dets), c)
    rows = np.unique(np.linspace(0, n - 1, 64).astype(np.int64))
    scale = G.row_scale(O, dets, c, rows)
    for k in ks:
        got = B.sigma(c[:k])
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got[:, rows] - ref[:k, rows]) <= SIGMA_REL * scale[:k] + 1e-300), k
        assert np.max(np.abs(got - ref[:k])) < 1e-10, k


@pytest.mark.parametrize("name,n_det", [
    ("sel_24o_6a6b_1m", 1), ("sel_24o_6a6b_1m", 2), ("sel_24o_6a6b_1m", 37), ("sel_24o_6a6b_1m", 20000),
    ("sel_20o_5a5b_1m", 4099), ("sel_76o_14a14b_50m", 3001), ("fci_10o_4a4b", None),
])
def test_upper_matches_oracle_and_both_triangles(P, oracle_mod, name, n_det):
    cfg, h, eri, ec, dets = G.system(name, n_det)
    O = oracle_mod.System(h, eri, ec)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    U = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_STORED_UPPER)
    assert U.stats()["mode"] == P.SHCI_STORED_UPPER
    assert U.nnz == ii.size
    ui, uj, uv = U.pairs()
    assert np.array_equal(ui, ii) and np.array_equal(uj, jj)
    ov = O.hij_list(dets, ii, jj)
    assert (np.max(np.abs(uv - ov)) if ov.size else 0.0) < HIJ_TOL
    F = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta)
    fi, fj, fv = F.pairs()
    assert np.array_equal(fi, ui) and np.array_equal(fj, uj)
    assert np.array_equal(fv.view(np.uint64), uv.view(np.uint64))
    F.close()
    with pytest.raises(P.ShciError):
        U.row(0)                                   # a row's lower part is not held as a row
    n = dets.shape[0]
    if n >= 2:
        _sigma_checks(P, U, O, oracle_mod, dets, ii, jj, (1, 2, 3, 4, 8), 17)
    if 37 <= n <= 20000:
        k = 2
        w = O.lowest_eigenpairs(dets, k, tol=1e-12)[0]
        e, vecs, it = U.davidson(k, tol=1e-10)
        np.testing.assert_allclose(e, w, atol=E_TOL, rtol=0)
    U.close()


def test_upper_interleaved_products_inside_davidson(P, oracle_mod):
    """Four roots (the interleaved products of blocks of up to four vectors)."""
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m", 6000)
    O = oracle_mod.System(h, eri, ec)
    U = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_STORED_UPPER)
    e, vecs, it = U.davidson(4, tol=1e-11)
    w = O.lowest_eigenpairs(dets, 4, tol=1e-12)[0]
    np.testing.assert_allclose(e, w, atol=E_TOL, rtol=0)
    hv = U.sigma(vecs)
    for a in range(4):
        assert np.linalg.norm(hv[a] - e[a] * vecs[a]) < 1e-4
    U.close()


@pytest.mark.parametrize("name,n_det,splits", [
    ("sel_24o_6a6b_1m", 6000, [4000, 5000, 5900]),
    ("sel_20o_5a5b_1m", 4099, [1, 2, 1000]),
])
def test_upper_grows_incrementally(P, oracle_mod, name, n_det, splits):
    """An upper-triangle matrix grown in steps equals a fresh upper build of the
    grown V bit for bit, and the oracle."""
    cfg, h, eri, ec, dets = G.system(name, n_det)
    U = G.Built(P, h, eri, ec, dets[:splits[0]], cfg.n_alpha, cfg.n_beta, mode=P.SHCI_STORED_UPPER)
    bounds = splits + [dets.shape[0]]
    for a, b in zip(bounds[:-1], bounds[1:]):
        nnz = P.shci_extend_connectivity(U.ctx.handle, G.dev(dets[a:b]), 1.0)
        st = U.stats()
        assert st["extend_incremental"] == 1 and st["mode"] == P.SHCI_STORED_UPPER
    U.dets, U.n, U.nnz = dets, dets.shape[0], nnz
    O = oracle_mod.System(h, eri, ec)
    ii, jj = oracle_mod.pairs_allpairs(dets)
    assert nnz == ii.size
    F = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_STORED_UPPER)
    fi, fj, fv = F.pairs()
    gi, gj, gv = U.pairs()
    assert np.array_equal(fi, gi) and np.array_equal(fj, gj) and np.array_equal(fi, ii) and np.array_equal(fj, jj)
    assert np.array_equal(fv.view(np.uint64), gv.view(np.uint64))
    F.close()
    _sigma_checks(P, U, O, oracle_mod, dets, ii, jj, (2,), 29)
    U.close()


def test_auto_picks_the_upper_triangle_when_memory_is_short(P, oracle_mod):
    """With free device memory between the upper triangle's and both triangles'
    size (after the 0.8 margin), SHCI_AUTO stores the upper triangle; with
    the memory back it stores both."""
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    f0 = torch.cuda.mem_get_info()[0]
    C = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_ON_THE_FLY)
    torch.cuda.synchronize()
    held = f0 - torch.cuda.mem_get_info()[0]     # lists, diagonal and row counts, held at the decision
    need = 12.0 * 2 * C.nnz                       # both triangles, bytes
    C.close()
    torch.cuda.synchronize()
    free = torch.cuda.mem_get_info()[0]
    # leave free memory F with 0.8 (F - held) = 0.75 need: between the upper (0.5 need) and both triangles
    target = max(held, 0) + int(0.9375 * need)
    assert need > (256 << 20) and free > target + (1 << 30)
    blocker = torch.empty(free - target, dtype=torch.uint8, device="cuda")
    try:
        U = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_AUTO)
        assert U.stats()["mode"] == P.SHCI_STORED_UPPER
        O = oracle_mod.System(h, eri, ec)
        c = S.random_vectors(dets.shape[0], 2, 3)
        got = U.sigma(c)
        rows = np.unique(np.linspace(0, dets.shape[0] - 1, 24).astype(np.int64))
        orc = O.sigma_rows(dets, c, rows)
        scale = G.row_scale(O, dets, c, rows)
        assert np.all(np.abs(got[:, rows] - orc) <= SIGMA_REL * scale + 1e-300)
        U.close()
    finally:
        del blocker
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    A = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_AUTO)
    assert A.stats()["mode"] == P.SHCI_STORED
    A.close()


def test_auto_growth_that_no_longer_fits_rebuilds(P, oracle_mod):
    """SHCI_AUTO, both triangles stored, grown incrementally (threshold 1.0) with
    free memory at which the grown matrix's both triangles do not fit but its
    upper triangle does: the update gives up and V is rebuilt (the old matrix
    released first), in the best form that then fits; the result matches the
    oracle."""
    cfg, h, eri, ec, dets = G.system("sel_24o_6a6b_1m")
    n0 = 600000
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    C = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_ON_THE_FLY)
    nnz_all = C.nnz
    need = 12.0 * 2 * nnz_all                     # the grown space's both triangles
    C.close()
    A = G.Built(P, h, eri, ec, dets[:n0], cfg.n_alpha, cfg.n_beta, mode=P.SHCI_AUTO)
    assert A.stats()["mode"] == P.SHCI_STORED
    torch.cuda.synchronize()
    free = torch.cuda.mem_get_info()[0]
    # the update's lists and counts take well under 0.5 GB here: 0.8 x the free
    # memory at its decision lies between the upper triangle (0.5 need) and need
    target = int(0.9375 * need) + (512 << 20)
    assert need > (1 << 30) and free > target + (1 << 30)
    blocker = torch.empty(free - target, dtype=torch.uint8, device="cuda")
    try:
        nnz = P.shci_extend_connectivity(A.ctx.handle, G.dev(dets[n0:]), 1.0)
        st = A.stats()
        assert st["extend_incremental"] == 0               # gave up the update and rebuilt V
        assert st["mode"] in (P.SHCI_STORED, P.SHCI_STORED_UPPER)
        assert nnz == nnz_all and st["n_det"] == dets.shape[0]
        A.dets, A.n, A.nnz = dets, dets.shape[0], nnz
        O = oracle_mod.System(h, eri, ec)
        c = S.random_vectors(dets.shape[0], 2, 8)
        got = A.sigma(c)
        rows = np.unique(np.linspace(0, dets.shape[0] - 1, 24).astype(np.int64))
        orc = O.sigma_rows(dets, c, rows)
        scale = G.row_scale(O, dets, c, rows)
        assert np.all(np.abs(got[:, rows] - orc) <= SIGMA_REL * scale + 1e-300)
        A.close()
    finally:
        del blocker
        torch.cuda.synchronize()
        torch.cuda.empty_cache()


def _batch_systems(n_sys, cap, seed):
    out = []
    for cfg in S.batch_configs(n_sys=n_sys, seed=seed):
        hh, ee, ec, dets = S.make_system(cfg, n_det=min(cfg.n_det, cap))
        out.append(dict(cfg=cfg, n_orb=cfg.n_orb, n_alpha=cfg.n_alpha, n_beta=cfg.n_beta, h=hh, eri=ee,
                        e_core=ec, dets=dets))
    return out


def test_batch_storage_plan_with_upper_triangles(P, oracle_mod):
    """The batch's plan by ascending pair count: a budget that holds every upper
    triangle plus the two smallest systems' lower ones stores those two in
    both triangles and the rest as upper triangles; one that holds only the
    three smallest upper triangles applies the others on the fly.  Energies
    match the oracle either way."""
    systems = _batch_systems(6, 3000, 5200)
    nnz = []
    for d in systems:
        C = G.Built(P, d["h"], d["eri"], d["e_core"], d["dets"], d["n_alpha"], d["n_beta"], mode=P.SHCI_ON_THE_FLY)
        nnz.append(C.nnz)
        C.close()
    nnz = np.array(nnz, np.float64)
    order = np.argsort(nnz, kind="stable")
    plans = [
        (12.0 * (nnz.sum() + nnz[order[:2]].sum()) + 64.0,
         {int(s): P.SHCI_STORED if r < 2 else P.SHCI_STORED_UPPER for r, s in enumerate(order)}),
        (12.0 * nnz[order[:3]].sum() + 64.0,
         {int(s): P.SHCI_STORED_UPPER if r < 3 else P.SHCI_ON_THE_FLY for r, s in enumerate(order)}),
    ]
    k = 3
    ref = [np.linalg.eigvalsh(oracle_mod.System(d["h"], d["eri"], d["e_core"]).dense_h(d["dets"]))[:k]
           for d in systems]
    for budget, want in plans:
        ctx = P.Context(0, torch.cuda.current_stream())
        b = P.shci_batch_create(ctx.handle, systems, stored_budget_bytes=budget)
        modes = P.shci_batch_get_modes(b, len(systems))
        assert [int(m) for m in modes] == [want[s] for s in range(len(systems))]
        st = P.shci_batch_get_stats(b)
        assert st["n_stored"] == sum(m == P.SHCI_STORED for m in want.values())
        assert st["n_stored_upper"] == sum(m == P.SHCI_STORED_UPPER for m in want.values())
        assert st["n_on_the_fly"] == sum(m == P.SHCI_ON_THE_FLY for m in want.values())
        e, it, conv, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), k, tol=1e-10, max_iter=400)
        assert rc == 0 and conv.all()
        for s in range(len(systems)):
            np.testing.assert_allclose(e[s], ref[s], atol=E_TOL, rtol=0)
        P.shci_batch_destroy(b)
        ctx.close()


def test_batch_all_upper_matches_sequential_upper_solves(P):
    """Every system stored as its upper triangle (a budget of exactly their
    size): the batched energies equal one-at-a-time SHCI_STORED_UPPER solves."""
    systems = _batch_systems(8, 40000, 5100)
    nnz = []
    for d in systems:
        C = G.Built(P, d["h"], d["eri"], d["e_core"], d["dets"], d["n_alpha"], d["n_beta"], mode=P.SHCI_ON_THE_FLY)
        nnz.append(C.nnz)
        C.close()
    ctx = P.Context(0, torch.cuda.current_stream())
    b = P.shci_batch_create(ctx.handle, systems, stored_budget_bytes=12.0 * float(sum(nnz)) + 64.0)
    assert all(int(m) == P.SHCI_STORED_UPPER for m in P.shci_batch_get_modes(b, len(systems)))
    e, it, conv, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), 4, tol=1e-10)
    assert rc == 0
    for s, d in enumerate(systems):
        U = G.Built(P, d["h"], d["eri"], d["e_core"], d["dets"], d["n_alpha"], d["n_beta"], mode=P.SHCI_STORED_UPPER)
        es, _, _ = U.davidson(4, tol=1e-10)
        U.close()
        np.testing.assert_allclose(e[s], es, atol=E_TOL, rtol=0)
    P.shci_batch_destroy(b)
    ctx.close()
