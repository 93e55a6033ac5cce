"""Batched solves: many uneven systems and several roots each in one
persistent launch, against the oracle and against one-at-a-time solves."""
import numpy as np
import pytest
import torch

import shci_synth as S
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

E_TOL = 1e-9


@pytest.fixture(scope="module")
def P():
    return G.lib()


def small_batch(n_sys=6, cap=3000, seed=5000):
    out = []
    for cfg in S.batch_configs(n_sys=n_sys, seed=seed):
        n = min(cfg.n_det, cap)
        h, eri, ec, dets = S.make_system(cfg, n_det=n)
        out.append(dict(cfg=cfg, n_orb=cfg.n_orb, n_alpha=cfg.n_alpha, n_beta=cfg.n_beta, h=h, eri=eri,
                        e_core=ec, dets=dets))
    return out


@pytest.mark.parametrize("budget,k", [(-1.0, 4), (0.0, 2), (2.0e7, 3)])
def test_batch_matches_oracle(P, oracle_mod, budget, k):
    systems = small_batch()
    ctx = P.Context(0, torch.cuda.current_stream())
    b = P.shci_batch_create(ctx.handle, systems, stored_budget_bytes=budget)
    st = P.shci_batch_get_stats(b)
    assert st["n_sys"] == len(systems)
    if budget == 0.0:
        assert st["n_on_the_fly"] == len(systems)
    e, it, conv, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), k, tol=1e-10, max_iter=400)
    assert rc == 0 and conv.all()
    for s, d in enumerate(systems):
        O = oracle_mod.System(d["h"], d["eri"], d["e_core"])
        w = np.linalg.eigvalsh(O.dense_h(d["dets"]))[:k]
        np.testing.assert_allclose(e[s], w, atol=E_TOL, rtol=0)
    st = P.shci_batch_get_stats(b)
    assert st["tuned_rows_per_item"] in (64, 256, 1024) and st["tuned_ctas_per_sm"] in (2, 3, 4)
    assert st["tuned_lanes_per_row"] in (8, 32) and st["tuned_vslice"] in (2048, 8192)
    assert st["graph"] in (0, 1) and st["max_iters"] >= 1
    # the per-phase times cover the solve: they add up to at most its device time
    ph = st["phase_ms"]
    assert all(x >= 0.0 for x in ph) and ph[1] > 0.0 and ph[4] > 0.0
    assert 0.5 * st["solve_ms"] < sum(ph) <= st["solve_ms"] * 1.01 + 0.1
    P.shci_batch_destroy(b)
    ctx.close()


def test_batch_matches_sequential_solves(P):
    systems = small_batch(n_sys=8, cap=40000, seed=5100)
    ctx = P.Context(0, torch.cuda.current_stream())
    b = P.shci_batch_create(ctx.handle, systems)
    e, it, conv, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), 4, tol=1e-10)
    assert rc == 0
    # a second solve reuses the tuned schedule and the captured graph: same answer
    e2, _, _, _ = P.shci_batch_davidson(ctx.handle, b, len(systems), 4, tol=1e-10)
    np.testing.assert_allclose(e2, e, atol=1e-12, rtol=0)
    for s, d in enumerate(systems):
        B = G.Built(P, d["h"], d["eri"], d["e_core"], d["dets"], d["n_alpha"], d["n_beta"])
        es, _, _ = B.davidson(4, tol=1e-10)
        B.close()
        np.testing.assert_allclose(e[s], es, atol=E_TOL, rtol=0)
    P.shci_batch_destroy(b)
    ctx.close()


@pytest.mark.parametrize("before_tuning", [False, True])
def test_batch_barrier_timeout_is_reported_and_recoverable(P, before_tuning):
    """The grid barrier's wait is bounded: with the bound forced to zero the
    first block that has to wait gives up, every block leaves the kernel and
    the call returns SHCI_ERR_TIMEOUT (no hang, no fault).  The context stays
    usable and the default bound solves the same batch to the same energies;
    both while the autotuner times its trials and in the captured graph."""
    systems = small_batch(n_sys=4, cap=2000, seed=5200)
    ctx = P.Context(0, torch.cuda.current_stream())
    b = P.shci_batch_create(ctx.handle, systems)
    e0 = None
    if not before_tuning:
        e0, _, _, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), 2, tol=1e-10)
        assert rc == 0
    P.shci_batch_set_wait_limit(b, 0)
    with pytest.raises(P.ShciError) as exc:
        P.shci_batch_davidson(ctx.handle, b, len(systems), 2, tol=1e-10)
    assert exc.value.code == P.SHCI_ERR_TIMEOUT
    assert "timed out" in P.shci_last_error(ctx.handle)
    torch.cuda.synchronize()                                 # no sticky error
    P.shci_batch_set_wait_limit(b, -1)
    e1, _, conv, rc = P.shci_batch_davidson(ctx.handle, b, len(systems), 2, tol=1e-10)
    assert rc == 0 and conv.all()
    if e0 is not None:
        np.testing.assert_allclose(e1, e0, atol=1e-12, rtol=0)
    for s, d in enumerate(systems):
        B = G.Built(P, d["h"], d["eri"], d["e_core"], d["dets"], d["n_alpha"], d["n_beta"])
        es, _, _ = B.davidson(2, tol=1e-10)
        B.close()
        np.testing.assert_allclose(e1[s], es, atol=E_TOL, rtol=0)
    P.shci_batch_destroy(b)
    ctx.close()


def test_batch_rejects_bad_arguments(P):
    systems = small_batch(n_sys=2, cap=500)
    ctx = P.Context(0, torch.cuda.current_stream())
    b = P.shci_batch_create(ctx.handle, systems)
    with pytest.raises(P.ShciError):
        P.shci_batch_davidson(ctx.handle, b, 2, 5)          # more than four roots
    P.shci_batch_destroy(b)
    big = dict(systems[0])
    big["n_orb"] = 70
    with pytest.raises(P.ShciError):
        P.shci_batch_create(ctx.handle, [big])
    ctx.close()
