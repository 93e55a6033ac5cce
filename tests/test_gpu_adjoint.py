"""The hand-written adjoint (dE/dh, dE/d(pq|rs)) against the oracle's density
matrices, identities that hold at any size, central finite differences, and
the torch.autograd wrapper.  Bar: gradients within 1e-7 relative."""
import numpy as np
import pytest
import torch

import shci_synth as S
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

GRAD_REL = 1e-7


@pytest.fixture(scope="module")
def P():
    return G.lib()


def gpu_gradient(P, B, c):
    n = B.h.shape[0]
    dh = torch.empty((n, n), dtype=torch.float64, device="cuda")
    de = torch.empty(B.eri.size, dtype=torch.float64, device="cuda")
    P.shci_energy_backward(B.ctx.handle, G.dev(c), 1.0, dh, de)
    return dh.cpu().numpy(), de.cpu().numpy()


def test_gradient_matches_oracle_rdms_small_fci(P, oracle_mod):
    n, na, nb = 6, 2, 2
    h, eri, _ = S.integrals(n, 6, 77)
    dets = S.fci_dets(n, na, nb)
    B = G.Built(P, h, eri, 0.0, dets, na, nb)
    e, vecs, _ = B.davidson(1, tol=1e-12)
    c = vecs[0]
    gh, ge = gpu_gradient(P, B, c)
    O = oracle_mod.System(h, eri, 0.0)
    oh, oe = O.energy_gradient(dets, c)
    np.testing.assert_allclose(gh, oh, atol=1e-12)
    np.testing.assert_allclose(ge, oe, atol=1e-12)
    B.close()


@pytest.mark.parametrize("name,n_det", [("sel_20o_5a5b_1m", 3000), ("sel_76o_14a14b_50m", 2000)])
def test_gradient_matches_oracle_on_selected_space(P, oracle_mod, name, n_det):
    cfg, h, eri, ec, dets = G.system(name, n_det)
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta)
    e, vecs, _ = B.davidson(1, tol=1e-12)
    c = vecs[0]
    gh, ge = gpu_gradient(P, B, c)
    n = cfg.n_orb
    # the full one-body density matrix
    g1 = oracle_mod.rdm1_full(dets, c, n)
    np.testing.assert_allclose(gh, g1, atol=1e-12)
    # sampled packed two-body slots (largest and random)
    rng = np.random.default_rng(4)
    slots = np.unique(np.concatenate([np.argsort(-np.abs(ge))[:20], rng.choice(ge.size, 40, replace=False)]))
    members = oracle_mod.slot_members(n) if n <= 20 else None
    if members is None:
        # 76 orbitals: enumerate members only for the sampled slots
        members = _members_for(slots, n)
    ref = oracle_mod.packed_gradient_entries(dets, c, n, slots, members)
    np.testing.assert_allclose(ge[slots], ref, atol=1e-12)
    B.close()


def _members_for(slots, n):
    want = set(int(s) for s in slots)
    pair = lambda p, q: max(p, q) * (max(p, q) + 1) // 2 + min(p, q)
    members = {s: [] for s in want}
    # invert slot -> (PQ, RS) -> (p, q), (r, s)
    inv = {}
    for p in range(n):
        for q in range(n):
            inv.setdefault(pair(p, q), []).append((p, q))
    for s in want:
        hi = int((np.sqrt(8 * s + 1) - 1) // 2)
        while hi * (hi + 1) // 2 > s:
            hi -= 1
        while (hi + 1) * (hi + 2) // 2 <= s:
            hi += 1
        lo = s - hi * (hi + 1) // 2
        for PQ, RS in ((hi, lo), (lo, hi)) if hi != lo else ((hi, lo),):
            for (p, q) in inv[PQ]:
                for (r, t) in inv[RS]:
                    members[s].append((p, q, r, t))
    return members


def test_gradient_identities_full_size(P):
    """|V| = 1e6, 20 orbitals, 5a5b: trace of gamma = N, and E = E_core + sum h*gamma
    + sum eri*dE/deri (E is linear in the integrals for a fixed vector)."""
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m")
    B = G.Built(P, h, eri, ec, dets, 5, 5)
    e, vecs, _ = B.davidson(1, tol=1e-11)
    gh, ge = gpu_gradient(P, B, vecs[0])
    assert abs(np.trace(gh) - 10.0) < 1e-9
    np.testing.assert_allclose(gh, gh.T, atol=1e-11)
    e_lin = ec + np.sum(h * gh) + np.dot(eri, ge)
    assert abs(e_lin - e[0]) < 1e-8 * max(1.0, abs(e[0]))
    B.close()


def _energy(P, h, eri, ec, dets, na, nb, tol=1e-13):
    B = G.Built(P, h, eri, ec, dets, na, nb)
    e, vecs, it = B.davidson(1, tol=tol, max_iter=600)
    B.close()
    return e[0], vecs[0]


@pytest.mark.parametrize("n_det", [20000])
def test_gradient_matches_central_differences(P, n_det):
    """Central differences of the energy along 16 seeded directions of all the
    integrals.  The step-1e-5 difference carries a truncation error (h^2 / 6
    times the third derivative) that reaches several 1e-7 on the heat-bath
    space, while below 1e-5 the energies' rounding (~1e-13) takes over, so the
    reference is the Richardson combination (4 D(h) - D(2h)) / 3 of the central
    differences at h = 1e-5 and 2e-5 (error O(h^4)).  The analytic gradient is
    first-order in the eigenvector's error, so its vector is solved to tol
    1e-14 (residual below 1e-8)."""
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m", n_det)
    e0, c = _energy(P, h, eri, ec, dets, 5, 5, tol=1e-14)
    B = G.Built(P, h, eri, ec, dets, 5, 5)
    gh, ge = gpu_gradient(P, B, c)
    B.close()
    rng = np.random.default_rng(4004)
    for _ in range(16):
        dh = rng.normal(size=h.shape)
        dh = 0.5 * (dh + dh.T)
        de = rng.normal(size=eri.size)
        fd = {}
        for step in (1e-5, 2e-5):
            ep, _ = _energy(P, h + step * dh, eri + step * de, ec, dets, 5, 5)
            em, _ = _energy(P, h - step * dh, eri - step * de, ec, dets, 5, 5)
            fd[step] = (ep - em) / (2 * step)
        rich = (4.0 * fd[1e-5] - fd[2e-5]) / 3.0
        an = np.sum(gh * dh) + np.dot(ge, de)
        assert abs(rich - an) <= GRAD_REL * max(1.0, abs(an)), (rich, fd, an)


def test_autograd_function(P):
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m", 5000)
    ht = torch.tensor(h, device="cuda", requires_grad=True)
    et = torch.tensor(eri, device="cuda", requires_grad=True)
    d = G.dev(dets)
    E = P.Energy.apply(ht, et, d, 5, 5)
    E.backward()
    e0, c = _energy(P, h, eri, ec, dets, 5, 5, tol=1e-12)
    assert abs(E.item() - e0) < 1e-9
    B = G.Built(P, h, eri, ec, dets, 5, 5)
    gh, ge = gpu_gradient(P, B, c)
    B.close()
    np.testing.assert_allclose(ht.grad.cpu().numpy(), gh, atol=1e-9)
    np.testing.assert_allclose(et.grad.cpu().numpy(), ge, atol=1e-9)
    # scaling by the incoming gradient
    ht.grad = None
    et.grad = None
    E2 = P.Energy.apply(ht, et, d, 5, 5)
    (3.0 * E2).backward()
    np.testing.assert_allclose(ht.grad.cpu().numpy(), 3.0 * gh, atol=3e-9)
