"""The seeded input recipe (no GPU): the properties the tests and the bench
rely on.  A selected space is in generation order, so a smaller space of the
same shape is its prefix: the incremental-update workload appends the tail of
a space to its head exactly as a later variational iteration would."""
import math

import numpy as np
import pytest

import shci_synth as S


def _popcounts(words):
    return np.array([sum(bin(int(w)).count("1") for w in row) for row in words])


@pytest.mark.parametrize("name,small,large", [("sel_24o_6a6b_1m", 2000, 5000), ("sel_76o_14a14b_50m", 1000, 3000),
                                              ("sel_20o_5a5b_1m", 700, 2100)])
def test_selected_space_is_in_generation_order(name, small, large):
    cfg = S.config(name)
    h, eri, ec, a = S.make_system(cfg, n_det=small)
    _, _, _, b = S.make_system(cfg, n_det=large)
    assert np.array_equal(a, b[:small])                       # prefix property
    W = S.n_words(cfg.n_orb)
    assert b.shape == (large, 2 * W) and b.dtype == np.uint64
    assert np.array_equal(b[0], S.hf_dets(cfg.n_orb, cfg.n_alpha, cfg.n_beta)[0])   # reference first
    assert np.unique(b, axis=0).shape[0] == large             # distinct
    assert np.all(_popcounts(b[:, :W]) == cfg.n_alpha) and np.all(_popcounts(b[:, W:]) == cfg.n_beta)
    for w in range(W):                                        # no orbital >= n_orb
        top = cfg.n_orb - 64 * w
        if top < 64:
            mask = ~np.uint64((1 << max(top, 0)) - 1)
            assert not np.any(b[:, w] & mask) and not np.any(b[:, W + w] & mask)


def test_full_ci_space_and_integral_layout():
    cfg = S.config("fci_10o_4a4b")
    h, eri, ec, d = S.make_system(cfg)
    assert d.shape[0] == math.comb(10, 4) ** 2
    assert np.unique(d, axis=0).shape[0] == d.shape[0]
    assert np.array_equal(h, h.T)
    assert eri.shape == (S.eri_len(10),)
    assert S.eri_len(10) == S.n_pair(10) * (S.n_pair(10) + 1) // 2


@pytest.mark.parametrize("name", ["sel_24o_6a6b_1m", "sel_20o_5a5b_1m"])
def test_stored_heat_bath_space(name, oracle_mod):
    """A stored heat-bath space: its SHA-256 matches the record, it is laid out
    as the library expects, its blocks add up, and its first two blocks are
    exactly what the oracle's selection (Sec. II.A, Eq. 2) gives from the aufbau
    determinant at eps1 = 1e-2 and, after the dense ground state(s) of that
    space, at 1e-2 x 0.7."""
    import os
    if not os.path.exists(os.path.join(S.SPACES_DIR, name + ".npz")):
        pytest.skip("space %s not stored" % name)
    cfg = S.config(name)
    meta = S.selected_space_meta(name)
    V = S.load_selected_space(name)                       # checks the SHA-256
    assert V.shape == (meta["n_det"], 2) and V.dtype == np.uint64
    blocks = meta["selection"]["blocks"]
    assert sum(blocks) == V.shape[0] and blocks[0] == 1
    assert np.array_equal(V[0], S.hf_dets(cfg.n_orb, cfg.n_alpha, cfg.n_beta)[0])
    assert np.unique(V, axis=0).shape[0] == V.shape[0]
    assert np.all(_popcounts(V[:, :1]) == cfg.n_alpha) and np.all(_popcounts(V[:, 1:]) == cfg.n_beta)
    h, eri, ec = S.integrals(cfg.n_orb, cfg.rank, cfg.seed, cfg.band, cfg.n_alpha)
    O = oracle_mod.System(h, eri, ec)
    eps1 = meta["selection"]["eps1_start"]
    b1 = O.select(V[:1], np.ones((1, 1)), eps1)
    assert np.array_equal(b1, V[1:1 + blocks[1]])
    n2 = 1 + blocks[1]
    k = min(meta["selection"]["roots"], n2)
    _, c = O.lowest_eigenpairs(V[:n2], k)
    b2 = O.select(V[:n2], c, eps1 * meta["selection"]["eps1_factor"])
    assert np.array_equal(b2, V[n2:n2 + blocks[2]])
