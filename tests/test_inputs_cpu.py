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
