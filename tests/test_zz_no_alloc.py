"""shci_sigma_noalloc: the allocation-free sigma entry point.

It exists for callers that cannot let the library call cudaMalloc: a process
whose device memory is already owned by another allocator (a caching pool
that reserved nearly all of HBM, so a cudaMalloc would fail), or a
latency-critical loop that must not pay cudaMalloc's implicit
synchronisation.  Its output must match the regular shci_sigma within the
sigma tolerance the other tests use, and the oracle's rows, on two calls in a
row; neither call may take device memory (the scratch is loaded when the
context is created).

This file is collected last on purpose; it also passes when run on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import shci_synth as S
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

SIGMA_REL = 1e-12      # per-row bound relative to sum_j |H_ij c_j|, as in test_gpu_parity
SIGMA_ABS = 1e-10      # whole-vector bound, as in test_gpu_parity
MAX_ELEMS = 524288     # k * n_det limit of the static scratch


@pytest.fixture(scope="module")
def P():
    return G.lib()


def _noalloc_raw(P, handle, x, y):
    """Call the C entry point directly through ctypes (the C ABI)."""
    lib = P.load_library()
    k = x.shape[0]
    return lib.shci_sigma_noalloc(handle, ctypes.c_int(k), ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()))


def _check(got, ref, orc, rows, scale):
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= SIGMA_ABS
    assert np.all(np.abs(got[:, rows] - ref[:, rows]) <= SIGMA_REL * scale + 1e-300)
    assert np.all(np.abs(got[:, rows] - orc) <= SIGMA_REL * scale + 1e-300)


def _case(P, O, B, dets, k, seed):
    n = dets.shape[0]
    c = S.random_vectors(n, k, seed)
    ref = B.sigma(c)                                  # the regular entry point
    rows = np.unique(np.linspace(0, n - 1, 24).astype(np.int64))
    orc = O.sigma_rows(dets, c, rows)                 # the oracle, brute force over all columns
    scale = G.row_scale(O, dets, c, rows)
    return G.dev(c), ref, orc, rows, scale


@pytest.mark.parametrize("name,n_det,k", [("fci_10o_4a4b", None, 2), ("sel_24o_6a6b_1m", 20000, 8),
                                          ("sel_20o_5a5b_1m", 3001, 1),
                                          ("sel_20o_5a5b_1m", MAX_ELEMS // 8, 8)])
def test_noalloc_matches_sigma_and_oracle_twice(P, oracle_mod, name, n_det, k):
    cfg, h, eri, ec, dets = G.system(name, n_det)
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta)
    O = oracle_mod.System(h, eri, ec)
    x, ref, orc, rows, scale = _case(P, O, B, dets, k, 31)
    dev0 = torch.cuda.current_device()
    for call in range(2):
        y = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = _noalloc_raw(P, B.ctx.handle, x, y)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert rc == 0, P.shci_last_error(B.ctx.handle)
        assert free1 == free0, "call %d took device memory" % call
        assert torch.cuda.current_device() == dev0
        _check(y.cpu().numpy(), ref, orc, rows, scale)
    B.close()


def test_noalloc_two_contexts_in_turn(P, oracle_mod):
    """Two contexts share the one scratch array; calls that follow one another
    on the same stream each give their own context's product."""
    built = []
    for name, n_det, k, seed in (("sel_24o_6a6b_1m", 20000, 4, 5), ("sel_20o_5a5b_1m", 3001, 3, 6)):
        cfg, h, eri, ec, dets = G.system(name, n_det)
        B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta)
        O = oracle_mod.System(h, eri, ec)
        built.append((B, _case(P, O, B, dets, k, seed)))
    for B, (x, ref, orc, rows, scale) in built + built[:1]:
        y = torch.full_like(x, float("nan"))
        assert _noalloc_raw(P, B.ctx.handle, x, y) == 0, P.shci_last_error(B.ctx.handle)
        _check(y.cpu().numpy(), ref, orc, rows, scale)
    for B, _ in built:
        B.close()


def test_noalloc_rejects_oversize_and_unbuilt(P):
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m", 70000)
    ctx = P.Context(0, torch.cuda.current_stream())
    x = torch.zeros((8, dets.shape[0]), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    assert _noalloc_raw(P, ctx.handle, x, y) == 6          # nothing built yet
    P.shci_load_integrals(ctx.handle, cfg.n_orb, ec, G.dev(h), G.dev(eri))
    P.shci_build_connectivity(ctx.handle, cfg.n_alpha, cfg.n_beta, G.dev(dets))
    assert _noalloc_raw(P, ctx.handle, x, y) == 1          # 8 * 70000 > 524288
    assert "static scratch" in P.shci_last_error(ctx.handle)
    ctx.close()


def test_noalloc_rejects_an_upper_triangle_matrix(P):
    """Only a matrix stored in both triangles qualifies (SHCI_ERR_STATE, before any launch)."""
    cfg, h, eri, ec, dets = G.system("sel_20o_5a5b_1m", 3001)
    B = G.Built(P, h, eri, ec, dets, cfg.n_alpha, cfg.n_beta, mode=P.SHCI_STORED_UPPER)
    x = torch.zeros((1, dets.shape[0]), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    assert _noalloc_raw(P, B.ctx.handle, x, y) == 6
    B.close()
