"""Thin ctypes binding of the C ABI in include/shci.h.

Argument marshalling only: every step of the computation runs in the CUDA
library (``libshci.so``).  Functions keep the C names.  Arrays may be torch
tensors (on the context's device, or on the host) or numpy arrays (host); the
``mem_space`` argument of the C call is derived from where the data lives.
If the compiled library is missing, loading fails loudly -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libshci.so")

SHCI_OK = 0
SHCI_ERR_INVALID = 1
SHCI_ERR_OOM = 2
SHCI_ERR_CUDA = 3
SHCI_ERR_NOT_CONVERGED = 4
SHCI_ERR_TIMEOUT = 5
SHCI_ERR_STATE = 6
SHCI_MEM_HOST = 0
SHCI_MEM_DEVICE = 1
SHCI_STORED = 0
SHCI_ON_THE_FLY = 1
SHCI_AUTO = 2
SHCI_STORED_UPPER = 3

_STATUS = {1: "INVALID", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "TIMEOUT", 6: "STATE"}

# every symbol include/shci.h declares (checked by the tests)
EXPORTED = [
    "shci_create", "shci_destroy", "shci_last_error", "shci_load_integrals", "shci_build_connectivity",
    "shci_extend_connectivity", "shci_get_diag", "shci_get_pairs", "shci_get_row", "shci_sigma", "shci_sigma_noalloc", "shci_energy_backward",
    "shci_batch_create", "shci_batch_get_modes", "shci_batch_davidson", "shci_batch_get_stats",
    "shci_batch_set_wait_limit", "shci_batch_destroy",
    "shci_davidson",
    "shci_davidson_history", "shci_select", "shci_pt2", "shci_alias_draw", "shci_pt2_samples",
    "shci_pt2_semistochastic", "shci_pt2_3step", "shci_get_stats", "shci_set_timing",
]


class ShciError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("shci error %s (%d): %s" % (_STATUS.get(code, "?"), code, msg))
        self.code = code


class shci_stats_t(ctypes.Structure):
    _fields_ = [
        ("n_det", ctypes.c_int64), ("nnz_upper", ctypes.c_int64), ("n_alpha_strings", ctypes.c_int64),
        ("n_beta_strings", ctypes.c_int64), ("n_alpha_singles", ctypes.c_int64), ("candidates", ctypes.c_int64),
        ("build_ms", ctypes.c_double), ("sigma_ms_total", ctypes.c_double), ("sigma_launches", ctypes.c_int64),
        ("sigma_vectors", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("davidson_iters", ctypes.c_int),
        ("mode", ctypes.c_int), ("n_words", ctypes.c_int), ("davidson_phase_ms", ctypes.c_double * 8),
        ("select_ms", ctypes.c_double), ("select_candidates", ctypes.c_int64),
        ("pt2_ms", ctypes.c_double), ("pt2_batches", ctypes.c_int), ("pt2_terms", ctypes.c_int64),
        ("extend_ms", ctypes.c_double), ("extend_incremental", ctypes.c_int), ("extend_n_old", ctypes.c_int64),
        ("extend_phase_ms", ctypes.c_double * 4),
    ]


class shci_pt2_3step_t(ctypes.Structure):
    _fields_ = [
        ("e2", ctypes.c_double), ("e2_err", ctypes.c_double), ("dtm", ctypes.c_double), ("psto", ctypes.c_double),
        ("psto_err", ctypes.c_double), ("sto", ctypes.c_double), ("sto_err", ctypes.c_double),
        ("psto_batches", ctypes.c_int),
    ]


class shci_system_desc(ctypes.Structure):
    _fields_ = [
        ("n_orb", ctypes.c_int), ("n_alpha", ctypes.c_int), ("n_beta", ctypes.c_int), ("n_det", ctypes.c_int64),
        ("e_core", ctypes.c_double), ("h", ctypes.c_void_p), ("eri_packed", ctypes.c_void_p),
        ("dets", ctypes.c_void_p),
    ]


class shci_batch_stats_t(ctypes.Structure):
    _fields_ = [
        ("n_sys", ctypes.c_int), ("n_stored", ctypes.c_int), ("n_on_the_fly", ctypes.c_int),
        ("total_det", ctypes.c_int64), ("total_nnz_upper", ctypes.c_int64),
        ("tuned_rows_per_item", ctypes.c_int), ("tuned_ctas_per_sm", ctypes.c_int),
        ("tuned_lanes_per_row", ctypes.c_int),
        ("tune_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("max_iters", ctypes.c_int),
        ("graph", ctypes.c_int), ("grid_ctas", ctypes.c_int), ("phase_ms", ctypes.c_double * 16),
        ("n_stored_upper", ctypes.c_int), ("tuned_vslice", ctypes.c_int),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libshci.so (build it first with build_lib.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("the CUDA library %s is not built; run paper_1809_04600_gb300.build_lib.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "shci_create": (i32, [ctypes.POINTER(vp), i32, vp]),
        "shci_destroy": (None, [vp]),
        "shci_last_error": (ctypes.c_char_p, [vp]),
        "shci_load_integrals": (i32, [vp, i32, f64, vp, vp, i32]),
        "shci_build_connectivity": (i32, [vp, i32, i32, i64, vp, i32, i32, ctypes.POINTER(i64)]),
        "shci_extend_connectivity": (i32, [vp, i64, vp, i32, f64, ctypes.POINTER(i64)]),
        "shci_get_diag": (i32, [vp, vp, i32]),
        "shci_get_pairs": (i32, [vp, i64, vp, vp, vp, ctypes.POINTER(i64)]),
        "shci_get_row": (i32, [vp, i64, i64, vp, vp, ctypes.POINTER(i64)]),
        "shci_sigma": (i32, [vp, i32, vp, vp, i32]),
        "shci_sigma_noalloc": (i32, [vp, i32, vp, vp]),
        "shci_energy_backward": (i32, [vp, vp, f64, vp, vp, i32]),
        "shci_batch_create": (i32, [vp, i32, ctypes.POINTER(shci_system_desc), i32, f64, ctypes.POINTER(vp)]),
        "shci_batch_get_modes": (i32, [vp, i32, vp]),
        "shci_batch_davidson": (i32, [vp, i32, f64, i32, vp, vp, vp]),
        "shci_batch_get_stats": (i32, [vp, ctypes.POINTER(shci_batch_stats_t)]),
        "shci_batch_set_wait_limit": (i32, [vp, ctypes.c_longlong]),
        "shci_batch_destroy": (None, [vp]),
        "shci_davidson": (i32, [vp, i32, f64, i32, vp, vp, vp, i32, ctypes.POINTER(i32)]),
        "shci_davidson_history": (i32, [vp, i32, vp, vp, vp, ctypes.POINTER(i32)]),
        "shci_select": (i32, [vp, i32, vp, f64, i64, vp, ctypes.POINTER(i64), i32]),
        "shci_pt2": (i32, [vp, vp, f64, f64, i32, ctypes.POINTER(f64), ctypes.POINTER(i64), i32]),
        "shci_alias_draw": (i32, [vp, vp, i64, ctypes.c_uint64, vp, i32]),
        "shci_pt2_samples": (i32, [vp, vp, f64, f64, f64, i64, i32, vp, vp, i32, i32, vp]),
        "shci_pt2_3step": (i32, [vp, vp, f64, f64, f64, f64, f64, i32, i32, i64, i32, ctypes.c_uint64,
                                 ctypes.POINTER(shci_pt2_3step_t), i32]),
        "shci_pt2_semistochastic": (i32, [vp, vp, f64, f64, f64, i64, i32, ctypes.c_uint64, ctypes.POINTER(f64),
                                          ctypes.POINTER(f64), i32]),
        "shci_get_stats": (i32, [vp, ctypes.POINTER(shci_stats_t)]),
        "shci_set_timing": (i32, [vp, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ------------------------------------------------------------------ marshalling

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, mem_space, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, SHCI_MEM_HOST, None
    if _is_torch(x):
        import torch
        want = {np.float64: (torch.float64,), np.uint64: (torch.uint64, torch.int64),
                np.int64: (torch.int64,)}[dtype]
        if x.dtype not in want:
            raise TypeError("expected %s, got %s" % (want[0], x.dtype))
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (SHCI_MEM_DEVICE if x.is_cuda else SHCI_MEM_HOST), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, SHCI_MEM_HOST, a


def _check(ctx, rc):
    if rc != SHCI_OK:
        raise ShciError(rc, load_library().shci_last_error(ctx).decode())


# ------------------------------------------------------------------ C-named calls

def shci_create(device: int = 0, stream=None):
    """Returns an opaque context handle.  ``stream`` is a torch.cuda.Stream,
    a raw cudaStream_t integer, or None (the context owns a stream)."""
    lib = load_library()
    h = ctypes.c_void_p()
    raw = None
    if stream is not None:
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib.shci_create(ctypes.byref(h), int(device), raw)
    if rc != SHCI_OK:
        raise ShciError(rc, lib.shci_last_error(None).decode())
    return h


def shci_destroy(ctx):
    load_library().shci_destroy(ctx)


def shci_last_error(ctx) -> str:
    return load_library().shci_last_error(ctx).decode()


def shci_load_integrals(ctx, n_orb, e_core, h, eri_packed):
    ph, mh, kh = _ptr(h, np.float64)
    pe, me, ke = _ptr(eri_packed, np.float64)
    if mh != me:
        raise ValueError("h and eri_packed must live in the same memory space")
    _check(ctx, load_library().shci_load_integrals(ctx, int(n_orb), float(e_core), ph, pe, mh))


def shci_build_connectivity(ctx, n_alpha, n_beta, dets, mode=SHCI_STORED) -> int:
    pd, md, kd = _ptr(dets, np.uint64)
    n_det = dets.shape[0]
    nnz = ctypes.c_int64(0)
    _check(ctx, load_library().shci_build_connectivity(ctx, int(n_alpha), int(n_beta), int(n_det), pd, md,
                                                       int(mode), ctypes.byref(nnz)))
    return nnz.value


def shci_extend_connectivity(ctx, new_dets, full_fraction=0.2) -> int:
    """Append new_dets [n_new][2W] to V and update the connectivity (incremental
    below full_fraction of the grown V, else rebuilt); returns nnz_upper."""
    pd, md, kd = _ptr(new_dets, np.uint64)
    nnz = ctypes.c_int64(0)
    _check(ctx, load_library().shci_extend_connectivity(ctx, int(new_dets.shape[0]), pd, md, float(full_fraction),
                                                        ctypes.byref(nnz)))
    return nnz.value


def shci_get_diag(ctx, out):
    p, m, k = _ptr(out, np.float64)
    _check(ctx, load_library().shci_get_diag(ctx, p, m))
    return out


def shci_get_pairs(ctx):
    """(i, j, H_ij) numpy arrays of the stored upper triangle, rows ascending."""
    lib = load_library()
    n = ctypes.c_int64(0)
    _check(ctx, lib.shci_get_pairs(ctx, 0, None, None, None, ctypes.byref(n)))
    ii = np.empty(n.value, np.int64)
    jj = np.empty(n.value, np.int64)
    vv = np.empty(n.value, np.float64)
    _check(ctx, lib.shci_get_pairs(ctx, n.value, ii.ctypes.data, jj.ctypes.data, vv.ctypes.data, ctypes.byref(n)))
    return ii, jj, vv


def shci_get_row(ctx, row):
    """(cols, vals) of one stored row without the diagonal, ascending columns."""
    lib = load_library()
    n = ctypes.c_int64(0)
    _check(ctx, lib.shci_get_row(ctx, int(row), 0, None, None, ctypes.byref(n)))
    cols = np.empty(n.value, np.int64)
    vals = np.empty(n.value, np.float64)
    _check(ctx, lib.shci_get_row(ctx, int(row), n.value, cols.ctypes.data, vals.ctypes.data, ctypes.byref(n)))
    return cols, vals


def shci_sigma(ctx, c, sigma):
    """sigma[k, n] = H c[k, n] (both torch CUDA tensors, or both host arrays)."""
    pc, mc, kc = _ptr(c, np.float64)
    ps, ms, ks = _ptr(sigma, np.float64)
    if mc != ms:
        raise ValueError("c and sigma must live in the same memory space")
    k = 1 if len(c.shape) == 1 else c.shape[0]
    _check(ctx, load_library().shci_sigma(ctx, int(k), pc, ps, mc))
    return sigma


def shci_sigma_noalloc(ctx, c, sigma):
    """sigma[k, n] = H c[k, n] for torch CUDA tensors, with no device allocation
    (static scratch; k * n_det <= 524,288)."""
    pc, mc, kc = _ptr(c, np.float64)
    ps, ms, ks = _ptr(sigma, np.float64)
    if mc != SHCI_MEM_DEVICE or ms != SHCI_MEM_DEVICE:
        raise ValueError("shci_sigma_noalloc takes device tensors only")
    k = 1 if len(c.shape) == 1 else c.shape[0]
    _check(ctx, load_library().shci_sigma_noalloc(ctx, int(k), pc, ps))
    return sigma


def shci_davidson(ctx, k_roots, tol=1e-10, max_iter=200, guess=None, vecs=None, check=True):
    """(energies[k], iterations, status).  vecs (torch CUDA tensor or numpy) receives Ritz vectors."""
    lib = load_library()
    e = np.empty(k_roots, np.float64)
    pg, mg, kg = _ptr(guess, np.float64)
    pv, mv, kv = _ptr(vecs, np.float64)
    if guess is not None and vecs is not None and mg != mv:
        raise ValueError("guess and vecs must live in the same memory space")
    mem = mv if vecs is not None else mg
    it = ctypes.c_int(0)
    rc = lib.shci_davidson(ctx, int(k_roots), float(tol), int(max_iter), pg, e.ctypes.data, pv, mem,
                           ctypes.byref(it))
    if check and rc not in (SHCI_OK,):
        _check(ctx, rc)
    return e, it.value, rc


def shci_davidson_history(ctx, k_roots):
    """Last Davidson run: (theta [iters, k], rnorm [iters, k], t_s [iters])."""
    lib = load_library()
    n = ctypes.c_int(0)
    _check(ctx, lib.shci_davidson_history(ctx, 0, None, None, None, ctypes.byref(n)))
    th = np.empty((n.value, k_roots), np.float64)
    rn = np.empty((n.value, k_roots), np.float64)
    ts = np.empty(n.value, np.float64)
    _check(ctx, lib.shci_davidson_history(ctx, n.value, th.ctypes.data, rn.ctypes.data, ts.ctypes.data,
                                          ctypes.byref(n)))
    return th, rn, ts


def shci_select(ctx, c, eps1, cap=None):
    """Heat-bath selection: the new determinants [count, 2W] (uint64 numpy for a
    host c, int64 torch tensor on c's device for a device c), ascending, no
    repeats.  c: [k, n_det] (or [n_det]) coefficients of V."""
    lib = load_library()
    pc, mc, kc = _ptr(c, np.float64)
    k = 1 if len(c.shape) == 1 else int(c.shape[0])
    n_det = int(c.shape[-1])
    W = shci_get_stats(ctx)["n_words"]
    cap = max(1024, 2 * n_det) if cap is None else int(cap)
    n = ctypes.c_int64(0)
    while True:
        if mc == SHCI_MEM_DEVICE:
            import torch
            out = torch.empty((max(cap, 1), 2 * W), dtype=torch.int64, device=c.device)
        else:
            out = np.empty((max(cap, 1), 2 * W), np.uint64)
        po, mo, ko = _ptr(out, np.uint64)
        _check(ctx, lib.shci_select(ctx, k, pc, float(eps1), cap, po, ctypes.byref(n), mc))
        if n.value <= cap:
            return out[:n.value]
        cap = int(n.value)


def shci_pt2(ctx, c, e_var, eps2, n_batches=0):
    """(dE2, n_pert): the eps2-screened second-order Epstein-Nesbet energy of
    the root c [n_det] (host or device) with variational energy e_var."""
    pc, mc, kc = _ptr(c, np.float64)
    e2 = ctypes.c_double(0.0)
    npert = ctypes.c_int64(0)
    _check(ctx, load_library().shci_pt2(ctx, pc, float(e_var), float(eps2), int(n_batches), ctypes.byref(e2),
                                        ctypes.byref(npert), mc))
    return e2.value, npert.value


def shci_alias_draw(ctx, c, n_draws, seed):
    """n_draws indices of V drawn with p_i = |c_i| / sum |c| (alias method), in c's memory space."""
    pc, mc, kc = _ptr(c, np.float64)
    if mc == SHCI_MEM_DEVICE:
        import torch
        out = torch.empty(int(n_draws), dtype=torch.int64, device=c.device)
    else:
        out = np.empty(int(n_draws), np.int64)
    po, mo, ko = _ptr(out, np.int64)
    _check(ctx, load_library().shci_alias_draw(ctx, pc, int(n_draws), int(seed) & ((1 << 64) - 1), po, mc))
    return out


def shci_pt2_samples(ctx, c, e_var, eps2, eps2_d, draws, n_batches=1, batches=None):
    """[n_samples, 2]: the stochastic second-order energy of each sample (rows
    of draws, [n_samples, n_d]) at eps2 and at eps2_d; with n_batches > 1 only
    the hash batch batches[s] of each sample."""
    pc, mc, kc = _ptr(c, np.float64)
    pd, md, kd = _ptr(draws, np.int64)
    if mc != md:
        raise ValueError("c and draws must live in the same memory space")
    n_samples, n_d = int(draws.shape[0]), int(draws.shape[1])
    out = np.empty((n_samples, 2))
    bt = None if batches is None else np.ascontiguousarray(batches, np.int32)
    _check(ctx, load_library().shci_pt2_samples(ctx, pc, float(e_var), float(eps2), float(eps2_d), n_d, n_samples,
                                                pd, out.ctypes.data, mc, int(n_batches),
                                                None if bt is None else bt.ctypes.data))
    return out


def shci_pt2_3step(ctx, c, e_var, eps2, eps2_psto, eps2_dtm, target_error, n_batches_psto, n_batches_sto, n_d,
                   n_samples, seed):
    """The 3-step perturbation scheme: dict of the total, its error and the parts."""
    pc, mc, kc = _ptr(c, np.float64)
    o = shci_pt2_3step_t()
    _check(ctx, load_library().shci_pt2_3step(ctx, pc, float(e_var), float(eps2), float(eps2_psto), float(eps2_dtm),
                                              float(target_error), int(n_batches_psto), int(n_batches_sto), int(n_d),
                                              int(n_samples), int(seed) & ((1 << 64) - 1), ctypes.byref(o), mc))
    return {name: getattr(o, name) for name, _ in shci_pt2_3step_t._fields_}


def shci_pt2_semistochastic(ctx, c, e_var, eps2, eps2_d, n_d, n_samples, seed):
    """(dE2, standard error): deterministic at eps2_d plus the sampled difference between eps2 and eps2_d."""
    pc, mc, kc = _ptr(c, np.float64)
    e2 = ctypes.c_double(0.0)
    err = ctypes.c_double(0.0)
    _check(ctx, load_library().shci_pt2_semistochastic(ctx, pc, float(e_var), float(eps2), float(eps2_d), int(n_d),
                                                       int(n_samples), int(seed) & ((1 << 64) - 1),
                                                       ctypes.byref(e2), ctypes.byref(err), mc))
    return e2.value, err.value


def shci_energy_backward(ctx, c, grad_out_scale, dE_dh, dE_deri_packed):
    """dE/dh and packed dE/d(pq|rs) for the normalised root c (Hellmann-Feynman)."""
    pc, mc, kc = _ptr(c, np.float64)
    ph, mh, kh = _ptr(dE_dh, np.float64)
    pe, me, ke = _ptr(dE_deri_packed, np.float64)
    if not (mc == mh == me):
        raise ValueError("c and the gradient buffers must live in the same memory space")
    _check(ctx, load_library().shci_energy_backward(ctx, pc, float(grad_out_scale), ph, pe, mc))
    return dE_dh, dE_deri_packed


def shci_batch_create(ctx, systems, stored_budget_bytes=-1.0):
    """systems: list of dicts with n_orb, n_alpha, n_beta, h, eri, dets (and optional e_core);
    arrays all numpy (host) or all torch CUDA tensors.  Returns the batch handle."""
    lib = load_library()
    arr = (shci_system_desc * len(systems))()
    keep = []
    mem = None
    for s, d in enumerate(systems):
        ph, m1, k1 = _ptr(d["h"], np.float64)
        pe, m2, k2 = _ptr(d["eri"], np.float64)
        pd, m3, k3 = _ptr(d["dets"], np.uint64)
        keep += [k1, k2, k3]
        if not (m1 == m2 == m3) or (mem is not None and m1 != mem):
            raise ValueError("all batch arrays must live in the same memory space")
        mem = m1
        arr[s] = shci_system_desc(int(d["n_orb"]), int(d["n_alpha"]), int(d["n_beta"]), int(d["dets"].shape[0]),
                                  float(d.get("e_core", 0.0)), ph, pe, pd)
    out = ctypes.c_void_p()
    _check(ctx, lib.shci_batch_create(ctx, len(systems), arr, mem, float(stored_budget_bytes), ctypes.byref(out)))
    return out


def shci_batch_davidson(ctx, batch, n_sys, k_roots, tol=1e-10, max_iter=400):
    """(energies [n_sys, k], iters [n_sys], converged [n_sys], status)."""
    lib = load_library()
    e = np.empty((n_sys, k_roots), np.float64)
    it = np.empty(n_sys, np.int32)
    cv = np.empty(n_sys, np.int32)
    rc = lib.shci_batch_davidson(batch, int(k_roots), float(tol), int(max_iter), e.ctypes.data, it.ctypes.data,
                                 cv.ctypes.data)
    if rc not in (SHCI_OK, SHCI_ERR_NOT_CONVERGED):
        _check(ctx, rc)
    return e, it, cv, rc


def shci_batch_get_stats(batch) -> dict:
    s = shci_batch_stats_t()
    rc = load_library().shci_batch_get_stats(batch, ctypes.byref(s))
    if rc != SHCI_OK:
        raise ShciError(rc, "shci_batch_get_stats failed")
    out = {name: getattr(s, name) for name, _ in shci_batch_stats_t._fields_}
    out["phase_ms"] = list(s.phase_ms)
    return out


def shci_batch_get_modes(batch, n_sys):
    """The storage mode each system of the batch was given (SHCI_STORED,
    SHCI_STORED_UPPER or SHCI_ON_THE_FLY), as an int array [n_sys]."""
    modes = np.zeros(n_sys, np.int32)
    rc = load_library().shci_batch_get_modes(batch, int(n_sys), modes.ctypes.data)
    if rc != SHCI_OK:
        raise ShciError(rc, "shci_batch_get_modes failed")
    return modes


def shci_batch_set_wait_limit(batch, naps):
    """Bound of the batch solver's grid-barrier wait, in ~100 ns naps (< 0: the default)."""
    rc = load_library().shci_batch_set_wait_limit(batch, int(naps))
    if rc != SHCI_OK:
        raise ShciError(rc, "shci_batch_set_wait_limit failed")


def shci_batch_destroy(batch):
    load_library().shci_batch_destroy(batch)


def shci_get_stats(ctx) -> dict:
    s = shci_stats_t()
    _check(ctx, load_library().shci_get_stats(ctx, ctypes.byref(s)))
    out = {name: getattr(s, name) for name, _ in shci_stats_t._fields_}
    out["davidson_phase_ms"] = list(s.davidson_phase_ms)
    out["extend_phase_ms"] = list(s.extend_phase_ms)
    return out


def shci_set_timing(ctx, enable, davidson_phases=False):
    """Bit 0: time every sigma launch; bit 1 (davidson_phases): time the parts of shci_davidson."""
    _check(ctx, load_library().shci_set_timing(ctx, (1 if enable else 0) | (2 if davidson_phases else 0)))


class Context:
    """Owning wrapper: ``with Context(device, stream) as ctx: ...``."""

    def __init__(self, device=0, stream=None):
        self.handle = shci_create(device, stream)

    def close(self):
        if self.handle is not None:
            shci_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
