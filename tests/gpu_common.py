"""Shared set-up for the GPU parity tests: build + load the CUDA library and
run the boundary calls on seeded inputs."""
import numpy as np
import torch

import shci_synth as S


def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_04600_gb300 as P
    P.build()
    P.load_library()
    return P


def dev(a, dtype=None):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to("cuda")


class Built:
    """A context with integrals loaded and connectivity built."""

    def __init__(self, P, h, eri, e_core, dets, n_alpha, n_beta, mode=None, host=False):
        self.P = P
        self.ctx = P.Context(0, torch.cuda.current_stream())
        self.h, self.eri, self.e_core, self.dets = h, eri, e_core, dets
        self.n_alpha, self.n_beta = n_alpha, n_beta
        self.n = dets.shape[0]
        if host:
            P.shci_load_integrals(self.ctx.handle, h.shape[0], e_core, h, eri)
            self.nnz = P.shci_build_connectivity(self.ctx.handle, n_alpha, n_beta, dets,
                                                 P.SHCI_STORED if mode is None else mode)
        else:
            P.shci_load_integrals(self.ctx.handle, h.shape[0], e_core, dev(h), dev(eri))
            self.nnz = P.shci_build_connectivity(self.ctx.handle, n_alpha, n_beta, dev(dets),
                                                 P.SHCI_STORED if mode is None else mode)

    def diag(self):
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        self.P.shci_get_diag(self.ctx.handle, out)
        return out.cpu().numpy()

    def sigma(self, c):
        c = np.atleast_2d(c)
        x = dev(c)
        y = torch.empty_like(x)
        self.P.shci_sigma(self.ctx.handle, x, y)
        return y.cpu().numpy()

    def pairs(self):
        return self.P.shci_get_pairs(self.ctx.handle)

    def row(self, i):
        return self.P.shci_get_row(self.ctx.handle, i)

    def davidson(self, k, tol=1e-10, max_iter=300, guess=None):
        vecs = torch.empty((k, self.n), dtype=torch.float64, device="cuda")
        g = None if guess is None else dev(guess)
        e, it, rc = self.P.shci_davidson(self.ctx.handle, k, tol, max_iter, guess=g, vecs=vecs)
        return e, vecs.cpu().numpy(), it

    def stats(self):
        return self.P.shci_get_stats(self.ctx.handle)

    def close(self):
        self.ctx.close()


def system(name, n_det=None):
    cfg = S.config(name)
    h, eri, ec, dets = S.make_system(cfg, n_det=n_det)
    return cfg, h, eri, ec, dets


def row_scale(O, dets, c, rows):
    """sum_j |H_ij c_j| for the given rows (oracle rows, for relative tolerances)."""
    out = np.zeros((c.shape[0], len(rows)))
    d = O.hdiag(dets[rows]) if len(rows) else np.zeros(0)
    for t, i in enumerate(rows):
        cols, vals = O.row(dets, int(i))
        out[:, t] = np.abs(c[:, cols]) @ np.abs(vals) + np.abs(d[t] * c[:, i])
    return out
