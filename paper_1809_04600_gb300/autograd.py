"""torch.autograd.Function around the variational energy and its adjoint.

    E = Energy.apply(h, eri_packed, dets, n_alpha, n_beta)
    E.backward()          # h.grad = dE/dh, eri_packed.grad = dE/d(packed slots)

Forward: shci_load_integrals + shci_build_connectivity + shci_davidson (the
lowest `root + 1` roots, tight tolerance) and returns E_root.  Backward: the
hand-written adjoint kernel shci_energy_backward (1- and 2-body density
matrices contracted on the fly from the root vector), scaled by the incoming
gradient.  The determinant set is held fixed.  PyTorch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import binding as B


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, eri_packed, dets, n_alpha, n_beta, root=0, e_core=0.0, tol=1e-12, max_iter=400,
                mode=B.SHCI_STORED):
        if not (h.is_cuda and eri_packed.is_cuda and dets.is_cuda):
            raise ValueError("Energy expects CUDA tensors")
        lib_ctx = B.Context(h.device.index or 0, torch.cuda.current_stream(h.device))
        H = lib_ctx.handle
        B.shci_load_integrals(H, h.shape[0], e_core, h.detach().contiguous(), eri_packed.detach().contiguous())
        B.shci_build_connectivity(H, n_alpha, n_beta, dets.contiguous(), mode)
        k = root + 1
        vecs = torch.empty((k, dets.shape[0]), dtype=torch.float64, device=h.device)
        e, it, rc = B.shci_davidson(H, k, tol, max_iter, vecs=vecs)
        ctx.lib_ctx = lib_ctx
        ctx.shapes = (h.shape, eri_packed.shape)
        ctx.save_for_backward(vecs[root].contiguous())
        return torch.tensor(float(e[root]), dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, grad_e):
        (c,) = ctx.saved_tensors
        hs, es = ctx.shapes
        dh = torch.empty(hs, dtype=torch.float64, device=c.device)
        deri = torch.empty(es, dtype=torch.float64, device=c.device)
        B.shci_energy_backward(ctx.lib_ctx.handle, c, float(grad_e), dh, deri)
        ctx.lib_ctx.close()
        return dh, deri, None, None, None, None, None, None, None, None
