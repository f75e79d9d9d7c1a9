"""torch.autograd binding of the energy/force path for training (Sec. II.B).

`DPForce.apply(params, model, natoms, coord, atype, boxes)` returns per-frame energies E [F]
and forces F [N, 3] of the frames as functions of the flat FP64 parameter vector `params`
(a torch CUDA tensor with requires_grad).  Its backward is dp_param_grad: the vector-Jacobian
product of (E, F) with the incoming cotangents, computed by the library's own tangent and
reverse kernels (a second derivative of E for the force part).  PyTorch only holds the
tensors and chains the loss; no framework autograd runs through the model itself.

`ef_loss` is the energy + force loss of Sec. II.B; `Trainer` is a plain Adam loop over it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dpgb


class DPForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, model, natoms, coord, atype, boxes):
        model.set_params(params)
        nat = np.ascontiguousarray(natoms, dtype=np.int32)
        if boxes is None:
            if nat.size != 1:
                raise ValueError("open boundaries need exactly one frame")
            e, f, v, _ = model.compute(coord, atype, None)
            v = v.reshape(1, 3, 3)
        else:
            e, f, v, _ = dpgb.compute_batch(model, nat, coord, atype, boxes)
        ctx.model = model
        ctx.frames = (nat, coord, atype, boxes)
        ctx.save_for_backward(params)
        ctx.mark_non_differentiable(v)
        return e, f, v

    @staticmethod
    def backward(ctx, g_e, g_f, g_v):
        (params,) = ctx.saved_tensors
        nat, coord, atype, boxes = ctx.frames
        if g_v is not None and bool(torch.any(g_v != 0)):
            raise NotImplementedError("the virial is not differentiable with respect to the parameters here")
        N = int(nat.sum())
        dev = params.device
        if g_e is None:
            g_e = torch.zeros(nat.size, dtype=torch.float64, device=dev)
        if g_f is None:
            g_f = torch.zeros((N, 3), dtype=torch.float64, device=dev)
        ctx.model.set_params(params)
        grad = dpgb.param_grad(ctx.model, nat, coord, atype, boxes, g_e.contiguous(), g_f.contiguous())
        return grad, None, None, None, None, None


def ef_loss(e, f, e_ref, f_ref, natoms, pE: float = 1.0, pF: float = 1.0):
    """L = (1/B) sum_f [ pE (E_f - E*_f)^2 / N_f + pF sum_{i in f} |F_i - F*_i|^2 / (3 N_f) ]."""
    nat = torch.as_tensor(np.asarray(natoms), dtype=torch.float64, device=e.device)
    B = nat.numel()
    frame = torch.repeat_interleave(torch.arange(B, device=e.device), nat.long())
    df2 = ((f - f_ref) ** 2).sum(dim=1)
    per_frame_f = torch.zeros(B, dtype=torch.float64, device=e.device).index_add_(0, frame, df2)
    return (pE * (e - e_ref) ** 2 / nat + pF * per_frame_f / (3.0 * nat)).sum() / B


class Trainer:
    """Adam on the flat parameter vector, one batch of frames per step."""

    def __init__(self, model, params, lr: float = 1e-3, pE: float = 1.0, pF: float = 1.0):
        self.model = model
        self.params = torch.nn.Parameter(torch.as_tensor(params, dtype=torch.float64, device=f"cuda:{model.device}"))
        self.opt = torch.optim.Adam([self.params], lr=lr)
        self.pE, self.pF = pE, pF

    def loss(self, natoms, coord, atype, boxes, e_ref, f_ref):
        e, f, _ = DPForce.apply(self.params, self.model, natoms, coord, atype, boxes)
        return ef_loss(e, f, e_ref, f_ref, natoms, self.pE, self.pF)

    def step(self, natoms, coord, atype, boxes, e_ref, f_ref) -> float:
        self.opt.zero_grad(set_to_none=True)
        L = self.loss(natoms, coord, atype, boxes, e_ref, f_ref)
        L.backward()
        self.opt.step()
        return float(L.detach())
