"""torch.autograd binding of the energy/force/virial path for training (Sec. II.B).

`DPForce.apply(params, model, natoms, coord, atype, boxes)` returns per-frame energies E [F],
forces F [N, 3] and virials Xi [F, 3, 3] of the frames as functions of the flat FP64 parameter
vector `params` (a torch CUDA tensor with requires_grad).  Its backward is dp_param_grad: the
vector-Jacobian product of (E, F, Xi) with the incoming cotangents, computed by the library's
own tangent and reverse kernels (second derivatives of E for the force and virial parts).
PyTorch only holds the tensors and chains the loss; no framework autograd runs through the
model itself.

`efv_loss` is the loss of Eq. (loss) with the energy, force and virial terms; `learning_rate`
is Eq. (learning_rate) and `prefactor` the schedule of p_eta(tau); `Trainer` is an Adam loop
that applies both schedules step by step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

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
        return e, f, v

    @staticmethod
    def backward(ctx, g_e, g_f, g_v):
        (params,) = ctx.saved_tensors
        nat, coord, atype, boxes = ctx.frames
        N = int(nat.sum())
        dev = params.device
        if g_e is None:
            g_e = torch.zeros(nat.size, dtype=torch.float64, device=dev)
        if g_f is None:
            g_f = torch.zeros((N, 3), dtype=torch.float64, device=dev)
        if g_v is not None and not bool(torch.any(g_v != 0)):
            g_v = None
        if g_v is not None and boxes is None:
            raise ValueError("the virial of an open-boundary frame has no parameter gradient here")
        ctx.model.set_params(params)
        grad = dpgb.param_grad(ctx.model, nat, coord, atype, boxes, g_e.contiguous(), g_f.contiguous(),
                               g_virial=None if g_v is None else g_v.contiguous())
        return grad, None, None, None, None, None


def efv_loss(e, f, v, e_ref, f_ref, v_ref, natoms, pE: float = 1.0, pF: float = 1.0, pV: float = 0.0):
    """Eq. (loss) for one step: (1/B) sum_f [ pE L_E + pF L_F + pV L_Xi ] with
    L_E = (E_f - E*_f)^2 / N_f, L_F = sum_{i in f} |F_i - F*_i|^2 / (3 N_f),
    L_Xi = sum_ab (Xi_f,ab - Xi*_f,ab)^2 / (9 N_f)."""
    nat = torch.as_tensor(np.asarray(natoms), dtype=torch.float64, device=e.device)
    B = nat.numel()
    frame = torch.repeat_interleave(torch.arange(B, device=e.device), nat.long())
    df2 = ((f - f_ref) ** 2).sum(dim=1)
    per_frame_f = torch.zeros(B, dtype=torch.float64, device=e.device).index_add_(0, frame, df2)
    L = pE * (e - e_ref) ** 2 / nat + pF * per_frame_f / (3.0 * nat)
    if pV != 0.0 and v_ref is not None:
        L = L + pV * ((v - v_ref) ** 2).reshape(B, 9).sum(dim=1) / (9.0 * nat)
    return L.sum() / B


def ef_loss(e, f, e_ref, f_ref, natoms, pE: float = 1.0, pF: float = 1.0):
    """The energy + force part of Eq. (loss)."""
    return efv_loss(e, f, None, e_ref, f_ref, None, natoms, pE, pF, 0.0)


def learning_rate(step: int, lr0: float, lr_stop: float, stop_steps: int, decay_steps: int) -> float:
    """Eq. (learning_rate): gamma(tau) = gamma0 r^floor(tau / s), r = (gamma_stop / gamma0)^(s / tau_stop)."""
    r = (lr_stop / lr0) ** (decay_steps / stop_steps)
    return lr0 * r ** math.floor(step / decay_steps)


def prefactor(lr: float, lr0: float, p_start: float, p_limit: float) -> float:
    """p_eta(tau) = p_limit (1 - gamma(tau)/gamma0) + p_start gamma(tau)/gamma0 (Sec. II.B)."""
    x = lr / lr0
    return p_limit * (1.0 - x) + p_start * x


@dataclass
class Schedule:
    """Hyper-parameters of Sec. II.B: learning rate gamma0 -> gamma_stop over stop_steps with
    decay every decay_steps, and start / limit prefactors of each loss term."""
    lr0: float = 1e-3
    lr_stop: float = 3.51e-8
    stop_steps: int = 1000000
    decay_steps: int = 5000
    pE: tuple = (0.02, 1.0)
    pF: tuple = (1000.0, 1.0)
    pV: tuple = (0.0, 0.0)

    def at(self, step: int):
        lr = learning_rate(step, self.lr0, self.lr_stop, self.stop_steps, self.decay_steps)
        return lr, tuple(prefactor(lr, self.lr0, *p) for p in (self.pE, self.pF, self.pV))


class Trainer:
    """Adam on the flat parameter vector, one batch of frames per step, with the learning rate
    of Eq. (learning_rate) and the prefactor schedule of Sec. II.B (a constant schedule when
    only lr / pE / pF / pV are given)."""

    def __init__(self, model, params, lr: float = 1e-3, pE: float = 1.0, pF: float = 1.0, pV: float = 0.0,
                 schedule: Schedule = None):
        self.model = model
        self.params = torch.nn.Parameter(torch.as_tensor(params, dtype=torch.float64, device=f"cuda:{model.device}"))
        self.sched = schedule or Schedule(lr0=lr, lr_stop=lr, stop_steps=1, decay_steps=1, pE=(pE, pE),
                                          pF=(pF, pF), pV=(pV, pV))
        self.opt = torch.optim.Adam([self.params], lr=self.sched.lr0)
        self.step_count = 0

    def loss(self, natoms, coord, atype, boxes, e_ref, f_ref, v_ref=None, pref=None):
        pE, pF, pV = pref if pref is not None else self.sched.at(self.step_count)[1]
        e, f, v = DPForce.apply(self.params, self.model, natoms, coord, atype, boxes)
        return efv_loss(e, f, v, e_ref, f_ref, v_ref, natoms, pE, pF, pV)

    def step(self, natoms, coord, atype, boxes, e_ref, f_ref, v_ref=None) -> float:
        lr, pref = self.sched.at(self.step_count)
        for g in self.opt.param_groups:
            g["lr"] = lr
        self.opt.zero_grad(set_to_none=True)
        L = self.loss(natoms, coord, atype, boxes, e_ref, f_ref, v_ref, pref)
        L.backward()
        self.opt.step()
        self.step_count += 1
        return float(L.detach())
