"""Parameter gradient of the energy + force loss (Sec. II.B) on the GPU (dp_param_grad).

The FP64 path must reproduce the oracle's exact (hyper-dual) loss derivative along parameter
directions, and central differences of the GPU's own FP64 loss with h = 1e-5; the FP32 path
(the training precision) must stay close to the FP64 gradient.  The torch.autograd.Function
must hand exactly this gradient to PyTorch, and a few optimiser steps must lower the loss.
"""
import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I
from _cases import tiny_frame, tiny_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pack(frames):
    nat = np.array([f.natoms for f in frames], dtype=np.int32)
    coord = np.concatenate([f.coord for f in frames])
    atype = np.concatenate([f.atype for f in frames]).astype(np.int32)
    boxes = np.stack([f.box for f in frames])
    return nat, coord, atype, boxes


def _targets(cfg, q, frames):
    """Reference energies and forces from the oracle under a second parameter set."""
    e, f = [], []
    for fr in frames:
        r = oracle.compute(cfg, q, fr.coord, fr.atype, fr.box)
        e.append(r.energy)
        f.append(r.force)
    return np.array(e), f


def _gpu_loss_and_seeds(m, frames, e_ref, f_ref, pE, pF):
    """Loss from the GPU energies/forces and the cotangents dL/dE_f, dL/dF_i."""
    from paper_2304_09409_gb300 import dpgb
    nat, coord, atype, boxes = _pack(frames)
    e, f, _, _ = dpgb.compute_batch(m, nat, coord, atype, boxes)
    B = len(frames)
    fref = np.concatenate(f_ref)
    per_atom_n = np.repeat(nat, nat).astype(np.float64)[:, None]
    L = float(np.sum(pE * (e - e_ref) ** 2 / nat + pF * np.array(
        [((fk - rk) ** 2).sum() for fk, rk in zip(np.split(f, np.cumsum(nat)[:-1]), f_ref)]) / (3 * nat)) / B)
    g_e = 2 * pE * (e - e_ref) / (nat * B)
    g_f = 2 * pF * (f - fref) / (3 * per_atom_n * B)
    return L, g_e, g_f


def _directions(cfg, n, seed):
    rng = I.Rng(seed)
    n_emb = sum(a * b + b for a, b in cfg.embed_layer_shapes()) * cfg.n_embed_nets
    last_bias = np.zeros(n)
    last_bias[-1] = 1.0  # output bias of the last type's fitting net
    return [rng.normal(n), np.r_[rng.normal(n_emb), np.zeros(n - n_emb)],
            np.r_[np.zeros(n_emb), rng.normal(n - n_emb)], last_bias]


@pytest.mark.parametrize("one_side", [0, 1])
def test_grad_fp64_matches_oracle_tiny(one_side):
    from paper_2304_09409_gb300 import dpgb
    cfg = tiny_model(one_side)
    p, q = I.make_params(cfg, 5), I.make_params(cfg, 6)
    frames = [tiny_frame(seed=s) for s in (3, 4, 7)]
    e_ref, f_ref = _targets(cfg, q, frames)
    m = dpgb.Model(cfg, p, precision="fp64")
    nat, coord, atype, boxes = _pack(frames)
    for pE, pF in ((1.0, 0.0), (0.0, 1.0), (0.3, 2.0)):
        L, g_e, g_f = _gpu_loss_and_seeds(m, frames, e_ref, f_ref, pE, pF)
        g = dpgb.param_grad(m, nat, coord, atype, boxes, g_e, g_f)
        for v in _directions(cfg, p.size, 11):
            L_o, dL_o = oracle.loss_dir(cfg, p, v, frames, e_ref, f_ref, pE, pF)
            assert abs(L - L_o) <= 1e-10 * max(1.0, abs(L_o))
            assert abs(g @ v - dL_o) <= 1e-9 * max(abs(dL_o), 1e-6 * abs(L_o)), (pE, pF, g @ v, dL_o)


def test_grad_fp64_matches_oracle_water():
    """Water frames of 192 atoms, targets from a second random-weight model."""
    from paper_2304_09409_gb300 import dpgb
    cfg = I.water_model()
    p, q = I.make_params(cfg, 0), I.make_params(cfg, 1)
    frames = [I.water_frame(s) for s in (1, 2)]
    e_ref, f_ref = _targets(cfg, q, frames)
    m = dpgb.Model(cfg, p, precision="fp64")
    nat, coord, atype, boxes = _pack(frames)
    L, g_e, g_f = _gpu_loss_and_seeds(m, frames, e_ref, f_ref, 0.02, 1.0)
    g = dpgb.param_grad(m, nat, coord, atype, boxes, g_e, g_f)
    for v in _directions(cfg, p.size, 12)[:2]:
        L_o, dL_o = oracle.loss_dir(cfg, p, v, frames, e_ref, f_ref, 0.02, 1.0)
        assert abs(L - L_o) <= 1e-10 * abs(L_o)
        assert abs(g @ v - dL_o) <= 1e-9 * abs(dL_o), (g @ v, dL_o)


def test_grad_fp64_vs_central_differences():
    """dL/dtheta . v against (L(theta + h v) - L(theta - h v)) / 2h, h = 1e-5, all on the GPU."""
    from paper_2304_09409_gb300 import dpgb
    cfg = I.water_model()
    p, q = I.make_params(cfg, 0), I.make_params(cfg, 1)
    frames = [I.water_frame(s) for s in (1, 2, 3)]
    e_ref, f_ref = _targets(cfg, q, frames)
    m = dpgb.Model(cfg, p, precision="fp64")
    nat, coord, atype, boxes = _pack(frames)
    L, g_e, g_f = _gpu_loss_and_seeds(m, frames, e_ref, f_ref, 0.02, 1.0)
    g = dpgb.param_grad(m, nat, coord, atype, boxes, g_e, g_f)
    h = 1e-5
    for v in _directions(cfg, p.size, 13):
        v = v / np.linalg.norm(v)
        m.set_params(p + h * v)
        Lp = _gpu_loss_and_seeds(m, frames, e_ref, f_ref, 0.02, 1.0)[0]
        m.set_params(p - h * v)
        Lm = _gpu_loss_and_seeds(m, frames, e_ref, f_ref, 0.02, 1.0)[0]
        m.set_params(p)
        fd = (Lp - Lm) / (2 * h)
        assert abs(g @ v - fd) <= 1e-6 * max(abs(fd), 1e-8 * L), (g @ v, fd)


def test_grad_batch_is_sum_of_frames():
    from paper_2304_09409_gb300 import dpgb
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    frames = [I.water_frame_n(27, seed=21), I.water_frame(4), I.water_frame_n(40, seed=22)]
    m = dpgb.Model(cfg, p, precision="fp64")
    nat, coord, atype, boxes = _pack(frames)
    rng = I.Rng(5)
    g_e = rng.normal(len(frames))
    g_f = rng.normal(3 * int(nat.sum())).reshape(-1, 3)
    g = dpgb.param_grad(m, nat, coord, atype, boxes, g_e, g_f)
    acc = np.zeros_like(g)
    off = np.concatenate([[0], np.cumsum(nat)])
    for k, fr in enumerate(frames):
        acc += dpgb.param_grad(m, nat[k:k + 1], fr.coord, fr.atype, fr.box[None], g_e[k:k + 1],
                               g_f[off[k]:off[k + 1]])
    assert np.abs(g - acc).max() <= 1e-10 * np.abs(acc).max()


def _c3_batch(n_frames=32):
    """Batches of 192-atom water frames (seeds 1..32) with targets from a second model."""
    cfg = I.water_model()
    frames = [I.water_frame(s) for s in range(1, n_frames + 1)]
    return cfg, frames


def test_grad_fp32_close_to_fp64_full_batch():
    """The FP32 gradient of the 32-frame training batch against the FP64 one, device arrays."""
    from paper_2304_09409_gb300 import dpgb
    cfg, frames = _c3_batch()
    p, q = I.make_params(cfg, 0), I.make_params(cfg, 1)
    nat, coord, atype, boxes = _pack(frames)
    ref = dpgb.Model(cfg, q, precision="fp64")
    e_ref, f_ref, _, _ = dpgb.compute_batch(ref, nat, coord, atype, boxes)
    m64 = dpgb.Model(cfg, p, precision="fp64")
    m32 = dpgb.Model(cfg, p, precision="fp32")
    e, f, _, _ = dpgb.compute_batch(m64, nat, coord, atype, boxes)
    B = len(frames)
    per_n = np.repeat(nat, nat).astype(np.float64)[:, None]
    g_e = 2 * 0.02 * (e - e_ref) / (nat * B)
    g_f = 2 * 1.0 * (f - f_ref) / (3 * per_n * B)
    dev = "cuda"
    args = (nat, torch.tensor(coord, device=dev), torch.tensor(atype, device=dev), boxes,
            torch.tensor(g_e, device=dev), torch.tensor(g_f, device=dev))
    g64 = dpgb.param_grad(m64, *args).cpu().numpy()
    g32 = dpgb.param_grad(m32, *args).cpu().numpy()
    rel = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    assert rel <= 1e-4, rel
    for v in _directions(cfg, p.size, 14)[:3]:
        assert abs(g32 @ v - g64 @ v) <= 1e-4 * abs(g64 @ v) + 1e-5 * np.linalg.norm(g64) * np.linalg.norm(v)


def test_autograd_function_and_training_steps():
    from paper_2304_09409_gb300 import dpgb
    from paper_2304_09409_gb300.autograd import DPForce, Trainer, ef_loss
    cfg, frames = _c3_batch(8)
    p, q = I.make_params(cfg, 0), I.make_params(cfg, 1)
    nat, coord, atype, boxes = _pack(frames)
    dev = "cuda"
    coord_t, atype_t = torch.tensor(coord, device=dev), torch.tensor(atype, device=dev)
    ref = dpgb.Model(cfg, q, precision="fp64")
    e_ref, f_ref, _, _ = dpgb.compute_batch(ref, nat, coord_t, atype_t, boxes)
    m = dpgb.Model(cfg, p, precision="fp64")
    params = torch.tensor(p, device=dev, requires_grad=True)
    e, f, _ = DPForce.apply(params, m, nat, coord_t, atype_t, boxes)
    L = ef_loss(e, f, e_ref, f_ref, nat, 0.02, 1.0)
    L.backward()
    # the same gradient straight from the C ABI
    B = len(frames)
    per_n = torch.tensor(np.repeat(nat, nat).astype(np.float64), device=dev)[:, None]
    nat_t = torch.tensor(nat.astype(np.float64), device=dev)
    g_e = 2 * 0.02 * (e.detach() - e_ref) / (nat_t * B)
    g_f = 2 * (f.detach() - f_ref) / (3 * per_n * B)
    g = dpgb.param_grad(m, nat, coord_t, atype_t, boxes, g_e, g_f)
    assert torch.allclose(params.grad, g, rtol=1e-10, atol=1e-12 * float(g.abs().max()))
    # FP32 training: the loss goes down over a few Adam steps
    m32 = dpgb.Model(cfg, p, precision="fp32")
    tr = Trainer(m32, p, lr=1e-3, pE=0.02, pF=1.0)
    losses = [tr.step(nat, coord_t, atype_t, boxes, e_ref, f_ref) for _ in range(6)]
    assert losses[-1] < losses[0], losses


def test_grad_rejects_compressed_and_bad_sizes():
    from paper_2304_09409_gb300 import dpgb
    cfg = tiny_model()
    p = I.make_params(cfg, 5)
    fr = tiny_frame()
    mc = dpgb.Model(cfg, p, precision="fp32", compressed=True)
    with pytest.raises(dpgb.DPError):
        dpgb.param_grad(mc, np.array([fr.natoms]), fr.coord, fr.atype, fr.box[None], np.zeros(1),
                        np.zeros((fr.natoms, 3)))
    with pytest.raises(dpgb.DPError):
        mc.set_params(p)
    m = dpgb.Model(cfg, p, precision="fp64")
    with pytest.raises(dpgb.DPError):
        m.set_params(p[:-1])


def _targets_v(cfg, q, frames):
    e, f, v = [], [], []
    for fr in frames:
        r = oracle.compute(cfg, q, fr.coord, fr.atype, fr.box)
        e.append(r.energy)
        f.append(r.force)
        v.append(r.virial)
    return np.array(e), f, np.array(v)


@pytest.mark.parametrize("one_side", [0, 1])
def test_grad_fp64_virial_term_matches_oracle(one_side):
    """The virial term of Eq. (loss): dp_param_grad with a virial cotangent (FP64) against the
    oracle's exact hyper-dual derivative, virial alone and with the energy and force terms."""
    from paper_2304_09409_gb300 import dpgb
    cfg = tiny_model(one_side)
    p, q = I.make_params(cfg, 5), I.make_params(cfg, 6)
    frames = [tiny_frame(seed=s) for s in (3, 4, 7)]
    e_ref, f_ref, v_ref = _targets_v(cfg, q, frames)
    m = dpgb.Model(cfg, p, precision="fp64")
    nat, coord, atype, boxes = _pack(frames)
    e, f, v, _ = dpgb.compute_batch(m, nat, coord, atype, boxes)
    B = len(frames)
    fref = np.concatenate(f_ref)
    per_n = np.repeat(nat, nat).astype(np.float64)[:, None]
    for pE, pF, pV in ((0.0, 0.0, 1.0), (0.3, 2.0, 0.7)):
        g_e = 2 * pE * (e - e_ref) / (nat * B)
        g_f = 2 * pF * (f - fref) / (3 * per_n * B)
        g_v = 2 * pV * (v - v_ref) / (9 * nat[:, None, None] * B)
        g = dpgb.param_grad(m, nat, coord, atype, boxes, g_e, g_f, g_virial=g_v)
        for d in _directions(cfg, p.size, 31):
            L_o, dL_o = oracle.loss_dir(cfg, p, d, frames, e_ref, f_ref, pE, pF, pV, v_ref)
            assert abs(g @ d - dL_o) <= 1e-9 * max(abs(dL_o), 1e-6 * abs(L_o)), (pE, pF, pV, g @ d, dL_o)


def test_trainer_with_virial_and_schedules():
    """Eq. (loss) with all three terms through the autograd Function (its gradient equal to the
    C ABI's), Eq. (learning_rate) and the prefactor schedule, and FP32 Adam steps that lower the
    loss."""
    from paper_2304_09409_gb300 import dpgb
    from paper_2304_09409_gb300.autograd import DPForce, Schedule, Trainer, efv_loss, learning_rate, prefactor
    cfg, frames = _c3_batch(4)
    p, q = I.make_params(cfg, 0), I.make_params(cfg, 1)
    nat, coord, atype, boxes = _pack(frames)
    dev = "cuda"
    coord_t, atype_t = torch.tensor(coord, device=dev), torch.tensor(atype, device=dev)
    ref = dpgb.Model(cfg, q, precision="fp64")
    e_ref, f_ref, v_ref, _ = dpgb.compute_batch(ref, nat, coord_t, atype_t, boxes)
    m = dpgb.Model(cfg, p, precision="fp64")
    params = torch.tensor(p, device=dev, requires_grad=True)
    e, f, v = DPForce.apply(params, m, nat, coord_t, atype_t, boxes)
    L = efv_loss(e, f, v, e_ref, f_ref, v_ref, nat, 0.02, 1.0, 0.5)
    L.backward()
    B = len(frames)
    per_n = torch.tensor(np.repeat(nat, nat).astype(np.float64), device=dev)[:, None]
    nat_t = torch.tensor(nat.astype(np.float64), device=dev)
    g_e = 2 * 0.02 * (e.detach() - e_ref) / (nat_t * B)
    g_f = 2 * (f.detach() - f_ref) / (3 * per_n * B)
    g_v = 2 * 0.5 * (v.detach() - v_ref) / (9 * nat_t[:, None, None] * B)
    g = dpgb.param_grad(m, nat, coord_t, atype_t, boxes, g_e, g_f, g_virial=g_v)
    assert torch.allclose(params.grad, g, rtol=1e-10, atol=1e-12 * float(g.abs().max()))
    # the schedules of Sec. II.B
    assert learning_rate(0, 1e-3, 1e-5, 1000, 100) == pytest.approx(1e-3)
    assert learning_rate(1000, 1e-3, 1e-5, 1000, 100) == pytest.approx(1e-5, rel=1e-9)
    assert learning_rate(150, 1e-3, 1e-5, 1000, 100) == pytest.approx(1e-3 * (1e-2) ** 0.1, rel=1e-9)
    assert prefactor(1e-3, 1e-3, 0.02, 1.0) == pytest.approx(0.02)
    assert prefactor(0.0, 1e-3, 0.02, 1.0) == pytest.approx(1.0)
    sched = Schedule(lr0=1e-3, lr_stop=1e-4, stop_steps=8, decay_steps=2, pE=(0.02, 1.0), pF=(1.0, 1.0),
                     pV=(0.5, 0.1))
    m32 = dpgb.Model(cfg, p, precision="fp32")
    tr = Trainer(m32, p, schedule=sched)
    fixed = (0.02, 1.0, 0.5)  # the prefactors move with the schedule: compare at fixed ones
    L0 = float(tr.loss(nat, coord_t, atype_t, boxes, e_ref, f_ref, v_ref, pref=fixed).detach())
    for _ in range(6):
        tr.step(nat, coord_t, atype_t, boxes, e_ref, f_ref, v_ref)
    assert tr.opt.param_groups[0]["lr"] == pytest.approx(learning_rate(5, 1e-3, 1e-4, 8, 2))
    L1 = float(tr.loss(nat, coord_t, atype_t, boxes, e_ref, f_ref, v_ref, pref=fixed).detach())
    assert L1 < L0, (L0, L1)
