"""Host side of training (Sec. II.B), on the CPU: the learning-rate schedule of Eq. (learning_rate), the
prefactor schedule p_eta(tau), and the loss of Eq. (loss) with the cotangents it hands to the GPU
parameter gradient."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_09409_gb300.autograd import Schedule, ef_loss, efv_loss, learning_rate, prefactor  # noqa: E402


def test_learning_rate_is_a_staircase_from_start_to_stop():
    lr0, lr_stop, stop, s = 1e-3, 1e-6, 12000, 400
    r = (lr_stop / lr0) ** (s / stop)
    assert learning_rate(0, lr0, lr_stop, stop, s) == pytest.approx(lr0, rel=1e-15)
    assert learning_rate(stop, lr0, lr_stop, stop, s) == pytest.approx(lr_stop, rel=1e-12)
    for k in range(stop // s):
        at = [learning_rate(k * s + d, lr0, lr_stop, stop, s) for d in (0, 1, s // 2, s - 1)]
        assert len(set(at)) == 1, "constant within one decay period"
        nxt = learning_rate((k + 1) * s, lr0, lr_stop, stop, s)
        assert nxt / at[0] == pytest.approx(r, rel=1e-12), "one factor r per period"


def test_default_schedule_decays_by_about_five_percent_per_period():
    """1e-3 -> 3.51e-8 over 10^6 steps with a decay every 5,000 steps is 200 periods of r = 0.95."""
    sch = Schedule()
    r = (sch.lr_stop / sch.lr0) ** (sch.decay_steps / sch.stop_steps)
    assert r == pytest.approx(0.95, abs=2e-5)
    assert sch.at(5000)[0] / sch.at(4999)[0] == pytest.approx(r, rel=1e-12)


def test_prefactor_moves_linearly_from_start_to_limit():
    lr0 = 2e-3
    for p_start, p_limit in ((0.02, 1.0), (1000.0, 1.0), (0.5, 0.5)):
        assert prefactor(lr0, lr0, p_start, p_limit) == pytest.approx(p_start, rel=1e-15)
        assert prefactor(0.0, lr0, p_start, p_limit) == pytest.approx(p_limit, rel=1e-15)
        a, b = prefactor(0.3 * lr0, lr0, p_start, p_limit), prefactor(0.7 * lr0, lr0, p_start, p_limit)
        mid = prefactor(0.5 * lr0, lr0, p_start, p_limit)
        assert mid == pytest.approx(0.5 * (a + b), rel=1e-12)


def test_schedule_prefactors_follow_the_learning_rate():
    sch = Schedule(lr0=1e-3, lr_stop=1e-5, stop_steps=100, decay_steps=10, pE=(0.02, 1.0), pF=(1000.0, 1.0),
                   pV=(0.0, 0.5))
    lr, (pE, pF, pV) = sch.at(0)
    assert (lr, pE, pF, pV) == pytest.approx((1e-3, 0.02, 1000.0, 0.0))
    lr, (pE, pF, pV) = sch.at(100)
    x = 1e-5 / 1e-3
    assert lr == pytest.approx(1e-5, rel=1e-12)
    assert pE == pytest.approx(1.0 * (1 - x) + 0.02 * x, rel=1e-12)
    assert pF == pytest.approx(1.0 * (1 - x) + 1000.0 * x, rel=1e-12)
    assert pV == pytest.approx(0.5 * (1 - x), rel=1e-12)


def _frames(seed=0):
    rng = np.random.default_rng(seed)
    nat = np.array([3, 5, 2])
    B, N = len(nat), int(nat.sum())
    t = lambda *s: torch.tensor(rng.normal(size=s), dtype=torch.float64)
    return nat, t(B), t(N, 3), t(B, 3, 3), t(B), t(N, 3), t(B, 3, 3)


def _loss_by_loops(nat, e, f, v, e_ref, f_ref, v_ref, pE, pF, pV):
    """Eq. (loss) term by term, frame by frame, atom by atom."""
    B, total, off = len(nat), 0.0, 0
    for k, n in enumerate(nat):
        le = (float(e[k]) - float(e_ref[k])) ** 2 / n
        lf = sum(float(f[off + i, a] - f_ref[off + i, a]) ** 2 for i in range(n) for a in range(3)) / (3 * n)
        lv = sum(float(v[k, a, b] - v_ref[k, a, b]) ** 2 for a in range(3) for b in range(3)) / (9 * n)
        total += pE * le + pF * lf + pV * lv
        off += n
    return total / B


@pytest.mark.parametrize("pE,pF,pV", [(1.0, 1.0, 0.0), (0.02, 1000.0, 0.5), (0.0, 0.0, 1.0)])
def test_efv_loss_matches_its_terms(pE, pF, pV):
    nat, e, f, v, e_ref, f_ref, v_ref = _frames()
    L = float(efv_loss(e, f, v, e_ref, f_ref, v_ref, nat, pE, pF, pV))
    assert L == pytest.approx(_loss_by_loops(nat, e, f, v, e_ref, f_ref, v_ref, pE, pF, pV), rel=1e-13)
    if pV == 0.0:
        assert float(ef_loss(e, f, e_ref, f_ref, nat, pE, pF)) == pytest.approx(L, rel=1e-15)


def test_efv_loss_cotangents():
    """The cotangents the loss passes back to E, F and Xi (what the GPU parameter gradient contracts):
    2 pE dE / (N B), 2 pF dF / (3 N B), 2 pXi dXi / (9 N B)."""
    nat, e, f, v, e_ref, f_ref, v_ref = _frames(1)
    pE, pF, pV = 0.02, 3.0, 0.5
    for x in (e, f, v):
        x.requires_grad_(True)
    efv_loss(e, f, v, e_ref, f_ref, v_ref, nat, pE, pF, pV).backward()
    B = len(nat)
    n_t = torch.tensor(nat, dtype=torch.float64)
    per_atom_n = torch.tensor(np.repeat(nat, nat), dtype=torch.float64)[:, None]
    torch.testing.assert_close(e.grad, 2 * pE * (e.detach() - e_ref) / (n_t * B), rtol=1e-13, atol=0)
    torch.testing.assert_close(f.grad, 2 * pF * (f.detach() - f_ref) / (3 * per_atom_n * B), rtol=1e-13, atol=0)
    torch.testing.assert_close(v.grad, 2 * pV * (v.detach() - v_ref) / (9 * n_t[:, None, None] * B), rtol=1e-13,
                               atol=0)
    assert math.isfinite(float(e.grad.sum()))
