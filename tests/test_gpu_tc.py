"""Tensor-core (tcgen05) GEMM and the BF16 fitting path, through the C-ABI.

The GEMM is checked against an FP64 product of the same BF16-rounded operands (the only
difference left is FP32 accumulation order); the BF16 path against the FP64 oracle with
the contract's mixed-precision bar (|dF| <= 1e-3 eV/A) and a bar relative to the force RMS.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2304_09409_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gemm(A, Bt):
    from paper_2304_09409_gb300 import dpgb
    L = dpgb.lib()
    L.dp_gemm_bf16.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]
    rows, K = A.shape
    N = Bt.shape[0]
    C = torch.empty((rows, N), dtype=torch.float32, device="cuda")
    rc = L.dp_gemm_bf16(rows, K, N, A.data_ptr(), Bt.data_ptr(), C.data_ptr(), None)
    assert rc == 0, dpgb.last_error()
    return C


@pytest.mark.parametrize("rows,K,N", [(1000, 1600, 240), (300, 240, 1600), (130, 64, 16), (257, 248, 96),
                                      (12288, 240, 240)])
def test_tc_gemm_matches_fp64_product_of_bf16_operands(rows, K, N):
    rng = I.Rng(rows + K + N)
    a = rng.normal(rows * K).reshape(rows, K)
    b = rng.normal(N * K).reshape(N, K)
    A = torch.tensor(a, dtype=torch.bfloat16, device="cuda")
    Bt = torch.tensor(b, dtype=torch.bfloat16, device="cuda")
    C = _gemm(A, Bt).cpu().numpy().astype(np.float64)
    ref = A.float().cpu().numpy().astype(np.float64) @ Bt.float().cpu().numpy().astype(np.float64).T
    err = np.abs(C - ref).max()
    assert err <= 1e-5 * np.sqrt(K) * np.abs(ref).max(), err


def test_tc_gemm_twice_same_result():
    rng = I.Rng(5)
    A = torch.tensor(rng.normal(512 * 256).reshape(512, 256), dtype=torch.bfloat16, device="cuda")
    Bt = torch.tensor(rng.normal(240 * 256).reshape(240, 256), dtype=torch.bfloat16, device="cuda")
    c1 = _gemm(A, Bt)
    c2 = _gemm(A, Bt)
    assert torch.equal(c1, c2)


@pytest.fixture(scope="module")
def water():
    cfg = I.water_model()
    p = I.make_params(cfg, 0)
    fr = I.water_frame(0)
    ref = oracle.compute(cfg, p, fr.coord, fr.atype, fr.box)
    return cfg, p, fr, ref


def test_bf16_compressed_water192(water):
    from paper_2304_09409_gb300 import dpgb
    cfg, p, fr, ref = water
    m = dpgb.Model(cfg, p, precision="bf16", compressed=True)
    e, f, v, ae = m.compute(fr.coord, fr.atype, fr.box, atom_energy=True)
    frms = np.sqrt((ref.force ** 2).mean())
    ferr = np.abs(f - ref.force).max()
    eerr = abs(float(e[0]) - ref.energy) / fr.natoms
    print(f"bf16: |dF|max={ferr:.3e} (F rms {frms:.3e}), |dE|/atom={eerr:.3e}")
    assert ferr <= 1e-3
    assert ferr <= 0.05 * frms
    assert eerr <= 1e-2
    assert np.abs(v - ref.virial).max() <= 0.05 * np.abs(ref.virial).max()


def test_bf16_compressed_water12288_replicas(water):
    from paper_2304_09409_gb300 import dpgb
    cfg, p, fr, ref = water
    big = I.replicate(fr, (4, 4, 4))
    m = dpgb.Model(cfg, p, precision="bf16", compressed=True)
    e, f, v, ae = m.compute(big.coord, big.atype, big.box, atom_energy=True)
    assert np.abs(f - np.tile(ref.force, (64, 1))).max() <= 1e-3
    assert abs(float(e[0]) - 64 * ref.energy) / big.natoms <= 1e-2
