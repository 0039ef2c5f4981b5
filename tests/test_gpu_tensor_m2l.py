"""Tensor-core M2L (tcgen05, BF16x3 / TF32x3 split products) against the FP32 CUDA-core M2L
and against the FP64 oracle.

The split products keep ~2^-16 (BF16x3) / ~2^-22 (TF32x3) relative error per translation, so
the FMM result must agree with the FP32 M2L path to about that level, and keep the p = 10
accuracy target against the oracle.
"""
import numpy as np
import pytest

import oracle
import workload as wl
from gpu_util import rel_l2, run_fmm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def field32():
    return wl.make_vortex_lattice(32, 4, 1)


@pytest.fixture(scope="module")
def fp32_ref(field32):
    f = field32
    return run_fmm(f["x"], f["alpha"], f["sigma"], p=10, depth=3, periodic_levels=2, m2l="fp32")


@pytest.mark.parametrize("m2l,tol", [("bf16x3", 2e-5), ("tf32x3", 5e-6)])
def test_tensor_m2l_matches_fp32_m2l(field32, fp32_ref, m2l, tol):
    f = field32
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, depth=3, periodic_levels=2, m2l=m2l)
    u32, s32, _ = fp32_ref
    eu, es = rel_l2(u, u32), rel_l2(s, s32)
    print(m2l, info, eu, es)
    assert eu < tol
    assert es < tol


@pytest.mark.parametrize("m2l", ["bf16x3", "tf32x3"])
def test_tensor_m2l_against_oracle_64cubed(m2l):
    f = wl.make_vortex_lattice(64, 8, 1)
    tid = wl.target_subset(64 ** 3, 96, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=1, targets=tid)
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, periodic_levels=0, m2l=m2l)
    assert info["depth"] == 4
    assert rel_l2(u[tid], uo) < 1e-4
    assert rel_l2(s[tid], so) < 1e-3


def test_tensor_m2l_deterministic(field32):
    # two evaluations give bitwise equal results (no atomics in the accumulation)
    f = field32
    a = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, depth=3, m2l="bf16x3")
    b = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, depth=3, m2l="bf16x3")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
