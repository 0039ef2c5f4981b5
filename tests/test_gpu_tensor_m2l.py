"""Tensor-core M2L (tcgen05, BF16x3 / TF32x3 split products) against the FP32 CUDA-core M2L
and against the FP64 oracle.

The split products keep ~2^-16 (BF16x3) / ~2^-22 (TF32x3) relative error per product.  The
tensor-core sums still sit further from FP64 than the FP32 CUDA-core M2L, by an amount that grows
with the number of MMA K-steps into one accumulator (TF32 takes K = 8 per instruction, BF16 16, so
TF32x3 lands behind BF16x3): with 189 leaf-level offsets (one near ring) about 1e-5 in u against
1.3e-6 for FP32.  That stays well inside the p = 10 accuracy target against the oracle.
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


@pytest.mark.parametrize("m2l,tol", [("bf16x3", 3e-5), ("tf32x3", 3e-5)])
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


@pytest.mark.parametrize("near_rings", [1, 2])
def test_m2l_precisions_against_fp64_fmm_same_lists(field32, near_rings):
    # one tree and one set of interaction lists in every run (rho_cut = 4 keeps the near field at
    # the requested rings with no correction), so the difference is the M2L arithmetic alone
    f = field32
    kw = dict(p=10, depth=3, periodic_levels=2, near_rings=near_rings, rho_cut=4.0)
    u64, s64, _ = run_fmm(f["x"], f["alpha"], f["sigma"], dtype="f64", m2l="fp64", **kw)
    for m2l, tol in (("fp32", 6e-6), ("tf32x3", 3e-5), ("bf16x3", 3e-5)):
        u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], m2l=m2l, **kw)
        assert info["near_rings"] == near_rings and info["correction_rings"] == 0
        eu, es = rel_l2(u, u64), rel_l2(s, s64)
        print("R=%d %s: u %.3e S %.3e" % (near_rings, m2l, eu, es))
        assert eu < tol and es < tol


@pytest.mark.parametrize("m2l", ["bf16x3", "tf32x3"])
def test_line_levels_match_fp32_m2l_128cubed(m2l):
    # depth 5: level 5 (16 cells per side and parity) runs the source-line kernel, levels 3-4 the
    # gathered one; every particle's u and S against the FP32 CUDA-core M2L on the same tree
    f = wl.make_vortex_lattice(128, 4, 1)
    kw = dict(p=10, depth=5, periodic_levels=2)
    u32, s32, _ = run_fmm(f["x"], f["alpha"], f["sigma"], m2l="fp32", **kw)
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], m2l=m2l, **kw)
    eu, es = rel_l2(u, u32), rel_l2(s, s32)
    print(m2l, info, eu, es)
    assert eu < 4e-5 and es < 4e-5


@pytest.mark.parametrize("m2l", ["bf16x3", "tf32x3"])
def test_line_levels_deep_tree_match_fp32_m2l(m2l):
    # 64^3 particles on a depth-7 tree: levels 5, 6, 7 (16, 32, 64 cells per side and parity)
    # all take the source-line kernel (its TMA tensor boxes of 2-byte and of 4-byte operands);
    # sparse leaves, one near ring (rho_cut sigma within one leaf width: no correction ring)
    f = wl.make_vortex_lattice(64, 8, 1)
    kw = dict(p=10, depth=7, periodic_levels=1, rho_cut=2.0)
    sig = 0.25 * f["sigma"]
    u32, s32, _ = run_fmm(f["x"], f["alpha"], sig, m2l="fp32", **kw)
    u, s, info = run_fmm(f["x"], f["alpha"], sig, m2l=m2l, **kw)
    eu, es = rel_l2(u, u32), rel_l2(s, s32)
    print(info, eu, es)
    assert info["depth"] == 7
    assert eu < 4e-5 and es < 4e-5
