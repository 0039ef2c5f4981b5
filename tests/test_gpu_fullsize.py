"""Parity at the benchmark sizes, in the launch configuration bench.py times.

* 256^3 (16,777,216 particles, p = 10, sigma = h, BF16x3 M2L): sampled targets against the FP64
  direct sum over the central 27 boxes (FMM with no super-level images: the same tree, lists
  and kernels as the benchmark, whose 27^3 images differ only by the root lattice operator).
* 128^3, all particles: the fully periodic field (Fourier series of the smoothed vorticity)
  against the FMM with 6 super-levels of images (2187^3 boxes), u compared after removing the
  uniform velocity that the cube-truncated image sum carries.
* Config sweeps: expansion order and leaf size at 64^3; core overlap and M2L precision at 128^3.
"""
import numpy as np
import pytest

import oracle
import workload as wl
from gpu_util import rel_l2, rel_l2_demeaned, run_fmm

pytestmark = pytest.mark.gpu


def test_bench_workload_256cubed_sampled():
    f = wl.make_vortex_lattice(256, 4, 1)
    tid = wl.target_subset(256 ** 3, 12, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=1, targets=tid)
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, periodic_levels=0, m2l="bf16x3")
    # one near ring; the second ring goes to the M2L with the Gaussian-tail correction
    assert info["depth"] == 6 and info["near_rings"] == 1 and info["correction_rings"] == 2
    eu, es = rel_l2(u[tid], uo), rel_l2(s[tid], so)
    print("256^3 sampled: u %.3e S %.3e" % (eu, es))
    assert eu < 1e-4 and es < 1e-3


def test_fully_periodic_128cubed_all_particles():
    f = wl.make_vortex_lattice(128, 4, 1)
    ul, sl = oracle.spectral.lattice(128, f["alpha"], f["sigma"])
    u, s, _ = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, periodic_levels=6, m2l="bf16x3")
    eu, es = rel_l2_demeaned(u, ul), rel_l2(s, sl)
    print("128^3 all particles vs periodic series: u %.3e S %.3e" % (eu, es))
    assert eu < 1e-4 and es < 1e-3


@pytest.fixture(scope="module")
def case64():
    f = wl.make_vortex_lattice(64, 8, 1)
    tid = wl.target_subset(64 ** 3, 64, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=1, targets=tid)
    return f, tid, uo, so


def test_order_sweep_64cubed(case64):
    # error falls geometrically with p (Section 5.1: O(p^3 N) work, error exponential in p)
    f, tid, uo, so = case64
    eu = []
    for p in (4, 6, 8, 10):
        u, s, _ = run_fmm(f["x"], f["alpha"], f["sigma"], p=p, periodic_levels=0, m2l="fp32")
        eu.append(rel_l2(u[tid], uo))
        print("p=%d u %.3e S %.3e" % (p, eu[-1], rel_l2(s[tid], so)))
    assert eu[0] > eu[1] > eu[2] > eu[3]
    assert eu[3] < 1e-4


@pytest.mark.parametrize("ncrit", [32, 64, 128, 256])
def test_leaf_size_sweep_64cubed(case64, ncrit):
    f, tid, uo, so = case64
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, ncrit=ncrit, periodic_levels=0, m2l="fp32")
    eu, es = rel_l2(u[tid], uo), rel_l2(s[tid], so)
    print("ncrit=%d depth=%d R=%d: u %.3e S %.3e" % (ncrit, info["depth"], info["near_rings"], eu, es))
    assert eu < 1e-4 and es < 1e-3


@pytest.mark.parametrize("ratio", [0.8, 1.0, 1.5])
def test_overlap_and_precision_128cubed(ratio):
    # config 3: sigma/h in {0.8, 1, 1.5}; M2L in FP32, TF32x3 and BF16x3 (P2P FP32, FP64 root)
    f = wl.make_vortex_lattice(128, 4, 1, sigma_over_h=ratio)
    tid = wl.target_subset(128 ** 3, 24, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=1, targets=tid)
    ncrit = 512 if ratio > 1.2 else 64   # sigma = 1.5 h needs 8h leaves for R <= 2
    for m2l in ("fp32", "tf32x3", "bf16x3"):
        u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, ncrit=ncrit, periodic_levels=0, m2l=m2l)
        eu, es = rel_l2(u[tid], uo), rel_l2(s[tid], so)
        print("sigma/h=%.1f %s depth=%d R=%d: u %.3e S %.3e" % (ratio, m2l, info["depth"], info["near_rings"], eu, es))
        assert eu < 1e-4 and es < 1e-3


def test_reduced_cutoff_with_spread_cores_128cubed():
    # rho_cut = 5 (the time-step setting): cores spread to 1.5 h stay on 4h leaves within two rings;
    # the dropped smoothing tail 1 - q(5) = 1.5e-5 keeps the p = 10 accuracy
    f = wl.make_vortex_lattice(128, 4, 1, sigma_over_h=1.5)
    tid = wl.target_subset(128 ** 3, 24, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=1, targets=tid)
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, rho_cut=5.0, periodic_levels=0, m2l="bf16x3")
    eu, es = rel_l2(u[tid], uo), rel_l2(s[tid], so)
    print("rho_cut=5 sigma/h=1.5 depth=%d R=%d: u %.3e S %.3e" % (info["depth"], info["near_rings"], eu, es))
    assert info["depth"] == 5 and info["near_rings"] == 1 and info["correction_rings"] == 2
    assert eu < 1e-4 and es < 1e-3
