"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerances (each follows from the arithmetic it bounds):
* direct sum, FP64 kernels: 1e-12 relative L2 (only summation order and erf/exp rounding
  differ);
* direct sum, FP32 kernels: 2e-5 (FP32 accumulation of ~1e5 terms plus the 1.5e-7 error of
  the Abramowitz-Stegun erf);
* FMM at p = 10: u <= 1e-4 and S <= 1e-3 relative L2 (the accuracy target, 4 digits in the
  paper's Section 4.1 performance paragraph).
"""
import numpy as np
import pytest

import oracle
import workload as wl
from gpu_util import rel_l2, rel_l2_demeaned, run_fmm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def field16():
    return wl.make_vortex_lattice(16, 4, 1)


@pytest.fixture(scope="module")
def oracle16_k1(field16):
    f = field16
    return oracle.direct(f["x"], f["alpha"], f["sigma"], K=1)


def test_direct_fp64_matches_oracle(field16, oracle16_k1):
    f = field16
    u, s, _ = run_fmm(f["x"], f["alpha"], f["sigma"], method="direct", direct_images=1, dtype="f64")
    uo, so = oracle16_k1
    assert rel_l2(u, uo) < 1e-12
    assert rel_l2(s, so) < 1e-12


def test_direct_fp32_matches_oracle(field16, oracle16_k1):
    f = field16
    u, s, _ = run_fmm(f["x"], f["alpha"], f["sigma"], method="direct", direct_images=1, dtype="f32")
    uo, so = oracle16_k1
    assert rel_l2(u, uo) < 2e-5
    assert rel_l2(s, so) < 2e-5


def test_direct_jittered_ragged_and_coincident():
    # non-lattice positions (ragged leaves), points outside [0, L) that must wrap, and two
    # coincident distinct particles (their stretching pair term is the finite r -> 0 limit)
    n = 7
    h = 2 * np.pi / n
    rng = np.random.default_rng(4)
    x = wl.jitter(wl.lattice_positions(n), h, 0.45, seed=2)
    x[5] += np.array([2 * np.pi, -2 * np.pi, 0.0])
    x = np.vstack([x, x[10:11]])
    g = rng.normal(size=x.shape)
    sigma = 0.9 * h
    xo = np.mod(x, 2 * np.pi)
    uo, so = oracle.direct(xo, g, sigma, K=1)
    u, s, _ = run_fmm(x, g, sigma, method="direct", direct_images=1, dtype="f64")
    assert rel_l2(u, uo) < 1e-12
    assert rel_l2(s, so) < 1e-12


@pytest.mark.parametrize("p", [4, 6, 8, 10])
def test_fmm_fp64_order_convergence(field16, oracle16_k1, p, request):
    f = field16
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], method="fmm", p=p, depth=2,
                         periodic_levels=0, dtype="f64")
    uo, so = oracle16_k1
    eu, es = rel_l2(u, uo), rel_l2(s, so)
    print("p=%d depth=%d R=%d: u %.3e S %.3e" % (p, info["depth"], info["near_rings"], eu, es))
    bound_u = {4: 3e-2, 6: 3e-3, 8: 5e-4, 10: 1e-4}[p]
    bound_s = {4: 1e-1, 6: 2e-2, 8: 5e-3, 10: 1e-3}[p]
    assert eu < bound_u
    assert es < bound_s


def test_fmm_fp32_matches_fp64_fmm(field16):
    # the same tree and lists in both precisions: two smoothed near rings, no correction
    f = field16
    kw = dict(method="fmm", p=10, depth=2, periodic_levels=1, near_rings=2)
    u64, s64, _ = run_fmm(f["x"], f["alpha"], f["sigma"], dtype="f64", **kw)
    u32, s32, _ = run_fmm(f["x"], f["alpha"], f["sigma"], dtype="f32", m2l="fp32", **kw)
    assert rel_l2(u32, u64) < 2e-5
    assert rel_l2(s32, s64) < 2e-5


def test_fmm_periodic_one_super_level(field16):
    f = field16
    tid = wl.target_subset(4096, 512, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=4, targets=tid)
    u, s, _ = run_fmm(f["x"], f["alpha"], f["sigma"], method="fmm", p=10, depth=2,
                      periodic_levels=1, dtype="f64")
    assert rel_l2(u[tid], uo) < 1e-4
    assert rel_l2(s[tid], so) < 1e-3


def test_fmm_periodic_27cubed_images(field16):
    # the paper's 3^3 x 3^3 x 3^3 image cube (S = 2, K = 13), on a seeded target subset
    f = field16
    tid = wl.target_subset(4096, 48, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=13, targets=tid)
    u, s, _ = run_fmm(f["x"], f["alpha"], f["sigma"], method="fmm", p=10, depth=2,
                      periodic_levels=2, dtype="f32", m2l="fp32")
    assert rel_l2(u[tid], uo) < 1e-4
    assert rel_l2(s[tid], so) < 1e-3


def test_fmm_64cubed_sampled_fp32():
    f = wl.make_vortex_lattice(64, 8, 1)
    tid = wl.target_subset(64 ** 3, 96, seed=3)
    uo, so = oracle.direct(f["x"], f["alpha"], f["sigma"], K=1, targets=tid)
    u, s, info = run_fmm(f["x"], f["alpha"], f["sigma"], method="fmm", p=10, periodic_levels=0,
                         dtype="f32", m2l="fp32")
    print(info, rel_l2(u[tid], uo), rel_l2(s[tid], so))
    assert rel_l2(u[tid], uo) < 1e-4
    assert rel_l2(s[tid], so) < 1e-3


def test_fmm_jittered_nonuniform_leaves():
    # random (not lattice) positions: empty and crowded leaves, ragged tails
    n = 24
    h = 2 * np.pi / n
    rng = np.random.default_rng(9)
    x = rng.uniform(0, 2 * np.pi, (n ** 3, 3))
    g = rng.normal(size=x.shape) * h ** 3
    g -= g.mean(0)
    sigma = h
    tid = wl.target_subset(len(x), 128, seed=5)
    uo, so = oracle.direct(x, g, sigma, K=1, targets=tid)
    u, s, info = run_fmm(x, g, sigma, method="fmm", p=10, depth=2, periodic_levels=0, dtype="f64")
    assert info["max_leaf"] > 216
    assert rel_l2(u[tid], uo) < 1e-4
    assert rel_l2(s[tid], so) < 1e-3


def test_errors_reported():
    torch = pytest.importorskip("torch")
    import paper_1110_2921_gb300 as vf
    h = vf.VortexFMM(m2l="fp32")
    try:
        g = torch.zeros(8, 3, device="cuda")
        with pytest.raises(vf.VfmmError) as e:
            h.eval(g, 0.1)
        assert e.value.status == -4
        x = torch.rand(8, 3, device="cuda")
        h.build_tree(x)
        with pytest.raises(vf.VfmmError) as e:
            h.eval(g, float("nan"))
        assert e.value.status == -1
        # a NaN or infinite position has no leaf: the tree build fails with VFMM_ERR_ARG, the
        # handle holds no tree, and a valid build afterwards works
        for bad in (float("nan"), float("inf"), -float("inf")):
            xb = x.clone()
            xb[3, 1] = bad
            with pytest.raises(vf.VfmmError) as e:
                h.build_tree(xb)
            assert e.value.status == -1
            with pytest.raises(vf.VfmmError) as e:
                h.eval(g, 0.1)
            assert e.value.status == -4
        h.build_tree(x)
        u, s = h.eval(g, 0.1)
        h.sync()
        assert bool(torch.isfinite(u).all())
        # a core so wide that rho_cut sigma exceeds two leaf widths: the near field would need
        # a third ring
        xx = torch.rand(4096, 3, device="cuda") * 6.28
        gg = torch.zeros(4096, 3, device="cuda")
        h2 = vf.VortexFMM(m2l="fp32", depth=3)
        try:
            h2.build_tree(xx)
            with pytest.raises(vf.VfmmError) as e:
                h2.eval(gg, 1.0)
            assert e.value.status == -7
            # the spectrum wants a power-of-two lattice
            with pytest.raises(vf.VfmmError) as e:
                h2.energy_spectrum(torch.zeros(12 ** 3, 3, device="cuda"), 12, 4)
            assert e.value.status == -7
        finally:
            h2.close()
    finally:
        h.close()


@pytest.mark.parametrize("sigma_over_h", [1.0, 1.4])
def test_ring_two_correction_off_lattice(sigma_over_h):
    # jittered positions and wide cores: ring-2 pairs reach rho ~ 2, where the singular kernel of
    # the M2L misses a large part of the smoothed one; the correction pairs must restore it
    f = wl.make_vortex_lattice(32, 4, 1)
    h = 2 * np.pi / 32
    x = wl.jitter(f["x"], h, 0.45, seed=5)
    sigma = sigma_over_h * f["sigma"]
    tid = wl.target_subset(32 ** 3, 256, seed=3)
    uo, so = oracle.direct(x, f["alpha"], sigma, K=1, targets=tid)
    u, s, info = run_fmm(x, f["alpha"], sigma, p=10, depth=3, periodic_levels=0, m2l="bf16x3", rho_cut=5.0)
    assert info["near_rings"] == 1 and info["correction_rings"] == 2
    eu, es = rel_l2(u[tid], uo), rel_l2(s[tid], so)
    print("sigma/h=%.1f: u %.3e S %.3e" % (sigma_over_h, eu, es))
    assert eu < 1e-4 and es < 1e-3
    if sigma_over_h > 1.2:
        # without the correction (rho_cut sigma within one leaf width: one ring, no correction
        # pairs) the same evaluation misses the ring-2 Gaussian tail
        u1, s1, info1 = run_fmm(x, f["alpha"], sigma, p=10, depth=3, periodic_levels=0, m2l="bf16x3", rho_cut=2.8)
        assert info1["near_rings"] == 1 and info1["correction_rings"] == 0
        eu1, es1 = rel_l2(u1[tid], uo), rel_l2(s1[tid], so)
        print("uncorrected: u %.3e S %.3e" % (eu1, es1))
        assert eu1 > 3 * eu and es1 > 3 * es


def test_concurrent_far_field_matches_in_line():
    # the far field on the side stream, added after the P2P, gives the same FP32 sums as the
    # in-line order (near field, then far field added in the P2P epilogue): bitwise
    f = wl.make_vortex_lattice(32, 4, 1)
    kw = dict(p=10, depth=3, periodic_levels=2, m2l="bf16x3")
    u1, s1, _ = run_fmm(f["x"], f["alpha"], f["sigma"], concurrent_far=1, **kw)
    u0, s0, _ = run_fmm(f["x"], f["alpha"], f["sigma"], concurrent_far=0, **kw)
    assert np.array_equal(u1, u0) and np.array_equal(s1, s0)


def test_fmm_fp32_random_positions_line_kernel_levels():
    # uniform random positions on a depth-5 tree (2^21 - 77 particles: empty and crowded
    # leaves, ragged counts, target chunks beyond 64 per leaf), BF16x3 on the source-line
    # kernel, one near ring + ring-2 correction, concurrent far field
    n_side = 128
    h = 2 * np.pi / n_side
    rng = np.random.default_rng(21)
    N = 2 ** 21 - 77
    x = rng.uniform(0, 2 * np.pi, (N, 3))
    g = rng.normal(size=x.shape) * h ** 3
    sigma = h
    tid = wl.target_subset(N, 48, seed=6)
    uo, so = oracle.direct(x, g, sigma, K=1, targets=tid)
    u, s, info = run_fmm(x, g, sigma, p=10, depth=5, periodic_levels=0, m2l="bf16x3")
    assert info["max_leaf"] > 64 and info["near_rings"] == 1 and info["correction_rings"] == 2
    eu, es = rel_l2(u[tid], uo), rel_l2(s[tid], so)
    print("random 2^21: max leaf %d, u %.3e S %.3e" % (info["max_leaf"], eu, es))
    assert eu < 1e-4 and es < 1e-3


@pytest.mark.parametrize("N", [1, 2, 65])
def test_fmm_tiny_inputs(N):
    # a handful of particles in a depth-2 tree (most leaves empty): the FMM still equals the
    # direct sum over the same 27 image boxes
    rng = np.random.default_rng(N)
    x = rng.uniform(0, 2 * np.pi, (N, 3))
    g = rng.normal(size=x.shape)
    sigma = 0.3
    uo, so = oracle.direct(x, g, sigma, K=1)
    u, s, _ = run_fmm(x, g, sigma, p=10, depth=2, periodic_levels=0, m2l="bf16x3")
    if N == 1:
        # only the particle's own images: they cancel in pairs, u = S = 0; the FMM leaves its
        # truncation error, measured against the field of the strength at one leaf width
        w = 2 * np.pi / 4
        gm = np.abs(g).max()
        assert np.abs(u).max() < 1e-4 * gm / (4 * np.pi * w ** 2)
        assert np.abs(s).max() < 1e-3 * gm ** 2 / (4 * np.pi * w ** 3)
    else:
        assert rel_l2(u, uo) < 1e-4 and rel_l2(s, so) < 1e-3


def test_eval_host_matches_device_path():
    # the host-memory entry point (copies in, tree, evaluation, copies out) gives the device
    # path's results, twice in a row with new positions (the strength copy overlaps the tree)
    torch = pytest.importorskip("torch")
    import paper_1110_2921_gb300 as vf
    f = wl.make_vortex_lattice(32, 4, 1)
    for it, x in enumerate((f["x"], wl.jitter(f["x"], f["h"], 0.3, seed=4))):
        u_dev, s_dev, _ = run_fmm(x, f["alpha"], f["sigma"], p=10, periodic_levels=2, m2l="bf16x3")
        h = vf.VortexFMM(p=10, periodic_levels=2, m2l="bf16x3")
        try:
            xh = torch.tensor(x, dtype=torch.float32).pin_memory()
            gh = torch.tensor(f["alpha"], dtype=torch.float32).pin_memory()
            u, s = h.eval_host(xh.numpy(), gh.numpy(), f["sigma"])
        finally:
            h.close()
        assert np.array_equal(u.astype(np.float64), u_dev) and np.array_equal(s.astype(np.float64), s_dev)
