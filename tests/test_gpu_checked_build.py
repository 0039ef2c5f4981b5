"""The range-checked build (-DVFMM_CHECK=1): every gather index of the GEMM (M2M, L2L, CUDA-core
M2L), of the tensor-core M2L (source rows, translation tiles) and of the P2P (source leaves) is
checked on the device, an out-of-range index would set the bounds bit (VFMM_ERR_BOUNDS at
vfmm_sync).  Valid inputs raise no bit, and the checked library computes what the default one
computes."""
import ctypes

import numpy as np
import pytest

import workload as wl
from gpu_util import run_fmm, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,depth", [(32, 3), (128, 5)])
def test_checked_build_valid_input_raises_no_bound_bit(n, depth):
    torch = torch_cuda()
    from paper_1110_2921_gb300 import build
    from paper_1110_2921_gb300 import _native as nv
    lib = ctypes.CDLL(build.build(checked=True))
    H = ctypes.c_void_p
    lib.vfmm_create.argtypes = [ctypes.POINTER(nv.vfmm_config), ctypes.POINTER(H)]
    lib.vfmm_build_tree.argtypes = [H, ctypes.c_int64, ctypes.c_void_p]
    lib.vfmm_eval_velocity_stretching.argtypes = [H, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                                  ctypes.c_void_p]
    lib.vfmm_sync.argtypes = [H]
    lib.vfmm_destroy.argtypes = [H]
    f = wl.make_vortex_lattice(n, 4, 1)
    cfg = nv.config_default()
    cfg.p, cfg.depth, cfg.periodic_levels = 10, depth, 2
    cfg.m2l_prec = nv.VFMM_M2L_BF16X3
    cfg.stream = torch.cuda.current_stream().cuda_stream
    X = torch.tensor(f["x"], dtype=torch.float32, device="cuda")
    G = torch.tensor(f["alpha"], dtype=torch.float32, device="cuda")
    U = torch.empty_like(G)
    S = torch.empty_like(G)
    h = H()
    assert lib.vfmm_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    try:
        assert lib.vfmm_build_tree(h, n ** 3, X.data_ptr()) == 0
        assert lib.vfmm_eval_velocity_stretching(h, G.data_ptr(), f["sigma"], U.data_ptr(), S.data_ptr()) == 0
        assert lib.vfmm_sync(h) == 0      # VFMM_ERR_BOUNDS (-5) if any index was out of range
    finally:
        lib.vfmm_destroy(h)
    u, s, _ = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, depth=depth, periodic_levels=2, m2l="bf16x3")
    assert np.allclose(U.double().cpu().numpy(), u, rtol=1e-6, atol=1e-6 * np.abs(u).max())
    assert np.allclose(S.double().cpu().numpy(), s, rtol=1e-6, atol=1e-6 * np.abs(s).max())


@pytest.mark.parametrize("jitter", [0.0, 0.35])
def test_checked_build_pair_count_matches_bench_accounting(jitter):
    # the checked library counts, on the device, the source-target pairs of real targets its
    # FP32 near-field kernel computes; the benchmark's roofline divides by the same number
    # counted on the host (bench.p2p_work: the near ring in full, ring-2 octants within
    # rho_cut sigma of each half of a warp's targets).  They agree exactly, on the lattice and
    # off it (32^3, depth 3: one near ring and the ring-2 correction)
    import math
    import os
    import sys
    torch = torch_cuda()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1110_2921_gb300 import build
    from paper_1110_2921_gb300 import _native as nv
    lib = ctypes.CDLL(build.build(checked=True))
    H = ctypes.c_void_p
    lib.vfmm_create.argtypes = [ctypes.POINTER(nv.vfmm_config), ctypes.POINTER(H)]
    lib.vfmm_build_tree.argtypes = [H, ctypes.c_int64, ctypes.c_void_p]
    lib.vfmm_eval_velocity_stretching.argtypes = [H, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                                  ctypes.c_void_p]
    lib.vfmm_get_tree_info.argtypes = [H, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    lib.vfmm_sync.argtypes = [H]
    lib.vfmm_destroy.argtypes = [H]
    n = 32
    f = wl.make_vortex_lattice(n, 4, 1)
    h_lat = 2 * math.pi / n
    x = wl.jitter(f["x"], h_lat, jitter, seed=11) if jitter > 0 else f["x"]
    cfg = nv.config_default()
    cfg.p, cfg.depth, cfg.periodic_levels = 10, 3, 2
    cfg.m2l_prec = nv.VFMM_M2L_BF16X3
    cfg.stream = torch.cuda.current_stream().cuda_stream
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    G = torch.tensor(f["alpha"], dtype=torch.float32, device="cuda")
    U = torch.empty_like(G)
    S = torch.empty_like(G)
    h = H()
    assert lib.vfmm_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    try:
        assert lib.vfmm_build_tree(h, n ** 3, X.data_ptr()) == 0
        assert lib.vfmm_eval_velocity_stretching(h, G.data_ptr(), f["sigma"], U.data_ptr(), S.data_ptr()) == 0
        assert lib.vfmm_sync(h) == 0
        out = (ctypes.c_int64 * 8)()
        assert lib.vfmm_get_tree_info(h, out, 8) == 0
    finally:
        lib.vfmm_destroy(h)
    depth, R, Rc, pairs_dev = out[0], out[1], out[6], out[7]
    assert (depth, R, Rc) == (3, 1, 2)
    pairs_host, _ = bench.p2p_work(x, 2 * math.pi, depth, R, f["sigma"], Rc, 5.0)
    print("pairs: device %d host %d" % (pairs_dev, pairs_host))
    assert pairs_dev == int(pairs_host)
