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
