"""vfmm_direct_eval_noalloc: the direct sum for callers that cannot allocate device memory
when they call in (a program that gives all device memory to its own pool, or a loop that
must not pay cudaMalloc's implicit synchronisation).  Its scratch lives in a static device
array; this test checks it against the FP64 oracle's direct sum over the central 27 boxes and
against the handle-based direct sum (VFMM_METHOD_DIRECT, FP32) on two calls in a row, the
second with a smaller n so stale scratch from the first would show.

The file name sorts last so a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workload as wl
from gpu_util import rel_l2, run_fmm, torch_cuda

pytestmark = pytest.mark.gpu

TOL = 2e-5   # the FP32 direct-sum tolerance of the parity tests


def _noalloc(lib, torch, x, g, sigma, images=1):
    X = torch.tensor(x, dtype=torch.float32, device="cuda").contiguous()
    G = torch.tensor(g, dtype=torch.float32, device="cuda").contiguous()
    U = torch.full_like(G, float("nan"))
    S = torch.full_like(G, float("nan"))
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.vfmm_direct_eval_noalloc(ctypes.c_int64(len(x)), ctypes.c_void_p(X.data_ptr()),
                                      ctypes.c_void_p(G.data_ptr()), ctypes.c_double(sigma),
                                      ctypes.c_double(2 * np.pi), ctypes.c_int(images),
                                      ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                      ctypes.c_void_p(st))
    torch.cuda.synchronize()
    return rc, U.double().cpu().numpy(), S.double().cpu().numpy()


def test_noalloc_direct_matches_oracle_and_handle_direct_twice():
    torch = torch_cuda()
    from paper_1110_2921_gb300 import _native
    lib = _native.lib()
    lib.vfmm_direct_eval_noalloc.restype = ctypes.c_int
    f = wl.make_vortex_lattice(16, 4, 1)
    cases = [(f["x"], f["alpha"]), (f["x"][:1000] + 0.01, f["alpha"][:1000] * 2.0)]
    for x, g in cases:
        rc, u, s = _noalloc(lib, torch, x, g, f["sigma"])
        assert rc == 0
        uo, so = oracle.direct(x, g, f["sigma"], K=1)
        assert rel_l2(u, uo) < TOL
        assert rel_l2(s, so) < TOL
        ur, sr, _ = run_fmm(x, g, f["sigma"], method="direct", direct_images=1, dtype="f32")
        assert rel_l2(u, ur) < TOL
        assert rel_l2(s, sr) < TOL


def test_noalloc_rejects_oversize():
    torch = torch_cuda()
    from paper_1110_2921_gb300 import _native
    lib = _native.lib()
    lib.vfmm_direct_eval_noalloc.restype = ctypes.c_int
    rc = lib.vfmm_direct_eval_noalloc(ctypes.c_int64(65537), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                      ctypes.c_double(0.1), ctypes.c_double(2 * np.pi), ctypes.c_int(1),
                                      ctypes.c_void_p(16), None, None)
    assert rc == _native.VFMM_ERR_UNSUPPORTED
