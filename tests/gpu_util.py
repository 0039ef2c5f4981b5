"""Helpers for the GPU parity tests (device handles, error norms)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_2921_gb300 import build
    build.build()
    return torch


def run_fmm(x, g, sigma, **kw):
    """Evaluate through the C-ABI on cuda:0; returns numpy (u, S) and the handle info."""
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    dt = torch.float64 if kw.get("dtype", "f32") == "f64" else torch.float32
    X = torch.tensor(np.asarray(x), dtype=dt, device="cuda").contiguous()
    G = torch.tensor(np.asarray(g), dtype=dt, device="cuda").contiguous()
    h = vf.VortexFMM(**kw)
    try:
        h.build_tree(X)
        u, s = h.eval(G, sigma)
        h.sync()
        info = h.tree_info()
        return u.double().cpu().numpy(), s.double().cpu().numpy(), info
    finally:
        h.close()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_l2_demeaned(a, b):
    d = a - b
    d = d - d.mean(0)
    return float(np.linalg.norm(d) / np.linalg.norm(b - b.mean(0)))
