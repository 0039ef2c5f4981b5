"""Adjoint (dL/dgamma, dL/dx for L = sum |u - u*|^2) through vfmm_eval_adjoint and the
torch.autograd.Function, against the FP64 gradient oracle and central differences."""
import numpy as np
import pytest

import oracle
import workload as wl
from gpu_util import rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _grads(x, g, sigma, ustar, **kw):
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    dt = torch.float64 if kw.get("dtype", "f32") == "f64" else torch.float32
    X = torch.tensor(x, dtype=dt, device="cuda", requires_grad=True)
    G = torch.tensor(g, dtype=dt, device="cuda", requires_grad=True)
    U = torch.tensor(ustar, dtype=dt, device="cuda")
    h = vf.VortexFMM(**kw)
    try:
        u, s = vf.biot_savart(X, G, h, sigma)
        loss = ((u - U) ** 2).sum()
        loss.backward()
        return (G.grad.double().cpu().numpy(), X.grad.double().cpu().numpy(), u.detach().double().cpu().numpy())
    finally:
        h.close()


@pytest.fixture(scope="module")
def case16():
    f = wl.make_vortex_lattice(16, 4, 1)
    ustar = wl.lattice_velocity(16, 6, 2)
    dg, dx, _ = oracle.gradient.loss_gradient(f["x"], f["alpha"], f["sigma"], ustar, K=1)
    return f, ustar, dg, dx


def test_adjoint_direct_fp64_matches_oracle(case16):
    f, ustar, dgo, dxo = case16
    dg, dx, _ = _grads(f["x"], f["alpha"], f["sigma"], ustar, method="direct", direct_images=1, dtype="f64")
    assert rel_l2(dg, dgo) < 1e-11
    assert rel_l2(dx, dxo) < 1e-11


def test_adjoint_fmm_fp64_matches_oracle(case16):
    f, ustar, dgo, dxo = case16
    dg, dx, _ = _grads(f["x"], f["alpha"], f["sigma"], ustar, method="fmm", p=10, depth=2, periodic_levels=0,
                       dtype="f64")
    assert rel_l2(dg, dgo) < 1e-4
    assert rel_l2(dx, dxo) < 1e-3


def test_adjoint_direct_fp64_central_differences():
    # the exact gradient of the evaluated sum: FD with eps = 1e-6 on 32 random entries
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    n = 8
    f = wl.make_vortex_lattice(n, 2, 3)
    x, g, sigma = f["x"], f["alpha"], f["sigma"]
    x = wl.jitter(x, f["h"], 0.2, seed=4)
    ustar = wl.lattice_velocity(n, 2, 2) * 0.5
    dg, dx, _ = _grads(x, g, sigma, ustar, method="direct", direct_images=1, dtype="f64")
    h = vf.VortexFMM(method="direct", direct_images=1, dtype="f64")
    U = torch.tensor(ustar, dtype=torch.float64, device="cuda")

    def loss(xa, ga):
        X = torch.tensor(xa, dtype=torch.float64, device="cuda")
        G = torch.tensor(ga, dtype=torch.float64, device="cuda")
        h.build_tree(X)
        u, _ = h.eval(G, sigma)
        return float(((u - U) ** 2).sum().item())

    rng = np.random.default_rng(21)
    eps = 1e-6
    errs = []
    try:
        for k in range(32):
            i, a = int(rng.integers(len(x))), int(rng.integers(3))
            wrt_x = k % 2 == 0
            base = x if wrt_x else g
            p, m = base.copy(), base.copy()
            p[i, a] += eps
            m[i, a] -= eps
            fd = (loss(p, g) - loss(m, g)) / (2 * eps) if wrt_x else (loss(x, p) - loss(x, m)) / (2 * eps)
            an = dx[i, a] if wrt_x else dg[i, a]
            errs.append(abs(fd - an) / max(abs(an), 1e-3 * np.abs(dx if wrt_x else dg).max()))
    finally:
        h.close()
    assert max(errs) < 1e-6, max(errs)


@pytest.mark.parametrize("m2l", ["bf16x3", "fp32"])
def test_adjoint_mixed_64cubed_sampled(m2l):
    # 64^3, target field of a second spectrum (k0 = 6); the oracle gradient at sampled
    # particles with the same weights w = 2 (u - u*)
    f = wl.make_vortex_lattice(64, 8, 1)
    ustar = wl.lattice_velocity(64, 6, 2)
    dg, dx, u = _grads(f["x"], f["alpha"], f["sigma"], ustar, method="fmm", p=10, periodic_levels=0, m2l=m2l)
    w = 2.0 * (u - ustar)
    tid = wl.target_subset(64 ** 3, 64, seed=3)
    dgo, dxo, _ = oracle.gradient.loss_gradient(f["x"], f["alpha"], f["sigma"], ustar, K=1, targets=tid, w=w)
    assert rel_l2(dg[tid], dgo) < 1e-4
    assert rel_l2(dx[tid], dxo) < 1e-3
