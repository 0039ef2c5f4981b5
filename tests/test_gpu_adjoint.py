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


def _handle(**kw):
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    return torch, vf.VortexFMM(**kw)


@pytest.mark.parametrize("n,kw,tol", [
    (16, dict(depth=2, periodic_levels=0, dtype="f64"), 1e-12),
    (16, dict(depth=2, periodic_levels=2, dtype="f64"), 1e-12),
    (32, dict(depth=3, periodic_levels=1, dtype="f64"), 1e-12),
    (32, dict(depth=3, periodic_levels=2, m2l="bf16x3"), 2e-5),
    (32, dict(depth=3, periodic_levels=0, m2l="fp32"), 2e-5),
])
def test_adjoint_fmm_is_the_transpose(n, kw, tol):
    # <w, A gamma> = <A^T w, gamma> for the FMM operator as evaluated (near rings of the
    # gradient path, M2L lists, expansions and lattice operator): the adjoint is its exact
    # transpose, not the FMM applied to w (which differs at the FMM's truncation error)
    f = wl.make_vortex_lattice(n, 4, 1)
    torch, h = _handle(p=10, **kw)
    dt = torch.float64 if kw.get("dtype") == "f64" else torch.float32
    try:
        X = torch.tensor(f["x"], dtype=dt, device="cuda")
        G = torch.tensor(f["alpha"], dtype=dt, device="cuda")
        W = torch.tensor(np.random.default_rng(7).normal(size=(n ** 3, 3)), dtype=dt, device="cuda")
        h.build_tree(X)
        u, _ = h.eval_gradient(G, f["sigma"])
        dg, _ = h.adjoint(G, f["sigma"], W)
        h.sync()
        lhs = float((W.double() * u.double()).sum())
        rhs = float((dg.double() * G.double()).sum())
        # the FMM applied to w, for contrast
        uw, _ = h.eval_gradient(W, f["sigma"])
        rhs_fmm = float((uw.double() * G.double()).sum())
    finally:
        h.close()
    rel = abs(lhs - rhs) / abs(lhs)
    print("n=%d %s: <w,Au> %.15e  <A^T w,g> %.15e  rel %.2e  (FMM on w: rel %.2e)"
          % (n, kw, lhs, rhs, rel, abs(lhs - rhs_fmm) / abs(lhs)))
    assert rel < tol


def _fd_check(n, k0, entries, eps_x, eps_g, tol_x, tol_g, seed=21, grad_u=False, **kw):
    """Central differences of L = sum |u - u*|^2 through the FMM (tree rebuilt at each perturbed
    position; lattice particles stay in their leaves) against vfmm_eval_adjoint, on `entries`
    random entries (alternately of dL/dx and dL/dgamma).  The error of an entry is taken relative
    to the largest magnitude of that gradient (the infinity norm): rounding in L over all N
    particles leaves a noise floor in L(+) - L(-) that is the same for every entry, so an entry
    far smaller than the others has a large error relative to itself alone."""
    f = wl.make_vortex_lattice(n, k0, 1)
    x, g, sigma = f["x"], f["alpha"], f["sigma"]
    ustar = wl.lattice_velocity(n, 6, 2)
    torch, h = _handle(p=10, **kw)
    dt = torch.float64 if kw.get("dtype") == "f64" else torch.float32
    try:
        X = torch.tensor(x, dtype=dt, device="cuda")
        G = torch.tensor(g, dtype=dt, device="cuda")
        Us = torch.tensor(ustar, dtype=torch.float64, device="cuda")

        def velocity(xa, ga):
            h.build_tree(torch.tensor(xa, dtype=dt, device="cuda"))
            Gt = torch.tensor(ga, dtype=dt, device="cuda")
            u = h.eval_gradient(Gt, sigma)[0] if grad_u else h.eval(Gt, sigma, stretching=False)[0]
            return u.double()

        h.build_tree(X)
        u0 = h.eval_gradient(G, sigma)[0] if grad_u else h.eval(G, sigma, stretching=False)[0]
        W = (2.0 * (u0.double() - Us)).to(dt).contiguous()
        dg, dx = h.adjoint(G, sigma, W)
        dg = dg.double().cpu().numpy()
        dx = dx.double().cpu().numpy()
        rng = np.random.default_rng(seed)
        ex, eg = [], []
        for k in range(entries):
            i, a = int(rng.integers(len(x))), int(rng.integers(3))
            wrt_x = k % 2 == 0
            eps = eps_x if wrt_x else eps_g
            base = x if wrt_x else g
            pp, mm = base.copy(), base.copy()
            pp[i, a] += eps
            mm[i, a] -= eps
            up = velocity(pp, g) if wrt_x else velocity(x, pp)
            um = velocity(mm, g) if wrt_x else velocity(x, mm)
            # L(+) - L(-) = sum (u+ - u-) . (u+ + u- - 2 u*), formed without cancellation
            dl = float(((up - um) * (up + um - 2.0 * Us)).sum())
            fd = dl / (2 * eps)
            an = dx[i, a] if wrt_x else dg[i, a]
            gmax = np.abs(dx if wrt_x else dg).max()
            (ex if wrt_x else eg).append(abs(fd - an) / gmax)
            print("  %s[%d,%d]: an %+.10e fd %+.10e |an|/max %.2e err/|an| %.2e err/max %.2e"
                  % ("dx" if wrt_x else "dg", i, a, an, fd, abs(an) / gmax, abs(fd - an) / max(abs(an), 1e-300),
                     abs(fd - an) / gmax))
    finally:
        h.close()
    print("n=%d %s: max FD error / max|grad|: dx %.2e, dgamma %.2e over %d entries"
          % (n, kw, max(ex), max(eg), entries))
    assert max(ex) < tol_x and max(eg) < tol_g, (ex, eg)
    return max(ex), max(eg)


@pytest.mark.parametrize("n,depth,S", [(16, 2, 0), (16, 2, 2), (64, 4, 2)])
def test_adjoint_fmm_fp64_central_differences(n, depth, S):
    # FP64 FMM (p = 10): the adjoint is the gradient of the evaluated sum, so central
    # differences with eps = 1e-6 agree to 1e-6 (of the gradient's largest entry) on 32 random
    # entries (16 of dL/dx, 16 of dL/dgamma), with the tree frozen (lattice particles stay in
    # their leaves).  Measured: at most 3e-9 at 16^3 and 3e-8 at 64^3.
    _fd_check(n, 4, 32, 1e-6, 1e-6, 1e-6, 1e-6, depth=depth, periodic_levels=S, dtype="f64")


@pytest.mark.parametrize("m2l", ["bf16x3", "fp32"])
def test_adjoint_fmm_mixed_central_differences_64cubed(m2l):
    # mixed precision (FP32 P2P and expansions; BF16x3 tensor-core M2L and its transpose, or the
    # FP32 CUDA-core M2L): u is evaluated by the velocity-gradient path (the operator the adjoint
    # transposes).  L is quadratic in gamma, so a large step is exact there and FP32 rounding
    # alone remains (measured <= 1e-5 of max |dL/dgamma|).  In x, FP32 rounding of u at all N
    # particles makes L a staircase at the scale of small steps: with a step of 2e-2 h
    # (truncation ~1e-4) the differences agree to a few 1e-3 of max |dL/dx| (measured 5.3e-3
    # with BF16x3 and 5.4e-3 with the FP32 M2L: FP32 rounding, not the BF16 split, sets it); the
    # FP64 path above carries the 1e-6 check, and the mixed adjoint matches the FP64 one below.
    h64 = 2 * np.pi / 64
    _fd_check(64, 4, 32, 2e-2 * h64, 0.05, 1e-2, 1e-4, grad_u=True, depth=4, periodic_levels=2, m2l=m2l)


def test_adjoint_fmm_mixed_matches_fp64_64cubed():
    # the mixed-precision adjoint against the FP64 one on the same tree and weights
    f = wl.make_vortex_lattice(64, 4, 1)
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    W = np.random.default_rng(9).normal(size=(64 ** 3, 3))
    out = {}
    for name, kw in (("f64", dict(dtype="f64")), ("mixed", dict(m2l="bf16x3"))):
        dt = torch.float64 if name == "f64" else torch.float32
        h = vf.VortexFMM(p=10, depth=4, periodic_levels=2, **kw)
        try:
            h.build_tree(torch.tensor(f["x"], dtype=dt, device="cuda"))
            dg, dx = h.adjoint(torch.tensor(f["alpha"], dtype=dt, device="cuda"), f["sigma"],
                               torch.tensor(W, dtype=dt, device="cuda"))
            out[name] = (dg.double().cpu().numpy(), dx.double().cpu().numpy())
        finally:
            h.close()
    eg = rel_l2(out["mixed"][0], out["f64"][0])
    ex = rel_l2(out["mixed"][1], out["f64"][1])
    print("mixed vs FP64 adjoint at 64^3: dgamma %.2e dx %.2e" % (eg, ex))
    assert eg < 1e-5 and ex < 1e-5
