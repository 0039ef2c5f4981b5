"""vfmm_rk_step (Heun step of Eqs. convection, stretching, csm) and vfmm_diagnostics against
the oracle's Heun step and FP64 sums."""
import math

import numpy as np
import pytest

import oracle
import workload as wl
from gpu_util import rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _step(x, g, sigma, dt, nu, nsteps=1, **kw):
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    dt_ = torch.float64 if kw.get("dtype", "f32") == "f64" else torch.float32
    X = torch.tensor(x, dtype=dt_, device="cuda")
    G = torch.tensor(g, dtype=dt_, device="cuda")
    h = vf.VortexFMM(**kw)
    try:
        s = sigma
        for _ in range(nsteps):
            s = h.rk_step(X, G, s, dt, nu)
        h.sync()
        return X.double().cpu().numpy(), G.double().cpu().numpy(), s
    finally:
        h.close()


def _wrapdiff(a, b):
    return np.mod(a - b + np.pi, 2 * np.pi) - np.pi


def test_rk_step_direct_fp64_matches_oracle():
    n = 6
    h = 2 * np.pi / n
    x = wl.jitter(wl.lattice_positions(n), h, 0.3, seed=41)
    g = np.random.default_rng(42).normal(size=x.shape) * h ** 3
    sigma, dt, nu = h, 0.05, 0.02
    xo, go, so = oracle.integrate.heun_step(x, g, sigma, dt, nu, K=1)
    xg, gg, sg = _step(x, g, sigma, dt, nu, method="direct", direct_images=1, dtype="f64")
    assert abs(sg - so) < 1e-15
    assert np.abs(_wrapdiff(xg, xo)).max() < 1e-12
    assert rel_l2(gg - g, go - g) < 1e-10


def test_rk_step_fmm_16cubed_matches_oracle():
    f = wl.make_vortex_lattice(16, 4, 1)
    x, g, sigma = f["x"], f["alpha"], f["sigma"]
    dt, nu = 0.01, 4.0e-3
    xo, go, so = oracle.integrate.heun_step(x, g, sigma, dt, nu, K=1)
    for kw in (dict(dtype="f64"), dict(dtype="f32", m2l="fp32")):
        xg, gg, sg = _step(x, g, sigma, dt, nu, method="fmm", p=10, depth=2, periodic_levels=0, **kw)
        assert abs(sg - so) < 1e-12
        # the increments are dt*u and dt*S to FMM accuracy
        assert rel_l2(_wrapdiff(xg, x), _wrapdiff(xo, x)) < 1e-4
        assert rel_l2(gg - g, go - g) < 1e-3


def test_ten_steps_64cubed_mixed():
    # ten RK2 steps with core spreading on a 64^3 field (mixed precision): sigma follows
    # sqrt(sigma0^2 + 2 nu t) exactly and the fields stay finite
    f = wl.make_vortex_lattice(64, 4, 1)
    nu = wl.viscosity_for_re_lambda(64, 4, 1, 100.0)
    x, g, s = _step(f["x"], f["alpha"], f["sigma"], 0.01, nu, nsteps=10, method="fmm", p=10, m2l="bf16x3")
    assert abs(s - math.sqrt(f["sigma"] ** 2 + 2 * nu * 0.1)) < 1e-12
    assert np.isfinite(x).all() and np.isfinite(g).all()
    assert (x >= 0).all() and (x < 2 * np.pi).all()


def test_diagnostics_match_numpy():
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    f = wl.make_vortex_lattice(16, 4, 1)
    u = wl.lattice_velocity(16, 4, 1)
    h = vf.VortexFMM(m2l="fp32")
    try:
        X = torch.tensor(f["x"], dtype=torch.float32, device="cuda")
        G = torch.tensor(f["alpha"], dtype=torch.float32, device="cuda")
        U = torch.tensor(u, dtype=torch.float32, device="cuda")
        d = h.diagnostics(X, G, U)
    finally:
        h.close()
    ref = oracle.integrate.diagnostics(X.double().cpu().numpy(), G.double().cpu().numpy(), U.double().cpu().numpy())
    got = np.concatenate([d["total_vorticity"], d["x_cross_gamma"], [d["sum_u2"]], [d["sum_gamma2"]]])
    scale = np.abs(f["alpha"]).sum() * 2 * np.pi
    assert np.abs(got[:6] - ref[:6]).max() < 1e-12 * scale
    assert abs(got[6] - ref[6]) < 1e-12 * ref[6] and abs(got[7] - ref[7]) < 1e-12 * ref[7]
