"""Energy spectrum and velocity-derivative moments on the GPU (Section 5.2) against the
numpy oracle, on the same inputs."""
import numpy as np
import pytest

import oracle
import workload as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _handle(dtype="f32"):
    import paper_1110_2921_gb300 as vf
    return vf.VortexFMM(dtype=dtype)


@pytest.mark.parametrize("n", [8, 32, 64])
def test_spectrum_matches_oracle_fp64(n):
    torch = torch_cuda()
    rng = np.random.default_rng(5)
    u = rng.standard_normal((n ** 3, 3))
    kmax = int(np.ceil(np.sqrt(3) * n / 2)) + 1
    h = _handle("f64")
    try:
        E = np.array(h.energy_spectrum(torch.tensor(u, device="cuda"), n, kmax))
    finally:
        h.close()
    Eo = oracle.diagnostics.energy_spectrum(u, n, kmax)
    assert np.allclose(E, Eo, rtol=1e-11, atol=1e-15 * Eo.sum())
    assert abs(E.sum() - 0.5 * (u ** 2).sum(1).mean()) < 1e-11 * E.sum()


def test_spectrum_of_fmm_velocity_fp32():
    # the lattice velocity of the FMM (particles on the lattice): library spectrum vs the
    # oracle's FFT of the same FP32 values; the low shells follow the prescribed spectrum
    torch = torch_cuda()
    from gpu_util import run_fmm
    n = 32
    f = wl.make_vortex_lattice(n, 4, 1)
    u, _, _ = run_fmm(f["x"], f["alpha"], f["sigma"], p=10, periodic_levels=2, m2l="bf16x3")
    u32 = u.astype(np.float32)
    h = _handle("f32")
    try:
        E = np.array(h.energy_spectrum(torch.tensor(u32, device="cuda"), n, 27))
    finally:
        h.close()
    Eo = oracle.diagnostics.energy_spectrum(u32.astype(np.float64), n, 27)
    assert np.allclose(E, Eo, rtol=1e-10, atol=1e-14)
    Eg = oracle.diagnostics.energy_spectrum(wl.lattice_velocity(n, 4, 1), n, 27)
    # Gaussian cores (Eq. cutoff) filter the field by exp(-k^2 sigma^2 / 2) in amplitude, so
    # the energy of shell k drops by about exp(-k^2 sigma^2) (shell-averaged k^2: a few %)
    k = np.arange(1, 5)
    assert np.all(np.abs(E[1:5] / Eg[1:5] / np.exp(-(k * f["sigma"]) ** 2) - 1.0) < 0.06)


def test_derivative_moments_match_oracle():
    torch = torch_cuda()
    rng = np.random.default_rng(9)
    g = rng.standard_normal((200_003, 9)) * np.array([1, 0, 0, 0, 2, 0, 0, 0, 3.0]) + 0.1
    for dt, tol in (("f64", 1e-12), ("f32", 1e-6)):
        h = _handle(dt)
        try:
            tdt = torch.float64 if dt == "f64" else torch.float32
            gg = g.astype(np.float64 if dt == "f64" else np.float32)
            out = np.array(h.derivative_moments(torch.tensor(gg, dtype=tdt, device="cuda")))
        finally:
            h.close()
        ref = np.array(oracle.diagnostics.derivative_moments(gg.astype(np.float64)))
        assert np.allclose(out, ref, rtol=tol)


def test_skewness_of_fmm_gradient_on_the_generated_field():
    # the FMM velocity gradient of the seeded field: library moments vs the oracle's moments
    # of the same gradient; a Gaussian random field has F3 ~ 0 and F4 ~ 3
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    n = 32
    f = wl.make_vortex_lattice(n, 4, 1)
    h = vf.VortexFMM(p=10, periodic_levels=2, m2l="bf16x3")
    try:
        X = torch.tensor(f["x"], dtype=torch.float32, device="cuda")
        G = torch.tensor(f["alpha"], dtype=torch.float32, device="cuda")
        h.build_tree(X)
        _, grad = h.eval_gradient(G, f["sigma"])
        grad = grad.reshape(-1, 9)
        out = np.array(h.derivative_moments(grad))
        ref = np.array(oracle.diagnostics.derivative_moments(grad.double().cpu().numpy()))
    finally:
        h.close()
    assert np.allclose(out, ref, rtol=1e-5)
    assert abs(out[3]) < 0.3 and abs(out[4] - 3.0) < 0.6
