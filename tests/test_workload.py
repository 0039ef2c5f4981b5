"""Properties of the seeded input generator (Section 4.2, Eq. initspec)."""
import numpy as np

import workload as wl


def test_lattice_layout():
    x = wl.lattice_positions(4)
    h = 2 * np.pi / 4
    assert x.shape == (64, 3)
    assert np.allclose(x[0], [h / 2] * 3)
    assert np.allclose(x[1], [h / 2, h / 2, 1.5 * h])      # iz fastest
    assert np.allclose(x[4], [h / 2, 1.5 * h, h / 2])


def test_field_is_solenoidal_hermitian_unit_energy():
    k, a = wl.solenoidal_modes(32, 4, 1)
    assert np.abs((k * a).sum(-1)).max() < 1e-12
    assert np.allclose(a, np.conj(a[::-1, ::-1, ::-1]))
    assert abs(0.5 * (np.abs(a) ** 2).sum() - 1.0) < 1e-12
    u = wl.lattice_velocity(32, 4, 1)
    assert abs(0.5 * (u ** 2).sum(1).mean() - 1.0) < 1e-12


def test_shell_spectrum_shape():
    k0 = 4
    k, a = wl.solenoidal_modes(64, k0, 2)
    shell = np.rint(np.sqrt((k * k).sum(-1))).astype(int)
    e = np.bincount(shell.ravel(), weights=0.5 * (np.abs(a) ** 2).sum(-1).ravel())
    s = np.arange(len(e), dtype=float)
    tgt = s ** 4 * np.exp(-2 * s ** 2 / k0 ** 2)
    ok = (s >= 1) & (s <= 12)
    ratio = e[ok] / tgt[ok]
    assert np.allclose(ratio, ratio[0], rtol=1e-10)


def test_vorticity_is_curl_and_zero_mean_strength():
    f = wl.make_vortex_lattice(16, 4, 1)
    n, h = 16, f["h"]
    assert abs(f["sigma"] - h) < 1e-15
    assert np.abs(f["alpha"].sum(0)).max() < 1e-13 * np.abs(f["alpha"]).sum()
    # the curl of the lattice velocity by spectral differentiation equals omega
    u = wl.lattice_velocity(16, 4, 1).reshape(n, n, n, 3)
    kf = np.fft.fftfreq(n, 1.0 / n)
    K = np.stack(np.meshgrid(kf, kf, kf, indexing="ij"), -1)
    uh = np.stack([np.fft.fftn(u[..., c]) for c in range(3)], -1)
    wh = 1j * np.cross(K, uh)
    w = np.stack([np.fft.ifftn(wh[..., c]).real for c in range(3)], -1).reshape(-1, 3)
    assert np.allclose(w, f["omega"], atol=1e-10 * np.abs(w).max())


def test_field_independent_of_resolution():
    # modes live in |k_i| <= 4 k0, so two lattices sample one continuous field
    u16 = wl.lattice_velocity(16, 1, 5).reshape(16, 16, 16, 3)
    u32 = wl.lattice_velocity(32, 1, 5).reshape(32, 32, 32, 3)
    # the 16-lattice centre (i+1/2)h16 = (2i+1) h32 is not a 32-lattice centre; compare
    # by interpolating spectrally: the field is band-limited so the mean square agrees
    assert abs((u16 ** 2).mean() - (u32 ** 2).mean()) < 1e-12


def test_viscosity_for_re_lambda():
    nu = wl.viscosity_for_re_lambda(256, 4, 1, 100.0)
    assert 3.5e-3 < nu < 4.5e-3
