"""Turbulence diagnostics of Section 5.2 in plain numpy (FP64): the energy spectrum of a
velocity field sampled on the lattice and the skewness / flatness of the velocity
derivatives.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import numpy as np


def energy_spectrum(u, n, kmax):
    """E(k), k = 0..kmax, of a velocity field u sampled on the n^3 lattice.

    Section 5.2 obtains the spectrum by evaluating the velocity on a lattice with the
    Biot-Savart law and taking a 3-D FFT.  With the Fourier coefficients of the periodic
    box [0, 2 pi)^3, u_hat(k) = n^-3 sum_x u(x) exp(-i k.x) over the lattice points and integer
    wave vectors k, the shell energy is E(k) = sum over |k| in [k - 1/2, k + 1/2) of
    0.5 |u_hat(k)|^2, so that sum_k E(k) = 0.5 <|u|^2> (Parseval) once kmax covers the
    corner of the cube.  u: (n^3, 3) in lattice order (ix n + iy) n + iz.
    """
    U = np.asarray(u, dtype=np.float64).reshape(n, n, n, 3)
    uh = np.fft.fftn(U, axes=(0, 1, 2)) / float(n) ** 3
    k = np.fft.fftfreq(n, 1.0 / n)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    shell = np.floor(np.sqrt(KX * KX + KY * KY + KZ * KZ) + 0.5).astype(np.int64)
    e = 0.5 * (np.abs(uh) ** 2).sum(axis=3)
    keep = shell <= kmax
    return np.bincount(shell[keep].ravel(), weights=e[keep].ravel(), minlength=kmax + 1)[: kmax + 1]


def derivative_moments(grad):
    """Moments of the longitudinal velocity derivatives and F_3, F_4 (Section 5.2).

    F_n = mean(u_x^n) / mean(u_x^2)^(n/2) with u_x = du/dx; an isotropic field gives three
    samples per point, du_a/dx_a for a = x, y, z.  grad: (N, 9) with du_a/dx_k at 3a + k.
    Returns (mean d^2, mean d^3, mean d^4, F_3, F_4).
    """
    g = np.asarray(grad, dtype=np.float64).reshape(-1, 9)
    d = g[:, [0, 4, 8]].ravel()
    m2, m3, m4 = (d ** 2).mean(), (d ** 3).mean(), (d ** 4).mean()
    return m2, m3, m4, m3 / m2 ** 1.5, m4 / m2 ** 2
