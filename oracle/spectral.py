"""Fully periodic regularised Biot-Savart field as a Fourier series (FP64 numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With Gaussian cores the periodic vorticity of Eq. (smoothingfunction),
omega(x) = sum_j gamma_j zeta_sigma(x - x_j) summed over all periodic copies, has the
absolutely convergent series
    omega_hat(k) = L^-3 sum_j gamma_j exp(-i k.x_j) exp(-|k|^2 sigma^2 / 2),  k in (2 pi/L) Z^3,
and the velocity solving Eq. (velocitypoisson) with zero mean is
    u_hat(k) = i k x omega_hat(k) / |k|^2   (k != 0),
so S = (gamma_i . grad) u is sum_k i (k . gamma_i) u_hat(k) exp(i k.x_i).

This is the infinite-lattice limit of the cube-of-images sum; the two differ by a
uniform velocity (the cube sum of the vortex dipole field is only conditionally
convergent) and by a tail that vanishes as the cube grows.  The stretching term has
no such uniform offset.
"""
import numpy as np

_E_CUT = 40.0  # modes with exp(-|k|^2 sigma^2/2) < e^-40 are dropped


def direct_series(x, gamma, sigma, xt=None, gt=None, L=2 * np.pi):
    """Evaluate the series by direct summation over modes (any positions; small N)."""
    x = np.asarray(x, float)
    g = np.asarray(gamma, float)
    if xt is None:
        xt, gt = x, g
    xt = np.asarray(xt, float)
    gt = np.asarray(gt, float)
    k1 = 2 * np.pi / L
    kc = np.sqrt(2 * _E_CUT) / sigma
    m = int(np.ceil(kc / k1))
    r = np.arange(-m, m + 1)
    # per-axis phase tables: exp(-i k_a x_a)
    Ex = np.exp(-1j * k1 * np.outer(x[:, 0], r))
    Ey = np.exp(-1j * k1 * np.outer(x[:, 1], r))
    Ez = np.exp(-1j * k1 * np.outer(x[:, 2], r))
    kk = k1 * r
    u = np.zeros((len(xt), 3))
    S = np.zeros((len(xt), 3))
    Tx = np.exp(1j * k1 * np.outer(xt[:, 0], r))
    Ty = np.exp(1j * k1 * np.outer(xt[:, 1], r))
    Tz = np.exp(1j * k1 * np.outer(xt[:, 2], r))
    for ia in range(len(r)):
        kx = kk[ia]
        A = g * Ex[:, ia:ia + 1]                                    # (N,3)
        B = np.einsum('jc,jb->bjc', A, Ey)                          # (ny,N,3)
        P = np.einsum('bjc,jz->bzc', B, Ez) / L ** 3                # (ny,nz,3)
        KY, KZ = np.meshgrid(kk, kk, indexing='ij')
        k2 = kx * kx + KY ** 2 + KZ ** 2
        damp = np.exp(-0.5 * k2 * sigma ** 2)
        keep = (0.5 * k2 * sigma ** 2 <= _E_CUT) & (k2 > 0)
        w = np.where(keep, damp / np.where(k2 > 0, k2, 1.0), 0.0)
        kv = np.stack([np.full_like(KY, kx), KY, KZ], -1)            # (ny,nz,3)
        uh = 1j * np.cross(kv, P) * w[..., None]                     # (ny,nz,3)
        # evaluate at targets
        ph = Tx[:, ia][:, None, None] * Ty[:, :, None] * Tz[:, None, :]   # (nt,ny,nz)
        u += np.einsum('tyz,yzc->tc', ph, uh).real
        kg = np.einsum('yzc,tc->tyz', kv, gt)
        S += np.einsum('tyz,yzc->tc', 1j * kg * ph, uh).real
    return u, S


def lattice(n, gamma, sigma, L=2 * np.pi):
    """Evaluate the series at the n^3 cell-centre lattice x = (j + 1/2) h (any n, by FFT).

    gamma is (n^3, 3) in lattice order (ix*n + iy)*n + iz.  For lattice sources the
    structure factor is n-periodic in k up to the sign (-1)^(m_x+m_y+m_z), which cancels
    against the same sign of the target phase, so every alias k + n m folds into the
    FFT bin k with weight sum_m (k + n m) g(k + n m), g(k) = exp(-|k|^2 sigma^2/2)/|k|^2.
    """
    if abs(L - 2 * np.pi) > 1e-15:
        raise ValueError("lattice series assumes L = 2 pi")
    h = L / n
    G = np.asarray(gamma, float).reshape(n, n, n, 3)
    f = np.fft.fftfreq(n, d=1.0 / n)                 # integer wave numbers
    kc = np.sqrt(2 * _E_CUT) / sigma
    mmax = int(np.ceil(kc / n + 0.5))
    half = np.exp(-1j * f * 0.5 * h)
    ph = half[:, None, None] * half[None, :, None] * half[None, None, :]
    Pk = np.stack([np.fft.fftn(G[..., c]) for c in range(3)], -1) * ph[..., None] / L ** 3
    u = np.zeros((n, n, n, 3))
    Sa = np.zeros((n, n, n, 3, 3))                    # Sa[..., a, :] multiplies gamma_a
    KX, KY, KZ = np.meshgrid(f, f, f, indexing='ij')
    V = np.zeros((n, n, n, 3))
    W = np.zeros((n, n, n, 3, 3))
    for mx in range(-mmax, mmax + 1):
        for my in range(-mmax, mmax + 1):
            for mz in range(-mmax, mmax + 1):
                kx = KX + n * mx
                ky = KY + n * my
                kz = KZ + n * mz
                k2 = kx * kx + ky * ky + kz * kz
                e = 0.5 * k2 * sigma ** 2
                if e.min() > _E_CUT:
                    continue
                w = np.where((k2 > 0) & (e <= _E_CUT), np.exp(-e) / np.where(k2 > 0, k2, 1.0), 0.0)
                kv = np.stack([kx, ky, kz], -1)
                V += kv * w[..., None]
                W += kv[..., :, None] * kv[..., None, :] * w[..., None, None]
    inv = lambda A: np.fft.ifftn(A * np.conj(ph)).real * n ** 3
    uh = 1j * np.cross(V, Pk)
    for c in range(3):
        u[..., c] = inv(uh[..., c])
    for a in range(3):
        sh = -np.cross(W[..., a, :], Pk)
        for c in range(3):
            Sa[..., a, c] = inv(sh[..., c])
    S = np.einsum('xyza,xyzac->xyzc', G, Sa)
    return u.reshape(-1, 3), S.reshape(-1, 3)
