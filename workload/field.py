"""Random solenoidal Fourier fields on a periodic lattice (input generator only)."""
import numpy as np

TWO_PI = 2.0 * np.pi


def lattice_positions(n, L=TWO_PI):
    """Cell-centre lattice x = (i + 1/2) h, flattened as (ix*n + iy)*n + iz; shape (n^3, 3)."""
    h = L / n
    g = (np.arange(n, dtype=np.float64) + 0.5) * h
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1)
    return X.reshape(-1, 3)


def _kmax(n, k0):
    return int(min(4 * k0, n // 2 - 1))


def solenoidal_modes(n, k0, seed):
    """Return (k, a): integer wave vectors k (M,M,M,3) and complex velocity modes a (M,M,M,3).

    a is divergence-free (k . a = 0), Hermitian (a(-k) = conj a(k)), zero at k = 0,
    with integer-shell energy 0.5*sum|a|^2 following k^4 exp(-2 k^2/k0^2) and
    total 0.5*sum|a|^2 = 1.  Modes live in the cube |k_i| <= kmax = min(4 k0, n/2 - 1),
    so the field is independent of n once n/2 - 1 >= 4 k0.
    """
    km = _kmax(n, k0)
    M = 2 * km + 1
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((M, M, M, 3)) + 1j * rng.standard_normal((M, M, M, 3))
    r = np.arange(-km, km + 1, dtype=np.float64)
    k = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1)
    k2 = (k * k).sum(-1)
    nz = k2 > 0
    kd = (k * a).sum(-1)
    a[nz] -= k[nz] * (kd[nz] / k2[nz])[:, None]
    a[~nz] = 0.0
    # Hermitian symmetry: index of -k is the flipped cube
    a = 0.5 * (a + np.conj(a[::-1, ::-1, ::-1]))
    kmag = np.sqrt(k2)
    shell = np.rint(kmag).astype(np.int64)
    e_mode = 0.5 * (np.abs(a) ** 2).sum(-1)
    smax = int(shell.max())
    e_cur = np.bincount(shell.ravel(), weights=e_mode.ravel(), minlength=smax + 1)
    s = np.arange(smax + 1, dtype=np.float64)
    e_tgt = s ** 4 * np.exp(-2.0 * s ** 2 / float(k0) ** 2)
    scale = np.zeros_like(e_tgt)
    ok = e_cur > 0
    scale[ok] = np.sqrt(e_tgt[ok] / e_cur[ok])
    a *= scale[shell][..., None]
    a[~nz] = 0.0
    a /= np.sqrt(0.5 * (np.abs(a) ** 2).sum())
    return k, a


def _to_lattice(k, coef, n):
    """Evaluate sum_k coef(k) exp(i k.x) at x = (j + 1/2) h (real part), coef (M,M,M,C)."""
    h = TWO_PI / n
    C = coef.shape[-1]
    grid = np.zeros((n, n, n, C), dtype=np.complex128)
    ki = k.astype(np.int64)
    phase = np.exp(1j * (k.sum(-1)) * (0.5 * h))
    idx = tuple(ki[..., d] % n for d in range(3))
    grid[idx] = coef * phase[..., None]
    out = np.empty((n, n, n, C))
    for c in range(C):
        out[..., c] = np.fft.ifftn(grid[..., c]).real * (n ** 3)
    return out.reshape(-1, C)


def lattice_velocity(n, k0, seed):
    """Velocity u of the seeded field at the n^3 lattice particles (N, 3)."""
    k, a = solenoidal_modes(n, k0, seed)
    return _to_lattice(k, a, n)


def make_vortex_lattice(n, k0=4, seed=1, sigma_over_h=1.0, L=TWO_PI):
    """Vortex particles of a seeded random field; dict with x, alpha, sigma, h, L, n, k0, seed."""
    if abs(L - TWO_PI) > 1e-15:
        raise ValueError("the generator is defined on [0, 2*pi)^3")
    k, a = solenoidal_modes(n, k0, seed)
    om = 1j * np.cross(k, a)
    h = L / n
    omega = _to_lattice(k, om, n)
    alpha = omega * h ** 3
    return {"x": lattice_positions(n, L), "alpha": alpha, "sigma": sigma_over_h * h,
            "h": h, "L": L, "n": n, "k0": k0, "seed": seed, "omega": omega}


def viscosity_for_re_lambda(n, k0, seed, re_lambda):
    """nu such that Re_lambda = u' lambda / nu on the discrete spectrum of the field.

    u'^2 = <|u|^2>/3, lambda^2 = 15 u'^2 / (2 sum k^2 E(k)), E per mode 0.5|a|^2.
    """
    k, a = solenoidal_modes(n, k0, seed)
    e_mode = 0.5 * (np.abs(a) ** 2).sum(-1)
    k2 = (k * k).sum(-1)
    u2 = 2.0 * e_mode.sum() / 3.0
    lam = np.sqrt(15.0 * u2 / (2.0 * (k2 * e_mode).sum()))
    return float(np.sqrt(u2) * lam / re_lambda)


def target_subset(N, count, seed=3):
    """Seeded sorted subset of particle indices (int64)."""
    count = min(count, N)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=count, replace=False)).astype(np.int64)


def jitter(x, h, amplitude, seed):
    """Displace positions by a seeded uniform offset of +-amplitude*h per coordinate."""
    rng = np.random.default_rng(seed)
    return x + rng.uniform(-amplitude, amplitude, x.shape) * h
