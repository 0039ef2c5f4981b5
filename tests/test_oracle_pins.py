"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test targets one plausible mistake: a wrong normalisation of q (Eq. cutoff), a
wrong sign or operand order in the cross products (Eq. biotsavart), a dropped or
mis-signed term in F (Eq. stretching), a wrong image lattice (Section 4.1).
"""
import itertools
import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf

import oracle
import workload as wl

FOUR_PI = 4.0 * np.pi


def test_q_matches_enclosed_gaussian_fraction():
    # q(rho) is the fraction of a 3-D Gaussian inside radius rho (Eq. cutoff derivation)
    for rho in [1e-3, 0.05, 0.3, 0.4999, 0.5, 0.5001, 1.0, 2.0, 3.7, 6.0, 8.0]:
        val, _ = integrate.quad(lambda s: s * s * np.exp(-0.5 * s * s), 0.0, rho,
                                epsabs=0, epsrel=1e-13, limit=200)
        ref = np.sqrt(2.0 / np.pi) * val
        assert abs(oracle.cutoff_q(rho) - ref) <= 2e-13 * ref + 1e-17, rho


def test_q_limits():
    assert oracle.cutoff_q(9.0) == 1.0          # 1 - q(9) < half an ulp of 1
    assert abs(oracle.cutoff_q(8.0) - 1.0) < 1e-13
    rho = 1e-4                                   # leading term sqrt(2/pi) rho^3 / 3
    assert abs(oracle.cutoff_q(rho) / (np.sqrt(2 / np.pi) * rho ** 3 / 3) - 1) < 1e-8


def _blob_psi(x, gamma, sigma):
    """Stream function of one Gaussian vortex blob at the origin: gamma erf(r/(sqrt2 s))/(4 pi r)."""
    r = np.linalg.norm(x)
    return gamma * erf(r / (np.sqrt(2) * sigma)) / (FOUR_PI * r)


def _curl_fd(f, x, eps):
    J = np.zeros((3, 3))   # J[c, k] = d f_c / d x_k
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        J[:, k] = (f(x + e) - f(x - e)) / (2 * eps)
    return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])


@pytest.mark.parametrize("sigma", [0.3, 1.0])
def test_single_blob_closed_form(sigma):
    # velocity of a single Gaussian blob = curl of its closed-form stream function
    rng = np.random.default_rng(11)
    g0 = np.array([0.3, -1.1, 0.7])
    src = np.zeros((1, 3))
    pts = rng.normal(size=(12, 3)) * sigma * np.array([[0.2], [0.5], [1], [1.5], [2], [3],
                                                       [4], [6], [0.8], [1.2], [2.5], [5]])
    u, _ = oracle.direct(src, g0[None], sigma, K=0, xt=pts)
    for i, x in enumerate(pts):
        ref = _curl_fd(lambda y: _blob_psi(y, g0, sigma), x, 1e-5 * sigma)
        assert np.allclose(u[i], ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max()), (i, u[i], ref)


def test_singular_far_limit_and_laplace_identity():
    # for rho >= 9 every q is exactly 1: u is the textbook singular Biot-Savart sum and
    # equals the curl of the Laplace vector potential sum gamma_j/(4 pi r)
    rng = np.random.default_rng(5)
    xs = rng.uniform(0, 1, (20, 3))
    gs = rng.normal(size=(20, 3))
    xt = rng.uniform(0, 1, (7, 3)) + np.array([3.0, 0, 0])
    sigma = 0.2   # min distance > 2 -> rho > 10
    u, S = oracle.direct(xs, gs, sigma, K=0, xt=xt, gt=np.ones_like(xt))
    for i in range(len(xt)):
        psi = lambda y: (gs / (FOUR_PI * np.linalg.norm(y - xs, axis=1))[:, None]).sum(0)
        ref = _curl_fd(psi, xt[i], 1e-5)
        assert np.allclose(u[i], ref, rtol=1e-8), (u[i], ref)


def _mp_sum(xs, gs, xt, gt, tidx, sigma, L, K):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    out_u, out_S = [], []
    s = mp.mpf(sigma)
    for i in range(len(xt)):
        u = [mp.mpf(0)] * 3
        S = [mp.mpf(0)] * 3
        xi = [mp.mpf(v) for v in xt[i]]
        gi = [mp.mpf(v) for v in gt[i]]
        for nx in range(-K, K + 1):
            for ny in range(-K, K + 1):
                for nz in range(-K, K + 1):
                    for j in range(len(xs)):
                        if nx == ny == nz == 0 and tidx[i] == j:
                            continue
                        r = [xi[0] - mp.mpf(xs[j][0]) - nx * mp.mpf(L),
                             xi[1] - mp.mpf(xs[j][1]) - ny * mp.mpf(L),
                             xi[2] - mp.mpf(xs[j][2]) - nz * mp.mpf(L)]
                        r2 = r[0] ** 2 + r[1] ** 2 + r[2] ** 2
                        rr = mp.sqrt(r2)
                        rho = rr / s
                        # q as the integral of the Gaussian shell density
                        q = mp.sqrt(2 / mp.pi) * mp.quad(lambda t: t * t * mp.exp(-t * t / 2), [0, rho])
                        Kk = q / (4 * mp.pi * rr ** 3)
                        # F = K'(r)/r by mpmath differentiation of K(r)
                        Kf = lambda R: (mp.sqrt(2 / mp.pi) * mp.quad(lambda t: t * t * mp.exp(-t * t / 2),
                                                                     [0, R / s])) / (4 * mp.pi * R ** 3)
                        F = mp.diff(Kf, rr) / rr
                        g = [mp.mpf(v) for v in gs[j]]
                        W = [g[1] * r[2] - g[2] * r[1], g[2] * r[0] - g[0] * r[2], g[0] * r[1] - g[1] * r[0]]
                        X = [g[1] * gi[2] - g[2] * gi[1], g[2] * gi[0] - g[0] * gi[2], g[0] * gi[1] - g[1] * gi[0]]
                        gr = gi[0] * r[0] + gi[1] * r[1] + gi[2] * r[2]
                        for a in range(3):
                            u[a] += Kk * W[a]
                            S[a] += Kk * X[a] + F * gr * W[a]
        out_u.append([float(v) for v in u])
        out_S.append([float(v) for v in S])
    return np.array(out_u), np.array(out_S)


@pytest.mark.slow
def test_bruteforce_mpmath_small():
    # N = 8 jittered lattice with one image layer, three targets, 40-digit arithmetic;
    # q and F come from numerical integration/differentiation, not from the erf formula
    L = 2 * np.pi
    n = 2
    h = L / n
    x = wl.jitter(wl.lattice_positions(n), h, 0.3, seed=4)
    g = np.random.default_rng(8).normal(size=x.shape)
    sigma = 0.8 * h
    tid = np.array([0, 3, 6])
    u, S = oracle.direct(x, g, sigma, K=1, targets=tid)
    um, Sm = _mp_sum(x, g, x[tid], g[tid], tid, sigma, L, 1)
    assert np.allclose(u, um, rtol=1e-12, atol=1e-14 * np.abs(um).max())
    assert np.allclose(S, Sm, rtol=1e-11, atol=1e-13 * np.abs(Sm).max())


def _cluster(sigma, seed):
    """Six sources whose pair distances fall between 0.05 sigma and 0.45 sigma (the series
    branch of K and F, rho < 0.5), with random strengths."""
    rng = np.random.default_rng(seed)
    c = np.array([1.1, 2.3, 0.7])
    d = rng.normal(size=(6, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    x = c + d * (np.array([0.0, 0.03, 0.08, 0.12, 0.17, 0.21])[:, None] * sigma)
    g = rng.normal(size=(6, 3))
    return x, g


@pytest.mark.slow
def test_bruteforce_mpmath_series_branch():
    # the same 40-digit brute force on a cluster where every pair sits at rho < 0.5: the
    # series of k = q/rho^3 and f = k'/rho (Eqs. cutoff, stretching) against quadrature and
    # numerical differentiation in mpmath
    sigma = 0.6
    x, g = _cluster(sigma, 17)
    tid = np.arange(6)
    r = np.linalg.norm(x[:, None] - x[None], axis=2)[np.triu_indices(6, 1)] / sigma
    assert 0.02 < r.min() and r.max() < 0.5
    u, S = oracle.direct(x, g, sigma, K=0, targets=tid)
    um, Sm = _mp_sum(x, g, x, g, tid, sigma, 2 * np.pi, 0)
    assert np.allclose(u, um, rtol=1e-12, atol=1e-14 * np.abs(um).max())
    assert np.allclose(S, Sm, rtol=1e-11, atol=1e-13 * np.abs(Sm).max())


def test_gradient_series_branch_matches_fd():
    # grad u at a point within 0.3 sigma of sources (rho < 0.5: F from its series) against
    # central differences of u, whose K alone is pinned by the single-blob closed form; and
    # S = (gamma_t . grad) u there (Eq. stretching)
    sigma = 0.6
    x, g = _cluster(sigma, 23)
    xt = (x[0] + np.array([0.11, -0.07, 0.05]) * sigma)[None]
    rho = np.linalg.norm(x - xt, axis=1) / sigma
    assert rho.min() < 0.2 and (rho < 0.5).sum() >= 4
    gt = np.array([[0.4, -0.9, 0.3]])
    u, S, G = oracle.direct(x, g, sigma, K=0, xt=xt, gt=gt, grad=True)
    eps = 1e-5 * sigma
    J = np.zeros((3, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        up, _ = oracle.direct(x, g, sigma, K=0, xt=xt + e)
        um, _ = oracle.direct(x, g, sigma, K=0, xt=xt - e)
        J[:, k] = (up[0] - um[0]) / (2 * eps)
    assert np.allclose(G[0], J, rtol=1e-7, atol=1e-9 * np.abs(J).max()), (G[0], J)
    assert np.allclose(S[0], J @ gt[0], rtol=1e-7, atol=1e-9 * np.abs(S).max())


def test_stretching_equals_directional_derivative_of_u():
    # S_i = (gamma_i . grad) u at x_i, checked by central differences of the oracle's own u;
    # the displaced point lies on the line through x_i along gamma_i, where the self blob's
    # velocity gamma_i x d vanishes, so the self term needs no special handling.
    f = wl.make_vortex_lattice(6, 2, 7)
    x, g, s = f["x"], f["alpha"], f["sigma"]
    tid = np.array([0, 17, 100, 215])
    u, S = oracle.direct(x, g, s, K=1, targets=tid)
    eps = 1e-4 * f["h"]
    for k, i in enumerate(tid):
        gi = g[i]
        gh = gi / np.linalg.norm(gi)
        up, _ = oracle.direct(x, g, s, K=1, xt=(x[i] + eps * gh)[None])
        um, _ = oracle.direct(x, g, s, K=1, xt=(x[i] - eps * gh)[None])
        fd = (up[0] - um[0]) / (2 * eps) * np.linalg.norm(gi)
        assert np.allclose(S[k], fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max()), (S[k], fd)


def test_gradient_tensor_matches_fd_and_invariants():
    f = wl.make_vortex_lattice(6, 2, 9)
    x, g, s = f["x"], f["alpha"], f["sigma"]
    tid = np.arange(0, 216, 7)
    u, S, G = oracle.direct(x, g, s, K=1, targets=tid, grad=True)
    # S = G gamma_i
    assert np.allclose(S, np.einsum("iak,ik->ia", G, g[tid]), rtol=1e-12, atol=1e-15)
    # divergence-free
    assert np.abs(np.trace(G, axis1=1, axis2=2)).max() < 1e-12 * np.abs(G).max()
    eps = 1e-4 * f["h"]
    for k, i in enumerate(tid[:5]):
        J = np.zeros((3, 3))
        for d in range(3):
            e = np.zeros(3)
            e[d] = eps
            # offset along an axis: the self blob contributes gamma_i x e K(eps), equal and
            # opposite at +-e, so remove it by excluding the source i explicitly
            mask = np.ones(len(x), bool)
            mask[i] = False
            up, _ = oracle.direct(x[mask], g[mask], s, K=1, xt=(x[i] + e)[None])
            um, _ = oracle.direct(x[mask], g[mask], s, K=1, xt=(x[i] - e)[None])
            # add back the images of particle i itself (n != 0)
            ui_p, _ = oracle.direct(x[i:i + 1], g[i:i + 1], s, K=1, kmin=1, xt=(x[i] + e)[None])
            ui_m, _ = oracle.direct(x[i:i + 1], g[i:i + 1], s, K=1, kmin=1, xt=(x[i] - e)[None])
            J[:, d] = ((up + ui_p) - (um + ui_m))[0] / (2 * eps)
        assert np.allclose(G[k], J, rtol=1e-6, atol=1e-8 * np.abs(J).max()), (G[k], J)


def test_transpose_scheme_conserves_total_vorticity():
    # sum_i (grad u_i)^T gamma_i = 0 exactly: each pair's two terms cancel
    f = wl.make_vortex_lattice(6, 2, 3)
    x, g, s = f["x"], f["alpha"], f["sigma"]
    _, _, G = oracle.direct(x, g, s, K=1, grad=True)
    tot = np.einsum("iak,ia->k", G, g)
    scale = np.abs(np.einsum("iak,ia->ik", G, g)).sum()
    assert np.abs(tot).max() < 1e-13 * scale


def test_pair_antisymmetry_linearity_symmetry():
    rng = np.random.default_rng(2)
    # two particles with equal strength: equal and opposite velocities (no images)
    x = np.array([[0.1, 0.2, 0.3], [0.5, -0.1, 0.2]])
    gsame = np.array([[0.3, 0.4, -0.2]] * 2)
    u, _ = oracle.direct(x, gsame, 0.3, K=0)
    assert np.allclose(u[0], -u[1], rtol=1e-14, atol=1e-16)
    # linearity and the symmetry <w, A gamma> = <A w, gamma> of the Biot-Savart matrix
    f = wl.make_vortex_lattice(5, 2, 1)
    x, s = f["x"], f["sigma"]
    a = rng.normal(size=x.shape)
    b = rng.normal(size=x.shape)
    ua, _ = oracle.direct(x, a, s, K=1)
    ub, _ = oracle.direct(x, b, s, K=1)
    uab, _ = oracle.direct(x, 2.0 * a - 3.0 * b, s, K=1)
    assert np.allclose(uab, 2.0 * ua - 3.0 * ub, rtol=1e-12, atol=1e-13 * np.abs(uab).max())
    lhs = np.sum(b * ua)
    rhs = np.sum(ub * a)
    assert abs(lhs - rhs) < 1e-12 * (np.abs(b * ua).sum())


def test_translation_invariance_of_full_lattice():
    # moving every particle (and so every image) by d leaves u and S unchanged
    f = wl.make_vortex_lattice(5, 2, 6)
    x, g, s = f["x"], f["alpha"], f["sigma"]
    tid = np.arange(0, 125, 9)
    u0, S0 = oracle.direct(x, g, s, K=1, targets=tid)
    u1, S1 = oracle.direct(x + np.array([0.3, -1.7, 2.2]), g, s, K=1, targets=tid)
    assert np.allclose(u0, u1, rtol=1e-10, atol=1e-12 * np.abs(u0).max())
    assert np.allclose(S0, S1, rtol=1e-10, atol=1e-12 * np.abs(S0).max())


def test_spectral_series_two_ways():
    # FFT-folded lattice series and the direct mode sum agree (independent evaluations)
    f = wl.make_vortex_lattice(8, 2, 1)
    us, Ss = oracle.spectral.direct_series(f["x"], f["alpha"], f["sigma"])
    ul, Sl = oracle.spectral.lattice(8, f["alpha"], f["sigma"])
    assert np.abs(us - ul).max() < 1e-12 * np.abs(ul).max()
    assert np.abs(Ss - Sl).max() < 1e-12 * np.abs(Sl).max()


def test_image_cube_converges_to_periodic_series():
    # the cube-of-images sum minus its uniform offset tends to the Fourier series,
    # and S tends to it with no offset (Section 4.1 periodic images)
    f = wl.make_vortex_lattice(8, 2, 1)
    x, g, s = f["x"], f["alpha"], f["sigma"]
    ul, Sl = oracle.spectral.lattice(8, g, s)
    errs_u, errs_S = [], []
    for K in (1, 2, 4):
        u, S = oracle.direct(x, g, s, K=K)
        d = u - ul
        d -= d.mean(0)
        errs_u.append(np.linalg.norm(d) / np.linalg.norm(ul))
        errs_S.append(np.linalg.norm(S - Sl) / np.linalg.norm(Sl))
    assert errs_u[0] > errs_u[1] > errs_u[2]
    assert errs_S[0] > errs_S[1] > errs_S[2]
    # the tail decays at least like 1/K^1.5
    assert errs_u[2] < errs_u[0] / 4 ** 1.5
    assert errs_S[2] < errs_S[0] / 4 ** 1.5


def test_coincident_distinct_particles_take_the_smooth_limit():
    # two different particles at one point: the smoothed kernel is finite there,
    # K(0) = lim q/(4 pi r^3) = sqrt(2/pi)/(12 pi sigma^3), so S_1 = K(0) gamma_2 x gamma_1
    sigma = 0.37
    x = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0]])
    g = np.array([[0.3, -0.2, 0.5], [-0.4, 0.9, 0.1]])
    u, S = oracle.direct(x, g, sigma, K=0)
    K0 = np.sqrt(2 / np.pi) / (12 * np.pi * sigma ** 3)
    assert np.allclose(u, 0.0, atol=1e-15)
    assert np.allclose(S[0], K0 * np.cross(g[1], g[0]), rtol=1e-13)
    # continuous with a tiny separation along gamma_1 (where the F term vanishes)
    d = 1e-7 * sigma * g[0] / np.linalg.norm(g[0])
    u2, S2 = oracle.direct(x[1:], g[1:], sigma, K=0, xt=(x[0] + d)[None], gt=g[:1])
    assert np.allclose(S2[0], S[0], rtol=1e-9)


def test_loss_gradient_matches_central_differences():
    # dL/dgamma = A w and dL/dx = (grad u^g)^T w + (grad u^w)^T g, against the oracle's own
    # central differences of L = sum |u - u*|^2 (one image layer, 27 jittered particles)
    n = 3
    h = 2 * np.pi / n
    x = wl.jitter(wl.lattice_positions(n), h, 0.3, seed=12)
    rng = np.random.default_rng(13)
    g = rng.normal(size=x.shape)
    sigma = 0.9 * h
    ustar = rng.normal(size=x.shape) * 0.1
    dg, dx, _ = oracle.gradient.loss_gradient(x, g, sigma, ustar, K=1)
    eps = 1e-6
    for (i, a) in [(0, 0), (4, 2), (13, 1), (26, 0)]:
        gp, gm = g.copy(), g.copy()
        gp[i, a] += eps
        gm[i, a] -= eps
        fd = (oracle.gradient.loss(x, gp, sigma, ustar) - oracle.gradient.loss(x, gm, sigma, ustar)) / (2 * eps)
        assert abs(fd - dg[i, a]) < 1e-7 * max(1.0, abs(fd)), (i, a, fd, dg[i, a])
        xp, xm = x.copy(), x.copy()
        xp[i, a] += eps
        xm[i, a] -= eps
        fd = (oracle.gradient.loss(xp, g, sigma, ustar) - oracle.gradient.loss(xm, g, sigma, ustar)) / (2 * eps)
        assert abs(fd - dx[i, a]) < 1e-7 * max(1.0, abs(fd)), (i, a, fd, dx[i, a])


def test_heun_step_is_second_order():
    # Heun's global error falls 4x per halving of dt (a first-order bug would give 2x)
    n = 3
    h = 2 * np.pi / n
    x0 = wl.jitter(wl.lattice_positions(n), h, 0.2, seed=31)
    g0 = np.random.default_rng(32).normal(size=x0.shape) * 0.5
    sigma, nu, T = 0.9 * h, 0.01, 0.4

    def run(nsteps):
        x, g, s = x0.copy(), g0.copy(), sigma
        dt = T / nsteps
        for _ in range(nsteps):
            x, g, s = oracle.integrate.heun_step(x, g, s, dt, nu, K=0)
        return x, g, s

    xr, gr, sr = run(64)
    errs = []
    for m in (4, 8, 16):
        x, g, s = run(m)
        assert abs(s - sr) < 1e-12   # core spreading is exact: sigma^2 = sigma0^2 + 2 nu t
        d = np.mod(x - xr + np.pi, 2 * np.pi) - np.pi
        errs.append(np.abs(d).max() + np.abs(g - gr).max())
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs


def test_gaussian_basis_is_normalised():
    # Eq. (gaussian): zeta integrates to one (lattice quadrature of a well-resolved core)
    n = 24
    h = 2 * np.pi / n
    xl = wl.lattice_positions(n)
    src = np.array([[np.pi, np.pi, np.pi]])
    w = oracle.reinit.gaussian_sum(xl, src, np.array([[1.0, 0.0, 0.0]]), 2.0 * h)
    assert abs(w[:, 0].sum() * h ** 3 - 1.0) < 1e-10


def test_reinit_deconvolves_a_single_gaussian():
    # one old particle of core sigma = 2h on a new lattice point, new core sigma0 = h: since
    # zeta_a * zeta_b = zeta_sqrt(a^2 + b^2), Z gamma' = omega is solved by lattice samples of a
    # Gaussian of width sqrt(sigma^2 - sigma0^2) (with its periodic images), times h^3
    import itertools
    m = 12
    h = 2 * np.pi / m
    xl = wl.lattice_positions(m)
    j = 400
    gj = np.array([[0.3, -0.5, 0.8]])
    sigma = 2.0 * h
    w = np.sqrt(sigma ** 2 - h ** 2)
    exact = np.zeros((len(xl), 1))
    for nimg in itertools.product((-1, 0, 1), repeat=3):
        d = xl - xl[j] - np.array(nimg) * 2 * np.pi
        exact[:, 0] += np.exp(-0.5 * (d * d).sum(1) / w ** 2) / (2 * np.pi * w * w) ** 1.5
    exact = exact * gj * h ** 3
    _, g, res, _ = oracle.reinit.reinit(xl[j:j + 1], gj, sigma, m, iters=300)
    assert res < 2e-5
    assert np.linalg.norm(g - exact) < 5e-4 * np.linalg.norm(exact)


def test_reinit_residual_decreases():
    m = 6
    h = 2 * np.pi / m
    x = wl.jitter(wl.lattice_positions(m), h, 0.3, seed=51)
    g = np.random.default_rng(52).normal(size=x.shape) * h ** 3
    res = [oracle.reinit.reinit(x, g, 1.1 * h, m, iters=k)[2] for k in (0, 1, 5, 20)]
    assert res[0] > res[1] > res[2] > res[3]


# ---------------------------------------------------------------------------------------
# Diagnostics of Section 5.2 (energy spectrum, derivative skewness and flatness)

def test_spectrum_single_mode_closed_form():
    # u_y = sin(m x): u_hat = -+i/2 at k = +-m e_x, so E(m) = 2 * 0.5 * 1/4 = 1/4 and
    # nothing else; 0.5 <u^2> = 1/4 as well
    n, m = 16, 3
    x = wl.lattice_positions(n)
    u = np.zeros((n ** 3, 3))
    u[:, 1] = np.sin(m * x[:, 0])
    E = oracle.diagnostics.energy_spectrum(u, n, 14)
    ref = np.zeros(15)
    ref[m] = 0.25
    assert np.allclose(E, ref, atol=1e-14)


def test_spectrum_oblique_mode_shell():
    # a mode along (1, 2, 2) has |k| = 3 exactly; one along (2, 2, 1) too; (1, 1, 1) lands in
    # shell round(sqrt 3) = 2
    n = 16
    x = wl.lattice_positions(n)
    u = np.zeros((n ** 3, 3))
    u[:, 0] = np.cos(x @ np.array([1.0, 2.0, 2.0]))
    u[:, 2] = 2.0 * np.cos(x @ np.array([1.0, 1.0, 1.0]))
    E = oracle.diagnostics.energy_spectrum(u, n, 14)
    assert abs(E[3] - 0.25) < 1e-13 and abs(E[2] - 1.0) < 1e-13
    assert abs(E.sum() - 1.25) < 1e-13


def test_spectrum_parseval_random_field():
    n = 16
    rng = np.random.default_rng(7)
    u = rng.standard_normal((n ** 3, 3))
    E = oracle.diagnostics.energy_spectrum(u, n, int(np.ceil(np.sqrt(3) * n / 2)) + 1)
    assert abs(E.sum() - 0.5 * (u ** 2).sum(1).mean()) < 1e-12 * E.sum()


def test_spectrum_of_generated_field_is_the_prescribed_spectrum():
    # the generator rescales every integer shell to k^4 exp(-2 k^2/k0^2) (Eq. initspec) with
    # unit energy; the lattice FFT of its velocity recovers exactly that (no aliasing: the
    # modes stay inside |k_i| <= n/2 - 1)
    n, k0 = 32, 4
    u = wl.lattice_velocity(n, k0, seed=1)
    E = oracle.diagnostics.energy_spectrum(u, n, 27)
    s = np.arange(28, dtype=np.float64)
    tgt = s ** 4 * np.exp(-2.0 * s ** 2 / k0 ** 2)
    smax = int(np.rint(np.sqrt(3) * min(4 * k0, n // 2 - 1)))
    tgt[smax + 1:] = 0.0
    tgt /= tgt.sum()
    assert np.allclose(E, tgt, rtol=1e-10, atol=1e-14)


def test_derivative_moments_closed_form():
    # u = (sin x, sin y, sin z): du_a/dx_a = cos of the coordinate; on a lattice of n >= 5
    # points the sample means of cos^2, cos^3, cos^4 are 1/2, 0, 3/8: F3 = 0, F4 = 3/2
    n = 12
    x = wl.lattice_positions(n)
    g = np.zeros((n ** 3, 9))
    g[:, 0], g[:, 4], g[:, 8] = np.cos(x[:, 0]), np.cos(x[:, 1]), np.cos(x[:, 2])
    g[:, 1] = 5.0  # off-diagonal entries are not samples
    m2, m3, m4, F3, F4 = oracle.diagnostics.derivative_moments(g)
    assert abs(m2 - 0.5) < 1e-14 and abs(m3) < 1e-14 and abs(m4 - 0.375) < 1e-14
    assert abs(F3) < 1e-13 and abs(F4 - 1.5) < 1e-13


def test_derivative_moments_gaussian_samples():
    # normal samples: F3 -> 0, F4 -> 3 (statistical: 3e6 samples, 5-sigma bounds)
    rng = np.random.default_rng(11)
    g = rng.standard_normal((1_000_000, 9))
    _, _, _, F3, F4 = oracle.diagnostics.derivative_moments(g)
    assert abs(F3) < 5 * np.sqrt(15.0 / 3e6) and abs(F4 - 3.0) < 5 * np.sqrt(96.0 / 3e6)


def test_far_images_is_the_cube_sum_beyond_the_central_boxes():
    # the far-image increment (image boxes 2 <= max|n| <= K, every pair >= 10 sigma apart) equals
    # the full smoothed-kernel cube sum over the same boxes (Section 4.1 images; there q = 1 to
    # FP64 rounding), and its S term is pinned by a 30-digit sum of the singular kernel
    # K = 1/(4 pi r^3), F = K'(r)/r = -3/(4 pi r^5) written out independently here
    rng = np.random.default_rng(17)
    L = 2 * np.pi
    xs = rng.uniform(0, L, (24, 3))
    gs = rng.normal(size=(24, 3))
    xt = rng.uniform(0, L, (3, 3))
    gt = rng.normal(size=(3, 3))
    sigma = 0.3
    uf, Sf = oracle.far_images(xs, gs, xt, gt, sigma, L=L, kmin=2, K=3)
    ud, Sd = oracle.direct(xs, gs, sigma, L=L, K=3, kmin=2, xt=xt, gt=gt)
    assert np.allclose(uf, ud, rtol=1e-11, atol=1e-13 * np.abs(ud).max())
    assert np.allclose(Sf, Sd, rtol=1e-11, atol=1e-13 * np.abs(Sd).max())
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for i in range(len(xt)):
        u = [mp.mpf(0)] * 3
        S = [mp.mpf(0)] * 3
        for n in itertools.product(range(-2, 3), repeat=3):
            if max(abs(v) for v in n) < 2:
                continue
            for j in range(len(xs)):
                r = [mp.mpf(xt[i][a]) - mp.mpf(xs[j][a]) - n[a] * mp.mpf(L) for a in range(3)]
                rr = mp.sqrt(r[0] ** 2 + r[1] ** 2 + r[2] ** 2)
                K = 1 / (4 * mp.pi * rr ** 3)
                F = -3 / (4 * mp.pi * rr ** 5)
                g = [mp.mpf(v) for v in gs[j]]
                h = [mp.mpf(v) for v in gt[i]]
                W = [g[1] * r[2] - g[2] * r[1], g[2] * r[0] - g[0] * r[2], g[0] * r[1] - g[1] * r[0]]
                X = [g[1] * h[2] - g[2] * h[1], g[2] * h[0] - g[0] * h[2], g[0] * h[1] - g[1] * h[0]]
                hr = h[0] * r[0] + h[1] * r[1] + h[2] * r[2]
                for a in range(3):
                    u[a] += K * W[a]
                    S[a] += K * X[a] + F * hr * W[a]
        u2, S2 = oracle.far_images(xs, gs, xt[i:i + 1], gt[i:i + 1], sigma, L=L, kmin=2, K=2)
        assert np.allclose(u2[0], [float(v) for v in u], rtol=1e-12, atol=1e-15)
        assert np.allclose(S2[0], [float(v) for v in S], rtol=1e-12, atol=1e-15)
    # boxes closer than 10 sigma are refused (the reduction to the singular kernel would not hold)
    with pytest.raises(ValueError):
        oracle.far_images(xs, gs, xt, gt, L / 9.0, L=L, kmin=2, K=3)
