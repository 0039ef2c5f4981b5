"""Reinitialisation oracle (TEST INFRASTRUCTURE ONLY), dense FP64 numpy for small lattices.

Section 2.2: the vorticity field is the superposition of Gaussian basis functions
(Eqs. smoothingfunction, gaussian), zeta_sigma(r) = (2 pi sigma^2)^(-3/2) exp(-r^2/(2 sigma^2)).
Reinitialisation interpolates it onto a lattice of new particles with core sigma0 by solving
sum_k gamma'_k zeta_sigma0(x_g - x_k) = omega(x_g) for gamma' (the paper uses GMRES with the
initial guess gamma' = omega dx^3, Section 5.3).  Here: 'iters' steepest-descent steps with
exact line search on 0.5 |Z gamma' - omega|^2 (Z symmetric):
    r = omega - Z gamma';  d = Z r;  q = Z d;  alpha = (r.q)/(q.q);  gamma' += alpha d;  r -= alpha q.
Periodic images: every image box n with max|n_i| <= K.
"""
import itertools

import numpy as np


def zeta(r2, sigma):
    return (2.0 * np.pi * sigma * sigma) ** -1.5 * np.exp(-0.5 * r2 / (sigma * sigma))


def gaussian_sum(xt, xs, gs, sigma, L=2 * np.pi, K=1):
    """omega(x_t) = sum_n sum_j gamma_j zeta_sigma(x_t - x_j - n L)."""
    out = np.zeros((len(xt), 3))
    for n in itertools.product(range(-K, K + 1), repeat=3):
        d = xt[:, None, :] - xs[None, :, :] - np.array(n) * L
        out += zeta((d * d).sum(-1), sigma) @ gs
    return out


def gaussian_matrix(x, sigma, L=2 * np.pi, K=1):
    Z = np.zeros((len(x), len(x)))
    for n in itertools.product(range(-K, K + 1), repeat=3):
        d = x[:, None, :] - x[None, :, :] - np.array(n) * L
        Z += zeta((d * d).sum(-1), sigma)
    return Z


def reinit(x, gamma, sigma, m, sigma0=None, iters=20, L=2 * np.pi, K=1):
    """New lattice particles: (x_lattice, gamma', residual |r|/|omega|, omega)."""
    from workload import lattice_positions   # the lattice positions only (no arithmetic of the method)
    h = L / m
    if sigma0 is None:
        sigma0 = h
    xl = lattice_positions(m, L)
    omega = gaussian_sum(xl, np.asarray(x, float), np.asarray(gamma, float), sigma, L, K)
    Z = gaussian_matrix(xl, sigma0, L, K)
    g = omega * h ** 3
    r = omega - Z @ g
    for _ in range(iters):
        d = Z @ r
        q = Z @ d
        alpha = (r * q).sum() / (q * q).sum()
        g = g + alpha * d
        r = r - alpha * q
    return xl, g, float(np.linalg.norm(r) / np.linalg.norm(omega)), omega
