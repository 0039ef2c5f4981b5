"""Time step and diagnostics oracle (TEST INFRASTRUCTURE ONLY).

The vortex method advances positions by the velocity (Eq. convection), strengths by the
stretching term (Eq. stretching) and the core by dsigma^2/dt = 2 nu (Eq. csm); the three
updates happen simultaneously (Section 2.2).  The paper integrates with forward Euler
(Section 4.1); the second-order Heun scheme (explicit trapezoid) is used here:
  stage 1: (u1, S1) at (x, gamma, sigma)
  stage 2: (u2, S2) at (x + dt u1, gamma + dt S1, sqrt(sigma^2 + 2 nu dt))
  x' = x + dt (u1 + u2)/2,  gamma' = gamma + dt (S1 + S2)/2,  sigma'^2 = sigma^2 + 2 nu dt,
positions wrapped into [0, L).
"""
import numpy as np

from . import direct as _direct


def heun_step(x, gamma, sigma, dt, nu, K=1, L=2 * np.pi):
    u1, s1 = _direct(np.mod(x, L), gamma, sigma, L=L, K=K)
    sig1 = float(np.sqrt(sigma * sigma + 2.0 * nu * dt))
    x1 = np.mod(x + dt * u1, L)
    g1 = gamma + dt * s1
    u2, s2 = _direct(x1, g1, sig1, L=L, K=K)
    xn = np.mod(x + 0.5 * dt * (u1 + u2), L)
    gn = gamma + 0.5 * dt * (s1 + s2)
    return xn, gn, sig1


def diagnostics(x, gamma, u):
    """FP64 sums: total vorticity sum gamma (3), sum x cross gamma (3), sum |u|^2, sum |gamma|^2."""
    x = np.asarray(x, float)
    g = np.asarray(gamma, float)
    u = np.asarray(u, float)
    return np.concatenate([g.sum(0), np.cross(x, g).sum(0), [(u * u).sum()], [(g * g).sum()]])
