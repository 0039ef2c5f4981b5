"""Gradient oracle for L = sum_i |u_i - u*_i|^2 (TEST INFRASTRUCTURE ONLY).

u_i is the periodic regularised Biot-Savart velocity of Eq. (biotsavart) (cube of image
boxes), u*_i fixed data.  With w_i = dL/du_i = 2 (u_i - u*_i):

* dL/dgamma = A^T w = A w: the Biot-Savart matrix with u = A gamma has blocks
  A_ij = -K(r_ij) [r_ij]x, and A_ji = A_ij^T because K is even and [r]x odd, so the
  strength gradient is the velocity induced at the particles by strengths w.
* dL/dx_m = (grad u^gamma(x_m))^T w_m + (grad u^w(x_m))^T gamma_m: the first term moves the
  target, the second the source (the kernel K(r) gamma x r is odd in r, so its gradient is
  even and the source derivative at x_m equals the gradient of the w-field there).

Both are formed from the direct sums of ``oracle.direct`` (velocity and its gradient).
"""
import numpy as np

from . import direct as _direct


def loss(x, gamma, sigma, u_star, K=1, L=2 * np.pi):
    u, _ = _direct(x, gamma, sigma, L=L, K=K)
    return float(((u - u_star) ** 2).sum())


def loss_gradient(x, gamma, sigma, u_star, K=1, L=2 * np.pi, targets=None, w=None):
    """(dL/dgamma, dL/dx, w) at the particles (or at ``targets``).

    w defaults to 2 (u - u*) from the oracle's own u; pass w to use given weights.
    """
    x = np.asarray(x, float)
    g = np.asarray(gamma, float)
    if w is None:
        u, _ = _direct(x, g, sigma, L=L, K=K)
        w = 2.0 * (u - u_star)
    tid = np.arange(len(x)) if targets is None else np.asarray(targets)
    _, _, Gg = _direct(x, g, sigma, L=L, K=K, targets=tid, grad=True)
    uw, _, Gw = _direct(x, w, sigma, L=L, K=K, targets=tid, grad=True)
    dx = np.einsum("iak,ia->ik", Gg, w[tid]) + np.einsum("iak,ia->ik", Gw, g[tid])
    return uw, dx, w
