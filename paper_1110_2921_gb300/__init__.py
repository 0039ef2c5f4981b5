"""GB300-native periodic FMM for the vortex-particle velocity and stretching term.

Python face of libvfmm (C-ABI in include/vfmm.h).  PyTorch supplies device memory and
streams; every step of the evaluation runs in the library's CUDA kernels.
"""
import math

from . import _native
from ._native import (VfmmError, vfmm_create, vfmm_destroy, vfmm_build_tree,  # noqa: F401
                      vfmm_eval_velocity_stretching, vfmm_eval_host, vfmm_sync,
                      vfmm_get_timings, vfmm_get_tree_info, vfmm_set_stream, config_default,
                      vfmm_eval_velocity_gradient, vfmm_eval_adjoint, vfmm_rk_step, vfmm_diagnostics,
                      vfmm_energy_spectrum, vfmm_derivative_moments,
                      vfmm_reinit)

PRECISIONS = {"fp32": _native.VFMM_M2L_FP32, "fp64": _native.VFMM_M2L_FP64,
              "tf32x3": _native.VFMM_M2L_TF32X3, "bf16x3": _native.VFMM_M2L_BF16X3}
PHASES = ["tree", "p2m", "m2m", "m2l", "periodic", "l2l", "l2p", "p2p"]


def make_config(p=10, depth=0, ncrit=64, near_rings=0, rho_cut=5.0, periodic_levels=2,
                box=2 * math.pi, dtype="f32", m2l="bf16x3", method="fmm", direct_images=1,
                stream=None, concurrent_far=1):
    c = config_default()
    c.p = p
    c.depth = depth
    c.ncrit = ncrit
    c.near_rings = near_rings
    c.rho_cut = rho_cut
    c.periodic_levels = periodic_levels
    c.box = box
    c.dtype = _native.VFMM_F64 if dtype in ("f64", "float64") else _native.VFMM_F32
    if c.dtype == _native.VFMM_F64:
        m2l = "fp64"
    c.m2l_prec = PRECISIONS[m2l]
    c.method = _native.VFMM_METHOD_DIRECT if method == "direct" else _native.VFMM_METHOD_FMM
    c.direct_images = direct_images
    c.stream = stream
    c.concurrent_far = int(concurrent_far)
    return c


class VortexFMM:
    """One handle of libvfmm bound to torch tensors on the current CUDA device."""

    def __init__(self, **kw):
        import torch
        self.torch = torch
        self.dtype = torch.float64 if kw.get("dtype", "f32") in ("f64", "float64") else torch.float32
        stream = torch.cuda.current_stream().cuda_stream
        self.cfg = make_config(stream=stream, **kw)
        self.h = vfmm_create(self.cfg)
        self.n = 0

    def close(self):
        if self.h:
            vfmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, t):
        torch = self.torch
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and t.dim() == 2 and t.shape[1] == 3):
            raise ValueError("expected a contiguous CUDA (n, 3) tensor of %s" % self.dtype)

    def build_tree(self, x):
        self._check(x)
        vfmm_set_stream(self.h, self.torch.cuda.current_stream().cuda_stream)
        vfmm_build_tree(self.h, x.shape[0], x.data_ptr())
        self.n = x.shape[0]

    def eval(self, gamma, sigma, stretching=True, out=None):
        self._check(gamma)
        if self.n and gamma.shape[0] != self.n:
            raise ValueError("gamma has %d rows, the tree %d" % (gamma.shape[0], self.n))
        torch = self.torch
        if out is None:
            u = torch.empty_like(gamma)
            s = torch.empty_like(gamma) if stretching else None
        else:
            u, s = out
        vfmm_set_stream(self.h, torch.cuda.current_stream().cuda_stream)
        vfmm_eval_velocity_stretching(self.h, gamma.data_ptr(), sigma, u.data_ptr(),
                                      s.data_ptr() if s is not None else 0)
        return u, s

    def eval_gradient(self, gamma, sigma):
        """Velocity (n, 3) and velocity gradient G (n, 3, 3), G[i, a, k] = du_a/dx_k."""
        self._check(gamma)
        torch = self.torch
        u = torch.empty_like(gamma)
        g = torch.empty(gamma.shape[0], 3, 3, dtype=gamma.dtype, device=gamma.device)
        vfmm_set_stream(self.h, torch.cuda.current_stream().cuda_stream)
        vfmm_eval_velocity_gradient(self.h, gamma.data_ptr(), sigma, u.data_ptr(), g.data_ptr())
        return u, g

    def adjoint(self, gamma, sigma, w):
        """(dL/dgamma, dL/dx) for dL/du = w on the current tree."""
        self._check(gamma)
        self._check(w)
        torch = self.torch
        dg = torch.empty_like(gamma)
        dx = torch.empty_like(gamma)
        vfmm_set_stream(self.h, torch.cuda.current_stream().cuda_stream)
        vfmm_eval_adjoint(self.h, gamma.data_ptr(), sigma, w.data_ptr(), 0, dg.data_ptr(), dx.data_ptr())
        return dg, dx

    def rk_step(self, x, gamma, sigma, dt, nu):
        """One Heun step in place on x, gamma; returns the new core size."""
        self._check(x)
        self._check(gamma)
        vfmm_set_stream(self.h, self.torch.cuda.current_stream().cuda_stream)
        s = vfmm_rk_step(self.h, x.shape[0], x.data_ptr(), gamma.data_ptr(), sigma, dt, nu)
        self.n = 0
        return s

    def reinit(self, x, gamma, sigma, m, sigma_new=0.0, iters=20):
        """New particles on the m^3 lattice: (x_new, gamma_new, residual)."""
        self._check(x)
        self._check(gamma)
        torch = self.torch
        xn = torch.empty(m ** 3, 3, dtype=x.dtype, device=x.device)
        gn = torch.empty_like(xn)
        vfmm_set_stream(self.h, torch.cuda.current_stream().cuda_stream)
        res = vfmm_reinit(self.h, x.shape[0], x.data_ptr(), gamma.data_ptr(), sigma, m, sigma_new, iters,
                          xn.data_ptr(), gn.data_ptr())
        self.n = 0
        return xn, gn, res

    def diagnostics(self, x, gamma, u=None):
        """FP64 total vorticity, sum x cross gamma, sum |u|^2, sum |gamma|^2."""
        vfmm_set_stream(self.h, self.torch.cuda.current_stream().cuda_stream)
        v = vfmm_diagnostics(self.h, x.shape[0], x.data_ptr(), gamma.data_ptr(), u.data_ptr() if u is not None else 0)
        return {"total_vorticity": v[0:3], "x_cross_gamma": v[3:6], "sum_u2": v[6], "sum_gamma2": v[7]}

    def energy_spectrum(self, u_lattice, n, kmax):
        """E(k), k = 0..kmax, of a velocity sampled on the n^3 lattice (device (n^3, 3), lattice order)."""
        self._check(u_lattice)
        return vfmm_energy_spectrum(self.h, n, u_lattice.data_ptr(), kmax)

    def derivative_moments(self, grad):
        """(mean d^2, mean d^3, mean d^4, F3, F4) of the longitudinal derivatives of grad (n, 9)."""
        if not (grad.is_cuda and grad.dtype == self.dtype and grad.is_contiguous() and grad.dim() == 2
                and grad.shape[1] == 9):
            raise ValueError("expected a contiguous CUDA (n, 9) tensor of %s" % self.dtype)
        return vfmm_derivative_moments(self.h, grad.shape[0], grad.data_ptr())

    def __call__(self, x, gamma, sigma, stretching=True):
        self.build_tree(x)
        return self.eval(gamma, sigma, stretching)

    def sync(self):
        vfmm_sync(self.h)

    def timings(self):
        return dict(zip(PHASES, vfmm_get_timings(self.h)))

    def tree_info(self):
        return vfmm_get_tree_info(self.h)

    def eval_host(self, x, gamma, sigma, u=None, s=None):
        """x, gamma: host numpy (n, 3) arrays of the handle's dtype (pinned for speed)."""
        import numpy as np
        npdt = np.float64 if self.dtype == self.torch.float64 else np.float32
        x = np.ascontiguousarray(x, dtype=npdt)
        gamma = np.ascontiguousarray(gamma, dtype=npdt)
        if u is None:
            u = np.empty_like(gamma)
        if s is None:
            s = np.empty_like(gamma)
        vfmm_eval_host(self.h, x.shape[0], x.ctypes.data, gamma.ctypes.data, sigma,
                       u.ctypes.data, s.ctypes.data)
        return u, s


def _autograd_function():
    import torch

    class BiotSavart(torch.autograd.Function):
        """u, S = (Biot-Savart velocity, stretching) of (x, gamma); differentiable in u.

        backward uses vfmm_eval_adjoint on the tree of the forward positions."""

        @staticmethod
        def forward(ctx, x, gamma, fmm, sigma):
            x = x.detach().contiguous()
            gamma = gamma.detach().contiguous()
            fmm.build_tree(x)
            u, s = fmm.eval(gamma, sigma)
            ctx.save_for_backward(x, gamma)
            ctx.fmm = fmm
            ctx.sigma = sigma
            ctx.mark_non_differentiable(s)
            return u, s

        @staticmethod
        def backward(ctx, gu, gs):
            x, gamma = ctx.saved_tensors
            if gs is not None and bool((gs != 0).any()):
                raise NotImplementedError("the stretching output is not differentiable")
            fmm = ctx.fmm
            fmm.build_tree(x)
            dgamma, dx = fmm.adjoint(gamma, ctx.sigma, gu.contiguous())
            return dx, dgamma, None, None

    return BiotSavart


_BS = None


def biot_savart(x, gamma, fmm, sigma):
    """Differentiable (u, S) of particles x with strengths gamma through the handle ``fmm``."""
    global _BS
    if _BS is None:
        _BS = _autograd_function()
    return _BS.apply(x, gamma, fmm, sigma)
