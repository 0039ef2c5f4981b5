"""FP64 CPU oracle for the periodic regularised Biot-Savart velocity and stretching.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` leg are the only callers.  Nothing in the GPU
package imports it, and it imports nothing from the GPU package.

Contents
--------
* ``direct`` (C + OpenMP, ``direct.c``): the plain double sum over particles and a cube of
  periodic image boxes, Eqs. (biotsavart), (cutoff), (stretching) and the image count of
  Section 4.1.  Optional full velocity gradient.
* ``spectral``: the fully periodic field as a Fourier series (independent of the direct sum).
* ``gradient``: dL/dgamma and dL/dx of L = sum |u - u*|^2 from the direct sums.
* ``integrate``: one Heun step of Eqs. (convection), (stretching), (csm); FP64 diagnostics.
* ``reinit``: Gaussian-basis reinitialisation onto a lattice (dense FP64, small lattices).
* ``diagnostics``: energy spectrum of a lattice velocity field, skewness and flatness of the
  velocity derivatives (Section 5.2).

Parity status: every function here is pinned by the ``tests/test_oracle_*.py`` checks
(closed forms, quadrature, mpmath brute force, invariants, spectral cross-check).
"""
import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force=False):
    """Compile direct.c with gcc (-O2 -fopenmp) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    # -fno-math-errno lets the singular far-image loop use vector square roots; it changes no
    # result (errno is never read)
    cmd = ["gcc", "-O2", "-fopenmp", "-fno-math-errno", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        lib.oracle_direct.argtypes = [ctypes.c_int64, P, P, ctypes.c_int64, P, P,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P,
                                      ctypes.c_int]
        lib.oracle_direct.restype = None
        lib.oracle_far_images.argtypes = [ctypes.c_int64, P, P, ctypes.c_int64, P, P, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int]
        lib.oracle_far_images.restype = ctypes.c_int
        lib.oracle_cutoff_q.argtypes = [ctypes.c_double]
        lib.oracle_cutoff_q.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def cutoff_q(rho):
    """q(rho) of Eq. (cutoff) (scalar)."""
    return _load().oracle_cutoff_q(float(rho))


def direct(x, gamma, sigma, L=2 * np.pi, K=1, targets=None, kmin=0, grad=False,
           xt=None, gt=None, nthreads=0):
    """Direct FP64 sum of u and S (and optionally grad u) at targets.

    x, gamma: (N, 3) sources.  targets: particle indices used as targets (self pair
    excluded), default all.  xt/gt: explicit target positions/strengths (no self
    exclusion) instead of ``targets``.  Image boxes n with kmin <= max|n_i| <= K.
    Returns (u, S) or (u, S, G) with G[i] = du_a/dx_k as a 3x3 matrix.
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    if xt is None:
        tid = (np.arange(len(x), dtype=np.int64) if targets is None
               else np.ascontiguousarray(targets, dtype=np.int64))
        xt = np.ascontiguousarray(x[tid])
        gt = np.ascontiguousarray(g[tid])
    else:
        xt = np.ascontiguousarray(xt, dtype=np.float64)
        gt = (np.zeros_like(xt) if gt is None else np.ascontiguousarray(gt, dtype=np.float64))
        tid = np.full(len(xt), -1, dtype=np.int64)
    nt = len(xt)
    u = np.zeros((nt, 3))
    S = np.zeros((nt, 3))
    G = np.zeros((nt, 3, 3)) if grad else None
    lib.oracle_direct(len(x), _p(x), _p(g), nt, _p(xt), _p(gt),
                      tid.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                      float(sigma), float(L), int(kmin), int(K), _p(u), _p(S),
                      _p(G) if grad else ctypes.POINTER(ctypes.c_double)(), int(nthreads))
    return (u, S, G) if grad else (u, S)


def far_images(x, gamma, xt, gt, sigma, L=2 * np.pi, kmin=2, K=13, nthreads=0):
    """Far-image increment: the image boxes kmin <= max|n_i| <= K of the cube sum at explicit
    targets (xt, gt), kmin >= 2, where every pair is at least 10 sigma apart so that the
    definition reduces exactly to the singular kernel (``oracle_far_images`` in direct.c).
    direct(..., K=1) + far_images(..., kmin=2, K=13) is the 27^3-box sum of Section 4.1.
    Returns (u, S)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    xt = np.ascontiguousarray(xt, dtype=np.float64)
    gt = np.ascontiguousarray(gt, dtype=np.float64)
    u = np.zeros((len(xt), 3))
    S = np.zeros((len(xt), 3))
    rc = lib.oracle_far_images(len(x), _p(x), _p(g), len(xt), _p(xt), _p(gt), float(sigma), float(L),
                               int(kmin), int(K), _p(u), _p(S), int(nthreads))
    if rc != 0:
        raise ValueError("far_images needs kmin >= 2 and (kmin - 1) L >= 10 sigma")
    return u, S


from . import spectral  # noqa: E402,F401
from . import gradient  # noqa: E402,F401
from . import integrate  # noqa: E402,F401
from . import reinit  # noqa: E402,F401
from . import diagnostics  # noqa: E402,F401
