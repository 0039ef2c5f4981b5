"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the benchmark.

This module holds no Biot-Savart or FMM arithmetic: it only builds the particle
set (positions, strengths, core size) that both sides consume.

Construction (Section 4.2, Eq. initspec of the paper; where the paper is silent the
readings are stated per item below):

* particles sit at the centres of an n^3 lattice in [0, 2*pi)^3, x = (i + 1/2) h,
  h = 2*pi/n (the paper places vortex elements between spectral grid points);
* the velocity is a random-phase solenoidal Fourier field whose integer shells carry
  E(k) proportional to k^4 exp(-2 k^2 / k0^2), normalised to unit kinetic energy
  0.5 <|u|^2> = 1;
* vorticity is the exact spectral curl omega = i k x u_hat, and the strengths are
  alpha = omega(x) h^3 (the paper's own initial guess for the RBF solve, Section 5.2);
* the core size is sigma = (sigma/h) * h.

Everything is FP64 numpy and deterministic per (n, k0, seed).
"""
from .field import (lattice_positions, solenoidal_modes, make_vortex_lattice,
                    lattice_velocity, viscosity_for_re_lambda, target_subset, jitter)

__all__ = ["lattice_positions", "solenoidal_modes", "make_vortex_lattice",
           "lattice_velocity", "viscosity_for_re_lambda", "target_subset", "jitter"]
