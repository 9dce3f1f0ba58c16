"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the lattice Boltzmann arithmetic: it only produces
macroscopic initial fields (density rho and velocity u at integer node
coordinates) and plain random numbers.  Both the CUDA path and the CPU oracle
turn these into populations with their own equilibrium code.

Workloads (the paper measures on no public dataset; these stand in for its
flows):

* ``taylor_green_2d``  -- periodic 2D Taylor-Green vortex, k = 2 pi / L,
  u_x = u0 sin(kx) cos(ky), u_y = -u0 cos(kx) sin(ky),
  rho = rho0 - (3 rho0 u0^2 / 4)(cos 2kx + cos 2ky)  (pressure p = rho/3).
* ``taylor_green_3d``  -- periodic 3D Taylor-Green vortex on [0, 2 pi)^3,
  u = u0 sin x cos y cos z, v = -u0 cos x sin y cos z, w = 0,
  rho = rho0 + 3 rho0 (u0^2/16)(cos 2x + cos 2y)(cos 2z + 2).
* ``shear_layer_2d``   -- the doubly periodic shear layer of Sec. IV
  (w = delta = 0.05): u_x = U0 tanh((4y-1)/w) for y <= 1/2 and
  U0 tanh((3-4y)/w) above, u_y = U0 delta sin(2 pi (x + 1/4)), x = i/L, y = j/L.
* ``random_vortex_2d`` -- random-phase streamfunction with a Gaussian shell
  spectrum peaked at |k| = k0, u = curl psi, rescaled to a target rms speed.
* ``population_noise`` -- multiplicative factors 1 + eps * U(-1, 1) used to push
  equilibrium populations off equilibrium in parity tests (one amplitude for all
  nodes, or one per node).

Every generator takes integer node coordinates so that a sub-box of a large
field can be regenerated exactly; ``grid`` builds the full coordinate arrays.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20221203


def grid(dims):
    """Integer coordinate arrays (x, y, z) of shape (nz, ny, nx), flattened in
    the node order n = (z*ny + y)*nx + x."""
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def taylor_green_2d(ix, iy, L, u0=0.01, rho0=1.0):
    k = 2.0 * np.pi / L
    X = k * np.asarray(ix, dtype=np.float64)
    Y = k * np.asarray(iy, dtype=np.float64)
    ux = u0 * np.sin(X) * np.cos(Y)
    uy = -u0 * np.cos(X) * np.sin(Y)
    rho = rho0 - 0.75 * rho0 * u0 * u0 * (np.cos(2 * X) + np.cos(2 * Y))
    return rho, np.stack([ux, uy])


def taylor_green_3d(ix, iy, iz, L, u0=0.05, rho0=1.0):
    k = 2.0 * np.pi / L
    X = k * np.asarray(ix, dtype=np.float64)
    Y = k * np.asarray(iy, dtype=np.float64)
    Z = k * np.asarray(iz, dtype=np.float64)
    ux = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz = np.zeros_like(ux)
    p = rho0 * u0 * u0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    rho = rho0 + 3.0 * p
    return rho, np.stack([ux, uy, uz])


def shear_layer_2d(ix, iy, L, U0=0.04, w=0.05, delta=0.05, rho0=1.0):
    x = np.asarray(ix, dtype=np.float64) / L
    y = np.asarray(iy, dtype=np.float64) / L
    ux = np.where(y <= 0.5, U0 * np.tanh((4 * y - 1) / w), U0 * np.tanh((3 - 4 * y) / w))
    uy = U0 * delta * np.sin(2 * np.pi * (x + 0.25))
    rho = np.full_like(ux, rho0)
    return rho, np.stack([ux, uy])


def random_vortex_2d(L, rms=0.03, k0=4.0, seed=DEFAULT_SEED, rho0=1.0):
    """Full L x L field (node order n = y*L + x) from a random-phase streamfunction."""
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(L, d=1.0 / L)
    KX, KY = np.meshgrid(kx, kx, indexing="xy")
    kk = np.sqrt(KX ** 2 + KY ** 2)
    amp = np.exp(-0.5 * (kk - k0) ** 2)
    amp[0, 0] = 0.0
    phase = np.exp(2j * np.pi * rng.random((L, L)))
    psi = np.real(np.fft.ifft2(amp * phase))
    # u = (d psi / dy, -d psi / dx) by spectral differentiation (unit box).
    psi_h = np.fft.fft2(psi)
    ux = np.real(np.fft.ifft2(1j * KY * psi_h))
    uy = np.real(np.fft.ifft2(-1j * KX * psi_h))
    s = rms / np.sqrt(np.mean(ux ** 2 + uy ** 2))
    ux, uy = ux * s, uy * s
    rho = np.full(L * L, rho0)
    return rho, np.stack([ux.ravel(), uy.ravel()])


def random_state_2d(L, rms=0.05, seed=DEFAULT_SEED):
    """Spatially random (white) density and velocity: rho in 1 +- 0.05, |u| ~ rms."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * (2 * rng.random(L * L) - 1)
    u = rms * rng.standard_normal((2, L * L))
    return rho, u


def population_noise(Q, N, eps, seed=DEFAULT_SEED):
    """Factors 1 + eps * U(-1, 1), shape (Q, N); eps a number or one amplitude per node."""
    rng = np.random.default_rng(seed)
    return 1.0 + eps * (2.0 * rng.random((Q, N)) - 1.0)
