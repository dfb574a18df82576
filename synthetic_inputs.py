"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only input generation: initial states, media and sources
drawn from fixed seeds. It contains none of the solver's arithmetic (no
residual, no derivative, no Krylov or Newton step), so that the CPU oracle
and the CUDA path can both consume the same inputs without sharing any code
of the method itself.

Layout of every state vector: one contiguous float64 array, field-major,
then row-major (y, x): index = f * ny * nx + j * nx + i. Cell centres of the
2D grids are at ((i + 1/2) / nx, (j + 1/2) / ny) on the unit square; the 1D
Burgers line has cells at x_i = i / N.
"""
from __future__ import annotations

import math

import numpy as np


def burgers_ic(N: int = 1024, seed: int = 0) -> np.ndarray:
    """Noisy sine wave for the 1D viscous Burgers step.

    u0_i = sin(2 pi x_i) + 0.1 * eta_i with x_i = i / N, where eta is standard
    normal noise from ``default_rng(seed)`` smoothed by three periodic passes
    of the (1, 2, 1) / 4 filter (damped Jacobi on the noise only).
    """
    rng = np.random.default_rng(seed)
    eta = rng.standard_normal(N)
    for _ in range(3):
        eta = 0.25 * (np.roll(eta, 1) + 2.0 * eta + np.roll(eta, -1))
    x = np.arange(N, dtype=np.float64) / N
    return np.sin(2.0 * math.pi * x) + 0.1 * eta


BURGERS2D_KINDS = ("tgv", "dsl", "4vc")

# Four-vortex collision layout: centres on the corners of a square of side
# 2 d around the domain centre, circulations of alternating sign going
# round it, all of the same magnitude.
VC4_R, VC4_D, VC4_GAMMA = 0.5, 1.0, 4.0


def burgers2d_ic(nx: int, ny: int | None = None, kind: str = "tgv", L: float = 2.0 * math.pi) -> np.ndarray:
    """Initial velocity [u, v] (flat) of the 2D Burgers benchmarks on the periodic square [0, L)^2.

    Nodes are at x_i = i L / nx, y_j = j L / ny (the grid of the 2D Burgers
    residual, unlike the cell-centred grids of the other 2D problems).
    Formulas for L = 2 pi (App. A, Burgers' Equation):

    * ``tgv``: Taylor-Green vortex u = sin x cos y, v = -cos x sin y.
    * ``dsl``: double shear layer, rho = 30, delta = 0.05:
      u = tanh(rho (y - pi/2)) for y <= pi, tanh(rho (3 pi/2 - y)) above;
      v = delta sin x.
    * ``4vc``: four Gaussian vortices of radius R = 0.5,
      U = sum_i Gamma_i (-(y - cy_i), x - cx_i) exp(-r_i^2 / R^2), with the
      centres (pi -+ 1, pi -+ 1) and Gamma = +4, -4, +4, -4 going round them
      (the paper gives R and the alternating signs only).
    """
    ny = nx if ny is None else ny
    x = np.arange(nx, dtype=np.float64) * (L / nx)
    y = np.arange(ny, dtype=np.float64) * (L / ny)
    X, Y = np.meshgrid(x, y)            # shape (ny, nx), row-major (y, x)
    pi = math.pi
    if kind == "tgv":
        u, v = np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)
    elif kind == "dsl":
        rho, delta = 30.0, 0.05
        u = np.where(Y <= pi, np.tanh(rho * (Y - pi / 2)), np.tanh(rho * (3 * pi / 2 - Y)))
        v = delta * np.sin(X)
    elif kind == "4vc":
        c, d = L / 2.0, VC4_D
        centres = ((c - d, c - d), (c + d, c - d), (c + d, c + d), (c - d, c + d))
        u = np.zeros_like(X)
        v = np.zeros_like(X)
        for k, (cx, cy) in enumerate(centres):
            g = VC4_GAMMA * (1.0 if k % 2 == 0 else -1.0)
            ex = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / VC4_R ** 2)
            u += -g * (Y - cy) * ex
            v += g * (X - cx) * ex
    else:
        raise ValueError(f"unknown 2D Burgers initial condition {kind!r}")
    return np.concatenate([u.reshape(-1), v.reshape(-1)])


RD_KINDS = ("gaussian", "multigauss", "sinusoidal")


def rd_ic(nx: int, ny: int | None = None, kind: str = "gaussian") -> np.ndarray:
    """Initial concentration of the paper's reaction-diffusion benchmark (App. A), flat, on the
    interior nodes x_i = -1/2 + (i + 1) / (nx + 1) of the square [-1/2, 1/2]^2 (u = 0 on its boundary).

    * ``gaussian``: exp(-r^2 / s^2), s = 0.1, centred at the origin.
    * ``multigauss``: four such peaks (s = 0.08) centred at (+-0.2, +-0.2).
    * ``sinusoidal``: |sin(kx pi x) sin(ky pi y)| with kx = ky = 4 (even, so zero on the walls).
    The paper names the three profiles and the sinusoidal formula; widths, centres and wave
    numbers are this module's choice.
    """
    ny = nx if ny is None else ny
    x = -0.5 + np.arange(1, nx + 1, dtype=np.float64) / (nx + 1)
    y = -0.5 + np.arange(1, ny + 1, dtype=np.float64) / (ny + 1)
    X, Y = np.meshgrid(x, y)
    if kind == "gaussian":
        u = np.exp(-(X * X + Y * Y) / 0.1 ** 2)
    elif kind == "multigauss":
        u = np.zeros_like(X)
        for cx in (-0.2, 0.2):
            for cy in (-0.2, 0.2):
                u += np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / 0.08 ** 2)
    elif kind == "sinusoidal":
        u = np.abs(np.sin(4 * math.pi * X) * np.sin(4 * math.pi * Y))
    else:
        raise ValueError(f"unknown reaction-diffusion initial condition {kind!r}")
    return u.reshape(-1)


def allen_cahn_ic(nx: int, ny: int | None = None, seed: int = 0) -> np.ndarray:
    """Uniform noise in [-0.1, 0.1] on an nx x ny periodic grid (flat, row-major)."""
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.1, 0.1, size=ny * nx).astype(np.float64)


def su_olson_ic(nx: int, ny: int | None = None, E0: float = 1e-6, a: float = 1.0) -> np.ndarray:
    """Cold start in equilibrium: E = E0 and a T^4 = E0 everywhere; returns [E, T] flat."""
    ny = nx if ny is None else ny
    n = nx * ny
    T0 = (E0 / a) ** 0.25
    return np.concatenate([np.full(n, E0), np.full(n, T0)])


def maxwell_medium(nx: int, ny: int | None = None, seed: int = 0, n_disc: int = 16,
                   r_lo: float = 0.02, r_hi: float = 0.08,
                   eps_lo: float = 1.0, eps_hi: float = 4.0) -> np.ndarray:
    """Piecewise-constant relative permittivity: background 1 plus random discs.

    Disc d has centre U[0,1]^2, radius U[r_lo, r_hi] and permittivity
    U[eps_lo, eps_hi], all drawn from ``default_rng(seed)`` in that order per
    disc; later discs overwrite earlier ones. Returns a flat (ny * nx) array.
    """
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    xc = (np.arange(nx) + 0.5) / nx
    yc = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(xc, yc)
    eps = np.ones((ny, nx))
    for _ in range(n_disc):
        cx, cy = rng.uniform(0.0, 1.0, size=2)
        r = rng.uniform(r_lo, r_hi)
        e = rng.uniform(eps_lo, eps_hi)
        eps[(X - cx) ** 2 + (Y - cy) ** 2 <= r * r] = e
    return eps.reshape(-1)


def maxwell_point_source(nx: int, ny: int | None = None) -> np.ndarray:
    """Point source of unit total strength at cell (nx // 2, ny // 2).

    Returns [f_re, f_im] flat (2 * ny * nx); f_re = 1 / (hx * hy) at that cell.
    """
    ny = nx if ny is None else ny
    f = np.zeros(2 * nx * ny)
    f[(ny // 2) * nx + nx // 2] = float(nx * ny)
    return f


MAXWELL_VEC_SOURCES = ("gauss", "dipole")


def maxwell_vec_source(nx: int, ny: int | None = None, kind: str = "gauss", sigma: float = 0.05,
                       x0: float = 0.5, y0: float = 0.5, sep: float = 0.1) -> np.ndarray:
    """The paper's applied currents J of the vector TE Maxwell problem on the node grid of the unit square
    (x_i = i/(nx - 1)): planes [Re Jx, Im Jx, Re Jy, Im Jy] with J_y = 0 and a real J_x,
      gauss:  J_x = exp(-((x - x0)^2 + (y - y0)^2) / (2 sigma^2)),
      dipole: J_x = exp(-((x - x0)^2 + (y - y1)^2) / (2 sigma^2)) - exp(-((x - x0)^2 + (y - y2)^2) / (2 sigma^2)),
    y1, y2 = y0 -+ sep. The paper does not give x0, the y's or sigma; these defaults are a reading of it."""
    ny = nx if ny is None else ny
    X, Y = np.meshgrid(np.arange(nx) / (nx - 1), np.arange(ny) / (ny - 1))
    g = lambda yc: np.exp(-((X - x0) ** 2 + (Y - yc) ** 2) / (2.0 * sigma * sigma))
    if kind == "gauss":
        jx = g(y0)
    elif kind == "dipole":
        jx = g(y0 - sep) - g(y0 + sep)
    else:
        raise ValueError(kind)
    z = np.zeros(nx * ny)
    return np.concatenate([jx.reshape(-1), z, z, z])


def maxwell_wavenumber(n: int, ppw: float = 10.0, eps_max: float = 4.0) -> float:
    """Wavenumber giving ``ppw`` cells per wavelength in the densest medium.

    k * sqrt(eps_max) * h = 2 pi / ppw with h = 1 / n.
    """
    return 2.0 * math.pi * n / (ppw * math.sqrt(eps_max))


def serving_requests(n_req: int, rate: float, seed: int = 0,
                     n_lo: int = 64, n_hi: int = 2048, tile: int = 64,
                     steps_hi: int = 20) -> list[dict]:
    """Poisson stream of mixed solves (arrival time, PDE, grid, steps, precision).

    Inter-arrival gaps are exponential with mean 1 / rate seconds. The PDE is
    uniform over the three 2D problems, the side n is log-uniform in
    [n_lo, n_hi] rounded down to a multiple of ``tile``, the step count is
    uniform in 1..steps_hi and the precision is uniform over {"mixed", "fp64"}.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_req):
        t += rng.exponential(1.0 / rate)
        pde = ["allen_cahn", "su_olson", "maxwell"][int(rng.integers(0, 3))]
        n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
        n = max(tile, (n // tile) * tile)
        steps = int(rng.integers(1, steps_hi + 1))
        prec = ["mixed", "fp64"][int(rng.integers(0, 2))]
        out.append({"id": r, "t_arrival": t, "pde": pde, "n": n, "steps": steps,
                    "precision": prec, "seed": int(rng.integers(0, 2**31 - 1))})
    return out
