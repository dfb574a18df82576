"""Jacobian-vector products of the discrete residual (oracle; test infrastructure).

* ``jvp_complex_step`` -- the Gateaux derivative of Eq. 6, d/de F(x + e v) at
  e = 0, computed as Im F(x + i h v) / h with h = 1e-30 (the complex-step
  derivative of Squire and Trapp, 1998). It has no subtractive cancellation,
  so it reaches the exact derivative of the implemented residual to rounding,
  which is what forward-mode AD returns (Eq. 9). It shares nothing with the
  dual-number arithmetic of the CUDA path.
* ``jvp_fd`` -- the forward-difference quotient of Eq. 7.
* ``fd_eps_paper`` / ``fd_eps_scaled`` -- the perturbation size of Eq. 8,
  sqrt(eps_mach) * max(1, ||x||), and the scaled rule
  sqrt(eps_mach) * (1 + ||x||) / ||v|| of the 1D Burgers benchmark.
* ``dense_jacobian`` -- J assembled column by column with the complex step.
"""
from __future__ import annotations

import math

import numpy as np

CS_STEP = 1e-30


def jvp_complex_step(F, x: np.ndarray, v: np.ndarray, h: float = CS_STEP):
    """Return (F(x), J(x) v) for a residual F written with complex-safe numpy (Eq. 6, Eq. 9)."""
    z = F(x.astype(np.complex128) + 1j * h * v)
    return z.real.copy(), z.imag / h


def fd_eps_paper(x: np.ndarray, eps_mach: float = np.finfo(np.float64).eps) -> float:
    """Eq. 8: sqrt(eps_mach) * max(1, ||x||_2)."""
    return math.sqrt(float(eps_mach)) * max(1.0, float(np.linalg.norm(x)))


def fd_eps_scaled(x: np.ndarray, v: np.ndarray, eps_mach: float = np.finfo(np.float64).eps) -> float:
    """Scaled rule sqrt(eps_mach) * (1 + ||x||_2) / ||v||_2 (requires v != 0)."""
    nv = float(np.linalg.norm(v))
    if nv == 0.0:
        raise ValueError("scaled FD step needs a nonzero direction")
    return math.sqrt(float(eps_mach)) * (1.0 + float(np.linalg.norm(x))) / nv


def jvp_fd(F, x: np.ndarray, v: np.ndarray, eps: float, Fx: np.ndarray | None = None):
    """Eq. 7: (F(x + eps v) - F(x)) / eps, in the dtype of x."""
    if Fx is None:
        Fx = F(x)
    e = x.dtype.type(eps)
    return (F(x + e * v) - Fx) / e


def dense_jacobian(F, x: np.ndarray) -> np.ndarray:
    """Dense J with J[:, c] = J e_c by the complex step (small problems only)."""
    n = x.size
    J = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        J[:, c] = jvp_complex_step(F, x, e)[1]
    return J
