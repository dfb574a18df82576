"""Matrix-free Krylov solvers (oracle; test infrastructure).

The Newton system J dx = -F (Eq. 4) is solved with the operator seen only as
v -> J v (Sec. 3.1). All solvers start from x0 = 0, so the initial residual
of Eq. 10 is r0 = b, and stop on the relative residual ||r|| <= tol ||b||
(relative tolerance semantics of the SciPy/CuPy solvers the paper drives).

* ``gmres``    restarted GMRES(m) (Saad and Schultz): Arnoldi with classical
               Gram-Schmidt applied twice (CGS2), Givens rotations on the
               Hessenberg matrix, least-squares update at the end of a cycle,
               at most ``max_cycles`` restart cycles (the paper's Krylov cap
               counts restart cycles for GMRES, Sec. 3.3).
* ``gmres_dcgs2`` the same GMRES(m) with the second Gram-Schmidt pass of each
               Arnoldi vector delayed by one step (delayed CGS2, Swirydowicz et
               al. 2020; Bielich et al. 2022), so that one set of inner products
               per step serves both passes. Same Krylov space, basis and
               iterates as CGS2 in exact arithmetic.
* ``bicgstab`` van der Vorst's BiCGSTAB with shadow residual r_hat = r0.
* ``cg``       Hestenes-Stiefel conjugate gradients for SPD systems.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class KrylovResult:
    x: np.ndarray
    iterations: int          # Arnoldi steps (GMRES) or iterations (BiCGSTAB, CG)
    matvecs: int             # every operator application, restarts included
    converged: bool
    breakdown: bool
    resid_est: float         # last residual estimate (Givens for GMRES, recurrence otherwise)


def givens(f: float, g: float):
    """Rotation (c, s) with [c s; -s c] [f; g] = [r; 0], r = hypot(f, g) >= 0.

    c = f / r, s = g / r; the identity rotation when f = g = 0.
    """
    r = float(np.hypot(f, g))
    if r == 0.0:
        return 1.0, 0.0
    return f / r, g / r


def gmres(A, b: np.ndarray, m: int, tol: float, max_cycles: int) -> KrylovResult:
    """Restarted GMRES(m) with CGS2 Arnoldi, starting from x = 0."""
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    its = 0
    mv = 0
    if bnorm == 0.0:
        return KrylovResult(x, 0, 0, True, False, 0.0)
    target = tol * bnorm
    resid = bnorm
    for cycle in range(max_cycles):
        if cycle == 0:
            r = b.copy()
        else:
            r = b - A(x)
            mv += 1
        beta = float(np.linalg.norm(r))
        resid = beta
        if beta <= target:
            return KrylovResult(x, its, mv, True, False, beta)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        done = False
        for j in range(m):
            w = A(V[j])
            mv += 1
            its += 1
            # classical Gram-Schmidt, applied twice
            h1 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h1
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            H[: j + 1, j] = h1 + h2
            hn = float(np.linalg.norm(w))
            H[j + 1, j] = hn
            # previous rotations, then the new one
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            resid = abs(g[j + 1])
            if resid <= target or hn == 0.0:
                done = True
                break
            V[j + 1] = w / hn
        # back substitution H[:k,:k] y = g[:k] (upper triangular after the rotations)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:k].T @ y
        if not np.all(np.isfinite(x)):
            return KrylovResult(x, its, mv, False, True, float("nan"))
        if done:
            return KrylovResult(x, its, mv, resid <= target, False, resid)
    return KrylovResult(x, its, mv, False, False, resid)


def gmres_dcgs2(A, b: np.ndarray, m: int, tol: float, max_cycles: int) -> KrylovResult:
    """Restarted GMRES(m) with delayed CGS2 Arnoldi, starting from x = 0.

    Step j holds a candidate u_j that has been projected once against
    q_0 .. q_{j-1} but neither projected a second time nor normalised; it is
    scaled to unit length (ut = u_j / ||u_j||) and the operator is applied to
    it, w = A ut. One set of inner products, s = Q^T ut, alpha = ut.ut,
    t = Q^T w, beta = ut.w, then gives
      * the second projection of the candidate: rho^2 = alpha - s.s is the
        squared norm of ut - Q s, q_j = (ut - Q s) / rho, and column j-1 of
        the Hessenberg matrix is completed as (first projection + s / sigma,
        rho / sigma) with sigma = 1 / ||u_j||, rotated and tested for
        convergence (one step after CGS2 would);
      * the first projection of A q_j: A q_j = (w - A Q s) / rho with
        A Q = Q_{j+1} H[:j+1, :j] (the completed columns), so
        h_i = (t_i - z_i) / rho for i < j and h_j = ((beta - s.t)/rho - z_j)/rho
        with z = H[:j+1, :j] s;
      * the next candidate u_{j+1} = A q_j - Q_{j+1} h.
    The last column of a cycle is completed by the inner products of u_m alone.
    """
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    its = 0
    mv = 0
    if bnorm == 0.0:
        return KrylovResult(x, 0, 0, True, False, 0.0)
    target = tol * bnorm
    resid = bnorm
    for cycle in range(max_cycles):
        if cycle == 0:
            r = b.copy()
        else:
            r = b - A(x)
            mv += 1
        beta0 = float(np.linalg.norm(r))
        resid = beta0
        if beta0 <= target:
            return KrylovResult(x, its, mv, True, False, beta0)
        Q = np.zeros((m + 1, n))
        Hraw = np.zeros((m + 1, m))      # completed columns, before rotation
        H = np.zeros((m + 1, m))         # the same columns, rotated
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        u = r
        sigma = 1.0 / beta0
        hprev = None
        k = 0
        done = False
        for j in range(m + 1):
            ut = sigma * u
            s = Q[:j] @ ut
            alpha = float(ut @ ut)
            if j < m:
                w = A(ut)
                mv += 1
                t = Q[:j] @ w
                bt = float(ut @ w)
            rho2 = alpha - float(s @ s)
            rho = float(np.sqrt(rho2)) if rho2 > 0.0 else 0.0
            if j == 0:
                g[0] = beta0 * rho       # r = beta0 * rho * q_0
            else:
                # complete column j-1, rotate it, test: A q_{j-1} = Q h + u_j and
                # u_j = ut / sigma = (Q s + rho q_j) / sigma
                c_ = j - 1
                Hraw[:j, c_] = hprev[:j] + s / sigma
                Hraw[j, c_] = rho / sigma
                H[: j + 1, c_] = Hraw[: j + 1, c_]
                for i in range(c_):
                    tt = cs[i] * H[i, c_] + sn[i] * H[i + 1, c_]
                    H[i + 1, c_] = -sn[i] * H[i, c_] + cs[i] * H[i + 1, c_]
                    H[i, c_] = tt
                cs[c_], sn[c_] = givens(H[c_, c_], H[c_ + 1, c_])
                H[c_, c_] = cs[c_] * H[c_, c_] + sn[c_] * H[c_ + 1, c_]
                H[c_ + 1, c_] = 0.0
                g[c_ + 1] = -sn[c_] * g[c_]
                g[c_] = cs[c_] * g[c_]
                its += 1
                k = j
                resid = abs(g[c_ + 1])
                if resid <= target or rho == 0.0:
                    done = True
                    break
                if j == m:
                    break
            Q[j] = (ut - Q[:j].T @ s) / rho
            z = Hraw[: j + 1, :j] @ s
            h = np.empty(j + 1)
            h[:j] = (t - z[:j]) / rho
            h[j] = ((bt - float(s @ t)) / rho - z[j]) / rho
            hprev = h
            u = (w - Q[: j + 1].T @ (z + rho * h)) / rho
            un = float(np.linalg.norm(u))
            sigma = 1.0 / un if un > 0.0 else 0.0
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Q[:k].T @ y
        if not np.all(np.isfinite(x)):
            return KrylovResult(x, its, mv, False, True, float("nan"))
        if done:
            return KrylovResult(x, its, mv, resid <= target, False, resid)
    return KrylovResult(x, its, mv, False, False, resid)


def bicgstab(A, b: np.ndarray, tol: float, maxiter: int) -> KrylovResult:
    """BiCGSTAB (van der Vorst, 1992) from x = 0 with r_hat = r0 = b."""
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return KrylovResult(x, 0, 0, True, False, 0.0)
    target = tol * bnorm
    r = b.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros(n)
    p = np.zeros(n)
    mv = 0
    resid = bnorm
    for it in range(1, maxiter + 1):
        rho = float(rhat @ r)
        if rho == 0.0 or not np.isfinite(rho):
            return KrylovResult(x, it - 1, mv, False, True, resid)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        mv += 1
        rv = float(rhat @ v)
        if rv == 0.0 or not np.isfinite(rv):
            return KrylovResult(x, it, mv, False, True, resid)
        alpha = rho / rv
        s = r - alpha * v
        snorm = float(np.linalg.norm(s))
        if snorm <= target:
            x = x + alpha * p
            return KrylovResult(x, it, mv, True, False, snorm)
        t = A(s)
        mv += 1
        tt = float(t @ t)
        if tt == 0.0 or not np.isfinite(tt):
            return KrylovResult(x, it, mv, False, True, resid)
        omega = float(t @ s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        resid = float(np.linalg.norm(r))
        if resid <= target:
            return KrylovResult(x, it, mv, True, False, resid)
        if omega == 0.0:
            return KrylovResult(x, it, mv, False, True, resid)
        rho_old = rho
    return KrylovResult(x, maxiter, mv, False, False, resid)


def cg(A, b: np.ndarray, tol: float, maxiter: int) -> KrylovResult:
    """Conjugate gradients (Hestenes and Stiefel, 1952) from x = 0."""
    n = b.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return KrylovResult(x, 0, 0, True, False, 0.0)
    target = tol * bnorm
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    mv = 0
    for it in range(1, maxiter + 1):
        q = A(p)
        mv += 1
        pq = float(p @ q)
        if pq == 0.0 or not np.isfinite(pq):
            return KrylovResult(x, it, mv, False, True, float(np.sqrt(rr)))
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        if np.sqrt(rr_new) <= target:
            return KrylovResult(x, it, mv, True, False, float(np.sqrt(rr_new)))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return KrylovResult(x, maxiter, mv, False, False, float(np.sqrt(rr)))
