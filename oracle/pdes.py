"""Discrete residuals of the benchmark PDEs (oracle; test infrastructure).

Each problem maps a flat state x (field-major, then row-major y, x) to the
spatial operator G(x). Every function works unchanged on complex arrays so
that ``oracle.jvp`` can differentiate it by the complex step: branches test
the real part only and no non-analytic function (abs, max) is applied to a
quantity that carries a derivative.

The nonlinear system of one implicit step is the theta-method residual of
Eq. 2 (x^k the Newton iterate, x* = x^n the previous state),

    F(x; b) = M(x) - theta * dt * G(x) - b,
    b       = M(x^n) + (1 - theta) * dt * G(x^n),

with M the identity except for the radiation problem, where the material
unknown T enters through its energy a T^4. theta = 1/2 is the paper's
Crank-Nicolson scheme (Sec. 3.2, App. A); theta = 1 is backward Euler. The
Maxwell problem is a boundary-value problem: F(x) = G(x).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _lap5_periodic(u: np.ndarray, hx: float, hy: float) -> np.ndarray:
    """Second-order 5-point Laplacian with periodic wrap; u has shape (ny, nx)."""
    return ((np.roll(u, -1, axis=1) - 2.0 * u + np.roll(u, 1, axis=1)) / (hx * hx)
            + (np.roll(u, -1, axis=0) - 2.0 * u + np.roll(u, 1, axis=0)) / (hy * hy))


class _ThetaProblem:
    """Shared theta-method plumbing (Eq. 2 with a one-step time scheme)."""

    bvp = False
    theta = 0.5
    dt = 0.1

    def M(self, x):
        return x

    def rhs(self, xn):
        """b = M(x^n) + (1 - theta) dt G(x^n), the constant part of F."""
        return self.M(xn) + (1.0 - self.theta) * self.dt * self.G(xn)

    def residual(self, x, b):
        """F(x; b) = M(x) - theta dt G(x) - b."""
        if self.bvp:
            return self.G(x)
        return self.M(x) - self.theta * self.dt * self.G(x) - b


@dataclass
class Burgers1D(_ThetaProblem):
    """1D viscous Burgers u_t + (u^2/2)_x = nu u_xx on the periodic unit line.

    Cells x_i = i h, h = 1/N. Conservative upwind convection: the face flux
    Phi_{i+1/2} takes u_i^2/2 when the face speed (u_i + u_{i+1})/2 is >= 0 and
    u_{i+1}^2/2 otherwise (this is the Roe flux for Burgers); diffusion is the
    3-point central second difference. The paper's Burgers benchmark is the
    2D central-difference form (App. A, Burgers' Equation); this is the 1D
    upwind variant of the benchmark configuration, with theta = 1.
    """

    N: int = 1024
    nu: float = 1e-2
    dt: float = 1e-3
    theta: float = 1.0

    @property
    def n_unknowns(self) -> int:
        return self.N

    def G(self, u):
        h = 1.0 / self.N
        up = np.roll(u, -1)   # u_{i+1}
        um = np.roll(u, 1)    # u_{i-1}
        face_speed = (u + up).real
        phi_p = np.where(face_speed >= 0.0, 0.5 * u * u, 0.5 * up * up)  # Phi_{i+1/2}
        phi_m = np.roll(phi_p, 1)                                        # Phi_{i-1/2}
        return -(phi_p - phi_m) / h + self.nu * (up - 2.0 * u + um) / (h * h)


def _dc_periodic(u: np.ndarray, h: float, axis: int) -> np.ndarray:
    """Second-order central first difference (u_{i+1} - u_{i-1}) / 2h with periodic wrap."""
    return (np.roll(u, -1, axis=axis) - np.roll(u, 1, axis=axis)) / (2.0 * h)


@dataclass
class Burgers2D(_ThetaProblem):
    """2D viscous Burgers U_t + (U . grad) U = nu lap U, U = (u, v), on the periodic square [0, L)^2.

    App. A, Burgers' Equation: the advection Adv(U) = u D_x U + v D_y U with
    second-order central first differences and the diffusion Lap(U) with the
    5-point Laplacian, both on nodes x_i = i hx, y_j = j hy (hx = L/nx,
    hy = L/ny). With theta = 1/2 the residual F = U - theta dt G(U) - b,
    G = -Adv + nu Lap, is the paper's Crank-Nicolson residual of that passage.

    ``courant`` > 0 makes dt adaptive: before each implicit step the time step
    is set from the state x^n by the CFL rule of the same passage,
        dt = C min(hx / max|u|, hy / max|v|, 1 / (2 nu (1/hx^2 + 1/hy^2))),
    a term with max|.| = 0 dropped (``cfl_dt``). ``courant`` = 0 keeps dt.
    """

    nx: int = 64
    ny: int = 64
    nu: float = 0.05
    dt: float = 1e-2
    theta: float = 0.5
    L: float = 2.0 * np.pi
    courant: float = 0.0

    @property
    def n_unknowns(self) -> int:
        return 2 * self.nx * self.ny

    @property
    def spacing(self):
        return self.L / self.nx, self.L / self.ny

    def G(self, x):
        n = self.nx * self.ny
        u = x[:n].reshape(self.ny, self.nx)
        v = x[n:].reshape(self.ny, self.nx)
        hx, hy = self.spacing
        out = []
        for w in (u, v):
            adv = u * _dc_periodic(w, hx, 1) + v * _dc_periodic(w, hy, 0)
            out.append((-adv + self.nu * _lap5_periodic(w, hx, hy)).reshape(-1))
        return np.concatenate(out)

    def cfl_dt(self, x) -> float:
        n = self.nx * self.ny
        hx, hy = self.spacing
        cands = [1.0 / (2.0 * self.nu * (1.0 / hx ** 2 + 1.0 / hy ** 2))] if self.nu > 0 else []
        umax, vmax = float(np.abs(x[:n]).max()), float(np.abs(x[n:]).max())
        if umax > 0.0:
            cands.append(hx / umax)
        if vmax > 0.0:
            cands.append(hy / vmax)
        return self.courant * min(cands)

    def rhs(self, xn):
        if self.courant > 0.0:
            self.dt = self.cfl_dt(xn)
        return super().rhs(xn)


def _lap5_dirichlet(u: np.ndarray, hx: float, hy: float) -> np.ndarray:
    """5-point Laplacian on interior nodes with u = 0 on the boundary nodes; u has shape (ny, nx)."""
    p = np.zeros((u.shape[0] + 2, u.shape[1] + 2), dtype=u.dtype)
    p[1:-1, 1:-1] = u
    return ((p[1:-1, 2:] - 2.0 * u + p[1:-1, :-2]) / (hx * hx)
            + (p[2:, 1:-1] - 2.0 * u + p[:-2, 1:-1]) / (hy * hy))


@dataclass
class AllenCahn2D(_ThetaProblem):
    """Allen-Cahn u_t = D lap u + u - u^3 with a 5-point Laplacian.

    The benchmark variant of the paper's reaction-diffusion problem
    (Sec. 3.2; App. A, Nonlinear Reaction-Diffusion), which has the sink
    -u^3 only; ``linear_coef`` = 1 adds the Allen-Cahn +u term and 0 recovers
    the paper's form D lap u - u^3.

    ``dirichlet`` = False: the periodic unit square, cells of width 1/nx.
    ``dirichlet`` = True: the paper's walls, u = 0 on the boundary of the
    square [-1/2, 1/2]^2; the unknowns are the interior nodes
    x_i = -1/2 + (i + 1) h, h = 1/(nx + 1) (and likewise in y).
    """

    nx: int = 64
    ny: int = 64
    D: float = 1e-3
    dt: float = 0.1
    theta: float = 0.5
    linear_coef: float = 1.0
    dirichlet: bool = False

    @property
    def n_unknowns(self) -> int:
        return self.nx * self.ny

    @property
    def spacing(self):
        if self.dirichlet:
            return 1.0 / (self.nx + 1), 1.0 / (self.ny + 1)
        return 1.0 / self.nx, 1.0 / self.ny

    def G(self, x):
        u = x.reshape(self.ny, self.nx)
        hx, hy = self.spacing
        lap = _lap5_dirichlet(u, hx, hy) if self.dirichlet else _lap5_periodic(u, hx, hy)
        g = self.D * lap + self.linear_coef * u - u * u * u
        return g.reshape(-1)


@dataclass
class SuOlson2D(_ThetaProblem):
    """Two-field radiation diffusion with a flux limiter and a Marshak boundary.

    Unknowns (E, T) on the unit square, cell-centred, nx x ny cells.
      radiation:  dE/dt       = div(D(E) grad E) - sigma (E - a T^4)
      material:   d(a T^4)/dt = sigma (E - a T^4)       (c_v = 4 a T^3)
    Face diffusion coefficient D_f = 1 / (3 sigma + R_f) with
    R_f = sqrt(|grad E|_f^2 / Ebar_f^2 + rho^2): the normal difference across
    the face, the tangential difference averaged over the four cells that
    touch the face (mirror values beyond the wall), Ebar_f the mean of the two
    cells. ``limiter=False`` gives D = 1 / (3 sigma), the linear diffusion of
    the paper's Su-Olson system (Sec. 3.2; App. A, Su-Olson).
    Boundaries: the left wall carries the Marshak condition
    E/4 - (D_b/2) dE/dn = a T_b^4 / 4 with D_b = 1/(3 sigma), discretised
    between the wall and the first cell centre, giving the inward flux
    q = 2 D_b (4 F_inc - E_0) / (h + 4 D_b), F_inc = a T_b^4 / 4; the other
    three walls carry zero flux.
    """

    nx: int = 64
    ny: int = 64
    sigma: float = 1.0
    a: float = 1.0
    Tb: float = 1.0
    rho: float = 1e-6
    limiter: bool = True
    dt: float = 1e-3
    theta: float = 0.5

    @property
    def n_unknowns(self) -> int:
        return 2 * self.nx * self.ny

    def _split(self, x):
        n = self.nx * self.ny
        return x[:n].reshape(self.ny, self.nx), x[n:].reshape(self.ny, self.nx)

    def M(self, x):
        E, T = self._split(x)
        return np.concatenate([E.reshape(-1), (self.a * T ** 4).reshape(-1)])

    def _face_coef(self, gn, gt, Ebar):
        if not self.limiter:
            return 1.0 / (3.0 * self.sigma) + 0.0 * gn
        R = np.sqrt((gn * gn + gt * gt) / (Ebar * Ebar) + self.rho * self.rho)
        return 1.0 / (3.0 * self.sigma + R)

    def marshak_flux(self, E0col):
        """Inward flux through the left wall for first-column values E0col."""
        hx = 1.0 / self.nx
        Db = 1.0 / (3.0 * self.sigma)
        Finc = 0.25 * self.a * self.Tb ** 4
        return 2.0 * Db * (4.0 * Finc - E0col) / (hx + 4.0 * Db)

    def diffusion(self, E):
        """div(D(E) grad E) with the wall conditions above; E has shape (ny, nx)."""
        ny, nx = E.shape
        hx, hy = 1.0 / nx, 1.0 / ny
        jp = np.minimum(np.arange(ny) + 1, ny - 1)
        jm = np.maximum(np.arange(ny) - 1, 0)
        ip = np.minimum(np.arange(nx) + 1, nx - 1)
        im = np.maximum(np.arange(nx) - 1, 0)
        # x faces between columns i and i+1 (i = 0 .. nx-2): shape (ny, nx-1)
        El, Er = E[:, :-1], E[:, 1:]
        gn = (Er - El) / hx
        Eu, Ed = E[jp, :], E[jm, :]
        gt = ((Eu[:, :-1] + Eu[:, 1:]) - (Ed[:, :-1] + Ed[:, 1:])) / (4.0 * hy)
        Fx_in = self._face_coef(gn, gt, 0.5 * (El + Er)) * gn     # D dE/dx at the face
        Fx = np.zeros((ny, nx + 1), dtype=E.dtype)
        Fx[:, 1:nx] = Fx_in
        Fx[:, 0] = -self.marshak_flux(E[:, 0])   # D dE/dx at x = 0 is minus the inward flux
        # y faces between rows j and j+1 (j = 0 .. ny-2): shape (ny-1, nx)
        Eb, Et = E[:-1, :], E[1:, :]
        gn = (Et - Eb) / hy
        Er_, El_ = E[:, ip], E[:, im]
        gt = ((Er_[:-1, :] + Er_[1:, :]) - (El_[:-1, :] + El_[1:, :])) / (4.0 * hx)
        Fy_in = self._face_coef(gn, gt, 0.5 * (Eb + Et)) * gn
        Fy = np.zeros((ny + 1, nx), dtype=E.dtype)
        Fy[1:ny, :] = Fy_in
        return (Fx[:, 1:] - Fx[:, :-1]) / hx + (Fy[1:, :] - Fy[:-1, :]) / hy

    def G(self, x):
        E, T = self._split(x)
        exch = self.sigma * (E - self.a * T ** 4)
        return np.concatenate([(self.diffusion(E) - exch).reshape(-1), exch.reshape(-1)])


@dataclass
class MaxwellTE2D(_ThetaProblem):
    """Scalar TE (E_z) Helmholtz with a Kerr term, as a real map on (Re E, Im E).

      G(E) = lap E + k^2 (eps_r + chi3 |E|^2) E - f

    5-point Laplacian on the unit square, nx x ny cells. First-order absorbing
    wall dE/dn = i k E (time factor e^{-i omega t}) imposed through a ghost
    value E_g = E_0 (1 + i k h/2) / (1 - i k h/2) beyond each wall. |E|^2 =
    Re^2 + Im^2 is not holomorphic in E, so the unknowns are the two real
    planes and the Jacobian is the real 2N x 2N one. This is the scalar
    variant of the paper's Kerr problem (Sec. 3.2; App. A, Time-Harmonic
    Maxwell's Equations in Kerr Media); a boundary-value problem, F = G.
    """

    nx: int = 64
    ny: int = 64
    k: float = 10.0
    chi3: float = 1e-3
    eps_r: np.ndarray = field(default=None, repr=False)
    f: np.ndarray = field(default=None, repr=False)
    bvp = True

    @property
    def n_unknowns(self) -> int:
        return 2 * self.nx * self.ny

    def ghost_coef(self, h):
        z = (1.0 + 0.5j * self.k * h) / (1.0 - 0.5j * self.k * h)
        return z.real, z.imag

    def G(self, x):
        ny, nx = self.ny, self.nx
        n = nx * ny
        A = x[:n].reshape(ny, nx)
        B = x[n:].reshape(ny, nx)
        hx, hy = 1.0 / nx, 1.0 / ny
        cxr, cxi = self.ghost_coef(hx)
        cyr, cyi = self.ghost_coef(hy)

        def lap(P, Q, sgn):
            # P is the plane itself, Q the other plane. The ghost beyond each
            # wall is c E_wall: Re = cr a - ci b, Im = cr b + ci a, i.e.
            # cr * P_wall + sgn * ci * Q_wall with sgn = -1 for Re, +1 for Im.
            west = np.concatenate([(cxr * P[:, :1] + sgn * cxi * Q[:, :1]), P[:, :-1]], axis=1)
            east = np.concatenate([P[:, 1:], (cxr * P[:, -1:] + sgn * cxi * Q[:, -1:])], axis=1)
            south = np.concatenate([(cyr * P[:1, :] + sgn * cyi * Q[:1, :]), P[:-1, :]], axis=0)
            north = np.concatenate([P[1:, :], (cyr * P[-1:, :] + sgn * cyi * Q[-1:, :])], axis=0)
            return (east - 2.0 * P + west) / (hx * hx) + (north - 2.0 * P + south) / (hy * hy)

        eps = self.eps_r.reshape(ny, nx) if self.eps_r is not None else np.ones((ny, nx))
        src = self.f if self.f is not None else np.zeros(2 * n)
        coef = self.k * self.k * (eps + self.chi3 * (A * A + B * B))
        Gr = lap(A, B, -1.0) + coef * A - src[:n].reshape(ny, nx)
        Gi = lap(B, A, +1.0) + coef * B - src[n:].reshape(ny, nx)
        return np.concatenate([Gr.reshape(-1), Gi.reshape(-1)])

    def cslp_diag(self, x, damping: float = 0.5):
        """Diagonal complex-shifted-Laplacian preconditioner at the field x (App. A, Preconditioning).

        Per cell, the diagonal of the operator lap + k^2 eps with the local permittivity
        eps(E) = eps_r + chi3 |E|^2 damped by the factor (1 - damping i):
          M = -(2/hx^2 + 2/hy^2) + k^2 eps(E) (1 - damping i)   (complex, one per cell).
        The absorbing walls are not part of it (the paper's form). Returns M (complex, nx*ny).
        """
        n = self.nx * self.ny
        A, B = x[:n], x[n:]
        eps = self.eps_r if self.eps_r is not None else np.ones(n)
        hx, hy = 1.0 / self.nx, 1.0 / self.ny
        eps_e = eps + self.chi3 * (A * A + B * B)
        return -(2.0 / (hx * hx) + 2.0 / (hy * hy)) + self.k * self.k * eps_e * (1.0 - damping * 1j)


@dataclass
class MaxwellVecTE2D(_ThetaProblem):
    """The paper's vector TE Maxwell problem in a Kerr medium (App. A, Time-Harmonic Maxwell's Equations).

    curl curl E - w^2 eps(E) E = i w J, E = (Ex, Ey), mu0 = eps0 = 1,
    eps(E) = (1 - 0.05 i)(1 + chi |E|), |E| = sqrt(|Ex|^2 + |Ey|^2), on the
    unit square with perfectly conducting walls, as the real map on the
    planes [Re Ex, Im Ex, Re Ey, Im Ey]:
      F = curl curl E - w^2 eps(E) E - i w J.
    Nodes x_i = i h, h = 1/(n - 1), the walls being nodes. Second-order
    central differences of (curl curl E)_x = d2 Ey/dxdy - d2 Ex/dy2 and
    (curl curl E)_y = d2 Ex/dxdy - d2 Ey/dx2 (the mixed derivative on the four
    corner neighbours). On the walls the tangential component's row is
    F = E_t (PEC); the normal component keeps its equation with neighbours
    beyond the wall taken by reflection: a tangential component odd, a normal
    component even across the wall (the image of a perfect conductor).
    |E| enters through a branch on its squared value: 0 where the field
    vanishes, so the derivative there is taken as 0.
    """

    nx: int = 32
    ny: int = 32
    omega: float = 5.0
    chi: float = 0.05
    J: np.ndarray | None = None      # [Re Jx, Im Jx, Re Jy, Im Jy] planes, or None (no source)
    bvp: bool = True
    theta: float = 0.0

    @property
    def n_unknowns(self) -> int:
        return 4 * self.nx * self.ny

    @property
    def spacing(self):
        return 1.0 / (self.nx - 1), 1.0 / (self.ny - 1)

    @staticmethod
    def _pad(u, sx, sy):
        """u (ny, nx) extended by one node per side by reflection about the wall nodes:
        factor sx across the x walls (left, right) and sy across the y walls."""
        p = np.zeros((u.shape[0] + 2, u.shape[1] + 2), dtype=u.dtype)
        p[1:-1, 1:-1] = u
        p[1:-1, 0] = sx * u[:, 1]
        p[1:-1, -1] = sx * u[:, -2]
        p[0, :] = sy * p[2, :]
        p[-1, :] = sy * p[-3, :]
        return p

    def curl_curl(self, ex, ey):
        """(curl curl E)_x, (curl curl E)_y of one real or imaginary part, on all nodes."""
        hx, hy = self.spacing
        px = self._pad(ex, 1.0, -1.0)   # Ex: normal to the x walls (even), tangential to the y walls (odd)
        py = self._pad(ey, -1.0, 1.0)   # Ey: tangential to the x walls (odd), normal to the y walls (even)
        dyy_ex = (px[2:, 1:-1] - 2.0 * ex + px[:-2, 1:-1]) / (hy * hy)
        dxx_ey = (py[1:-1, 2:] - 2.0 * ey + py[1:-1, :-2]) / (hx * hx)
        dxy_ey = (py[2:, 2:] - py[:-2, 2:] - py[2:, :-2] + py[:-2, :-2]) / (4.0 * hx * hy)
        dxy_ex = (px[2:, 2:] - px[:-2, 2:] - px[2:, :-2] + px[:-2, :-2]) / (4.0 * hx * hy)
        return dxy_ey - dyy_ex, dxy_ex - dxx_ey

    def _planes(self, x):
        n = self.nx * self.ny
        return [x[k * n:(k + 1) * n].reshape(self.ny, self.nx) for k in range(4)]

    def G(self, x):
        a, b, c, d = self._planes(x)
        cxa, cya = self.curl_curl(a, c)          # real parts
        cxb, cyb = self.curl_curl(b, d)          # imaginary parts
        s2 = a * a + b * b + c * c + d * d
        m = np.where(s2.real > 0.0, np.sqrt(np.where(s2.real > 0.0, s2, 1.0)), 0.0)
        e = 1.0 + self.chi * m
        w2 = self.omega * self.omega
        J = np.zeros(4 * self.nx * self.ny) if self.J is None else self.J
        ja, jb, jc, jd = self._planes(J)
        # - i w J: real part + w Im J, imaginary part - w Re J
        F = [cxa - w2 * e * (a + 0.05 * b) + self.omega * jb,
             cxb - w2 * e * (b - 0.05 * a) - self.omega * ja,
             cya - w2 * e * (c + 0.05 * d) + self.omega * jd,
             cyb - w2 * e * (d - 0.05 * c) - self.omega * jc]
        # PEC: the tangential component's rows are E_t on the walls
        for k, comp in ((0, a), (1, b)):        # Ex is tangential to the y walls (bottom, top)
            F[k] = F[k].copy()
            F[k][0, :] = comp[0, :]
            F[k][-1, :] = comp[-1, :]
        for k, comp in ((2, c), (3, d)):        # Ey is tangential to the x walls (left, right)
            F[k] = F[k].copy()
            F[k][:, 0] = comp[:, 0]
            F[k][:, -1] = comp[:, -1]
        return np.concatenate([f.reshape(-1) for f in F])

    def cslp_diag(self, x, damping: float = 0.5):
        """Block-diagonal complex-shifted-Laplacian preconditioner (App. A, Preconditioning):
        per node M_xx = 2/hy^2 - w^2 eps_p, M_yy = 2/hx^2 - w^2 eps_p with eps_p = eps(E)(1 - damping i);
        1 on the PEC rows (their Jacobian rows are the identity). Returns [M_xx, M_yy] (complex, 2 n)."""
        a, b, c, d = self._planes(x)
        hx, hy = self.spacing
        s2 = a * a + b * b + c * c + d * d
        m = np.where(s2 > 0.0, np.sqrt(np.where(s2 > 0.0, s2, 1.0)), 0.0)
        epsp = (1.0 - 0.05j) * (1.0 + self.chi * m) * (1.0 - damping * 1j)
        w2 = self.omega * self.omega
        mxx = (2.0 / (hy * hy) - w2 * epsp).astype(complex)
        myy = (2.0 / (hx * hx) - w2 * epsp).astype(complex)
        mxx[0, :] = 1.0
        mxx[-1, :] = 1.0
        myy[:, 0] = 1.0
        myy[:, -1] = 1.0
        return np.concatenate([mxx.reshape(-1), myy.reshape(-1)])

    def apply_diag(self, c, v):
        """The planes [a, b, c, d] of v with (a + ib) times c[:n] and (c + id) times c[n:], node by node."""
        n = self.nx * self.ny
        zx = c[:n] * (v[:n] + 1j * v[n:2 * n])
        zy = c[n:] * (v[2 * n:3 * n] + 1j * v[3 * n:])
        return np.concatenate([zx.real, zx.imag, zy.real, zy.imag])

    def born(self):
        """The chi = 0 problem (the Born start of App. A: the field linearised at E = 0)."""
        import copy as _copy
        q = _copy.copy(self)
        q.chi = 0.0
        return q


def apply_cell_complex(c, v):
    """(Re, Im) planes of v multiplied cell by cell by the complex array c."""
    n = c.size
    z = c * (v[:n] + 1j * v[n:])
    return np.concatenate([z.real, z.imag])


def make(pde: str, **kw):
    """Construct a problem by name: burgers1d, burgers2d, allen_cahn, su_olson, maxwell."""
    return {"burgers1d": Burgers1D, "burgers2d": Burgers2D, "allen_cahn": AllenCahn2D,
            "su_olson": SuOlson2D, "maxwell": MaxwellTE2D, "maxwell_vec": MaxwellVecTE2D}[pde](**kw)
