// pdes.cuh -- per-cell discrete residuals of the benchmark PDEs.
//
// Each PDE is a struct with a static `cell` function that, given the values
// of the 3 x 3 neighbourhood of cell (i, j) for every field, returns per
// field the "mass" term M_f(x) and the spatial operator G_f(x) at that cell.
// Values outside the grid are supplied by the PDE's boundary policy (periodic
// wrap or clamp to the wall cell); walls with other conditions (the Marshak
// and zero-flux faces of the radiation problem, the absorbing ghosts of the
// Maxwell problem) are handled inside `cell` from (i, j). The value type V is
// a plain float/double (residual, FD quotient) or a Dual (AD JVP): the same
// source computes F(x) and, on dual numbers, J(x) v (Eq. 9). Branches test
// primal values only, so AD differentiates the branch taken.
//
// The theta-method residual of an implicit step (Eq. 2) is assembled by the
// caller as F = M - theta dt G - b; the Maxwell problem is a boundary-value
// problem, F = G.
#pragma once

#include "common.cuh"

namespace jfnk {

// Problem description as the kernels see it. Derived constants are computed
// once on the host in double precision.
struct ProbDev {
  int pde, nx, ny, nf;
  long long ncell;        // nx * ny
  double thdt;            // theta * dt (unused by the boundary-value problem)
  double c_old;           // (1 - theta) * dt
  double dt;              // time step installed by set_dt
  double theta;           // theta of the time scheme (0 for the boundary-value problem)
  double cfl;             // Courant number of an adaptive step (0: fixed dt)
  double hx, hy;          // grid spacing
  double invhx, invhy, invhx2, invhy2;
  double p0, p1, p2, p3;  // PDE parameters (see jfnk_pde)
  int flag;               // Su-Olson: flux limiter on
  int bvp;
  // Su-Olson Marshak wall: inward flux q = mq_a - mq_b * E_0
  double mq_a, mq_b;
  // Maxwell first-order absorbing wall: E_ghost = (cr + i ci) E_wall
  double cxr, cxi, cyr, cyi;
  const double* eps64; const float* eps32;   // eps_r plane or null (= 1)
  const double* src64; const float* src32;   // source planes (Re, Im) or null
};

// Install the time step dt of an implicit step (theta method).
inline void set_dt(ProbDev* P, double dt) {
  if (P->bvp) return;
  P->dt = dt;
  P->thdt = P->theta * dt;
  P->c_old = (1.0 - P->theta) * dt;
}

// CFL rule of the 2D Burgers problem from umax = max|u|, vmax = max|v| (App. A,
// Burgers' Equation): C min(hx / umax, hy / vmax, 1 / (2 nu (1/hx^2 + 1/hy^2))),
// a term with a zero denominator left out (none left: +Inf); NaN when a
// maximum is not finite.
__host__ __device__ inline double cfl_rule(double umax, double vmax, double hx, double hy, double nu, double C) {
  if (!(umax <= 1.7976931348623157e308) || !(vmax <= 1.7976931348623157e308)) return 0.0 / 0.0;
  double dt = 1.0 / 0.0;
  if (nu > 0.0) dt = 1.0 / (2.0 * nu * (1.0 / (hx * hx) + 1.0 / (hy * hy)));
  if (umax > 0.0) dt = fmin(dt, hx / umax);
  if (vmax > 0.0) dt = fmin(dt, hy / vmax);
  return C * dt;
}

template <class T> __device__ __forceinline__ const T* eps_of(const ProbDev& P);
template <> __device__ __forceinline__ const double* eps_of<double>(const ProbDev& P) { return P.eps64; }
template <> __device__ __forceinline__ const float* eps_of<float>(const ProbDev& P) { return P.eps32; }
template <class T> __device__ __forceinline__ const T* src_of(const ProbDev& P);
template <> __device__ __forceinline__ const double* src_of<double>(const ProbDev& P) { return P.src64; }
template <> __device__ __forceinline__ const float* src_of<float>(const ProbDev& P) { return P.src32; }

enum BoundaryPolicy { BP_WRAP = 0, BP_CLAMP = 1 };

// Neighbourhood of one cell: centre, the four face neighbours and the four
// corner neighbours (corners only for PDEs with DIAG) of each field.
template <class V, int NF>
struct Nb {
  V c[NF], e[NF], w[NF], n[NF], s[NF];
  V ne[NF], nw[NF], se[NF], sw[NF];
};

// Per-cell coefficients read from problem arrays (Maxwell: eps_r, source;
// the vector form's current: fr + i fi = J_x, gr + i gi = J_y).
template <class T>
struct CellAux {
  T eps, fr, fi, gr, gi;
};

// sqrt of a sum of squares with the derivative taken as 0 where the sum is 0
// (|E| at a node where the field vanishes: the residual's branch there)
template <class T> __device__ __forceinline__ Dual<T> sqrt0(Dual<T> s) {
  return primal(s) > T(0) ? dsqrt(s) : Dual<T>(T(0), T(0));
}
__device__ __forceinline__ double sqrt0(double s) { return s > 0.0 ? sqrt(s) : 0.0; }
__device__ __forceinline__ float sqrt0(float s) { return s > 0.0f ? sqrtf(s) : 0.0f; }

// ---------------------------------------------------------------------------
// 1D viscous Burgers, periodic, cells x_i = i/N. Conservative upwind flux
// Phi_{i+1/2} = u_i^2/2 if u_i + u_{i+1} >= 0 else u_{i+1}^2/2 (the Roe flux),
// central second difference for viscosity:
//   G_i = -(Phi_{i+1/2} - Phi_{i-1/2}) / h + nu (u_{i+1} - 2u_i + u_{i-1}) / h^2
// ---------------------------------------------------------------------------
struct Burgers1D {
  static constexpr bool PRECOND = false;
  static constexpr int NSRC = 0;
  static constexpr int NF = 1;
  static constexpr bool DIAG = false;
  static constexpr int POLICY = BP_WRAP;
  static constexpr bool AUX = false;
  template <class T, class V>
  __device__ __forceinline__ static void cell(const ProbDev& P, int, int, const Nb<V, 1>& q, const CellAux<T>&,
                                              V* M, V* G) {
    const V u = q.c[0], um = q.w[0], up = q.e[0];
    const T half = T(0.5);
    V phip = (primal(u) + primal(up) >= T(0)) ? half * u * u : half * up * up;
    V phim = (primal(um) + primal(u) >= T(0)) ? half * um * um : half * u * u;
    M[0] = u;
    G[0] = (phim - phip) * T(P.invhx) + T(P.p0) * ((up - T(2) * u + um) * T(P.invhx2));
  }
};

// ---------------------------------------------------------------------------
// 2D viscous Burgers U_t + (U . grad) U = nu lap U, U = (u, v), periodic
// square of side L on nodes x_i = i hx, y_j = j hy (App. A, Burgers'
// Equation). Second-order central differences for the advection and the
// 5-point Laplacian for the diffusion, per field w in {u, v}:
//   G_w = nu lap w - (u (w_e - w_w) / 2hx + v (w_n - w_s) / 2hy)
// invhx, invhy are 1/hx, 1/hy of the square (not of the unit square).
// ---------------------------------------------------------------------------
struct Burgers2D {
  static constexpr bool PRECOND = false;
  static constexpr int NSRC = 0;
  static constexpr int NF = 2;
  static constexpr bool DIAG = false;
  static constexpr int POLICY = BP_WRAP;
  static constexpr bool AUX = false;
  template <class T, class V>
  __device__ __forceinline__ static void cell(const ProbDev& P, int, int, const Nb<V, 2>& q, const CellAux<T>&,
                                              V* M, V* G) {
    const V u = q.c[0], v = q.c[1];
    const T hix = T(0.5) * T(P.invhx), hiy = T(0.5) * T(P.invhy);
    const T ihx2 = T(P.invhx2), ihy2 = T(P.invhy2), nu = T(P.p0);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const V w = q.c[f];
      V lap = (q.e[f] - T(2) * w + q.w[f]) * ihx2 + (q.n[f] - T(2) * w + q.s[f]) * ihy2;
      V adv = u * ((q.e[f] - q.w[f]) * hix) + v * ((q.n[f] - q.s[f]) * hiy);
      M[f] = w;
      G[f] = nu * lap - adv;
    }
  }
};

// ---------------------------------------------------------------------------
// Allen-Cahn u_t = D lap u + c u - u^3 (c = 1; c = 0 is the paper's
// reaction-diffusion sink), 5-point Laplacian: periodic unit square, or
// (P.flag) homogeneous Dirichlet walls, the unknowns being the interior
// nodes, so that a neighbour beyond a wall is 0.
// ---------------------------------------------------------------------------
struct AllenCahn2D {
  static constexpr bool PRECOND = false;
  static constexpr int NSRC = 0;
  static constexpr int NF = 1;
  static constexpr bool DIAG = false;
  static constexpr int POLICY = BP_WRAP;
  static constexpr bool AUX = false;
  template <class T, class V>
  __device__ __forceinline__ static void cell(const ProbDev& P, int i, int j, const Nb<V, 1>& q,
                                              const CellAux<T>&, V* M, V* G) {
    const V u = q.c[0];
    V e = q.e[0], w = q.w[0], n = q.n[0], s = q.s[0];
    if (P.flag) {
      if (i == 0) w = V(T(0));
      if (i == P.nx - 1) e = V(T(0));
      if (j == 0) s = V(T(0));
      if (j == P.ny - 1) n = V(T(0));
    }
    V lap = (e - T(2) * u + w) * T(P.invhx2) + (n - T(2) * u + s) * T(P.invhy2);
    M[0] = u;
    G[0] = T(P.p0) * lap + T(P.p1) * u - u * u * u;
  }
};

// ---------------------------------------------------------------------------
// Two-field radiation diffusion (E, T) with a flux limiter and a Marshak wall.
//   G_E = div(D(E) grad E) - sigma (E - a T^4),  M_E = E
//   G_T = sigma (E - a T^4),                      M_T = a T^4
// Face coefficient D_f = 1 / (3 sigma + R_f), R_f = sqrt(|g|^2 / Ebar^2 + rho^2),
// g = (normal difference, tangential difference averaged over the four cells
// touching the face, mirror values beyond a wall), Ebar the mean of the two
// cells; limiter off: D = 1/(3 sigma). Left wall: inward Marshak flux
// q = 2 D_b (4 F_inc - E_0)/(h + 4 D_b) = mq_a - mq_b E_0; other walls: no flux.
// The clamp policy supplies the mirror values.
// ---------------------------------------------------------------------------
struct SuOlson2D {
  static constexpr bool PRECOND = false;
  static constexpr int NSRC = 0;
  static constexpr int NF = 2;
  static constexpr bool DIAG = true;
  static constexpr int POLICY = BP_CLAMP;
  static constexpr bool AUX = false;
  template <class T, class V>
  __device__ __forceinline__ static V face_flux(const ProbDev& P, V gn, V gt, V Ebar) {
    const T three_sigma = T(3) * T(P.p0);
    if (!P.flag) return gn * (T(1) / three_sigma);
    const T rho = T(P.p3);
    V R = dsqrt((gn * gn + gt * gt) / (Ebar * Ebar) + rho * rho);
    return gn / (three_sigma + R);
  }
  template <class T, class V>
  __device__ __forceinline__ static void cell(const ProbDev& P, int i, int j, const Nb<V, 2>& q, const CellAux<T>&,
                                              V* M, V* G) {
    const int nx = P.nx, ny = P.ny;
    const V E00 = q.sw[0], E10 = q.s[0], E20 = q.se[0];
    const V E01 = q.w[0], E11 = q.c[0], E21 = q.e[0];
    const V E02 = q.nw[0], E12 = q.n[0], E22 = q.ne[0];
    const V Tc = q.c[1];
    const T ihx = T(P.invhx), ihy = T(P.invhy), qq = T(0.25), half = T(0.5);
    V fe, fw, fn, fs;
    if (i < nx - 1) {
      fe = face_flux<T>(P, (E21 - E11) * ihx, ((E12 + E22) - (E10 + E20)) * (qq * ihy), half * (E11 + E21));
    } else {
      fe = V(T(0));
    }
    if (i > 0) {
      fw = face_flux<T>(P, (E11 - E01) * ihx, ((E02 + E12) - (E00 + E10)) * (qq * ihy), half * (E01 + E11));
    } else {
      fw = E11 * T(P.mq_b) - T(P.mq_a);   // D dE/dx at the wall = -q
    }
    if (j < ny - 1) {
      fn = face_flux<T>(P, (E12 - E11) * ihy, ((E21 + E22) - (E01 + E02)) * (qq * ihx), half * (E11 + E12));
    } else {
      fn = V(T(0));
    }
    if (j > 0) {
      fs = face_flux<T>(P, (E11 - E10) * ihy, ((E20 + E21) - (E00 + E01)) * (qq * ihx), half * (E10 + E11));
    } else {
      fs = V(T(0));
    }
    V div = (fe - fw) * ihx + (fn - fs) * ihy;
    const T a = T(P.p1), sigma = T(P.p0);
    V T2 = Tc * Tc;
    V aT4 = a * (T2 * T2);
    V exch = sigma * (E11 - aT4);
    M[0] = E11;
    G[0] = div - exch;
    M[1] = aT4;
    G[1] = exch;
  }
};

// ---------------------------------------------------------------------------
// Scalar TE (E_z) Helmholtz with a Kerr term, as a real map on (Re, Im):
//   G = lap E + k^2 (eps_r + chi3 |E|^2) E - f
// 5-point Laplacian; beyond each wall a ghost E_g = (cr + i ci) E_wall, the
// first-order absorbing condition dE/dn = i k E discretised at the wall.
// ---------------------------------------------------------------------------
struct MaxwellTE2D {
  static constexpr bool PRECOND = false;
  static constexpr int NSRC = 2;
  static constexpr int NF = 2;
  static constexpr bool DIAG = false;
  static constexpr int POLICY = BP_CLAMP;
  static constexpr bool AUX = true;
  template <class T, class V>
  __device__ __forceinline__ static void cell(const ProbDev& P, int i, int j, const Nb<V, 2>& q,
                                              const CellAux<T>& aux, V* M, V* G) {
    const int nx = P.nx, ny = P.ny;
    const V A = q.c[0], B = q.c[1];
    const T cxr = T(P.cxr), cxi = T(P.cxi), cyr = T(P.cyr), cyi = T(P.cyi);
    const V gxA = cxr * A - cxi * B, gxB = cxr * B + cxi * A;   // ghost beyond an x wall
    const V gyA = cyr * A - cyi * B, gyB = cyr * B + cyi * A;   // ghost beyond a y wall
    const V Aw = i > 0 ? q.w[0] : gxA, Bw = i > 0 ? q.w[1] : gxB;
    const V Ae = i < nx - 1 ? q.e[0] : gxA, Be = i < nx - 1 ? q.e[1] : gxB;
    const V As = j > 0 ? q.s[0] : gyA, Bs = j > 0 ? q.s[1] : gyB;
    const V An = j < ny - 1 ? q.n[0] : gyA, Bn = j < ny - 1 ? q.n[1] : gyB;
    const T ihx2 = T(P.invhx2), ihy2 = T(P.invhy2);
    V LA = (Ae - T(2) * A + Aw) * ihx2 + (An - T(2) * A + As) * ihy2;
    V LB = (Be - T(2) * B + Bw) * ihx2 + (Bn - T(2) * B + Bs) * ihy2;
    const T k2 = T(P.p0) * T(P.p0), chi = T(P.p1);
    V coef = k2 * (aux.eps + chi * (A * A + B * B));
    M[0] = A;
    M[1] = B;
    G[0] = LA + coef * A - aux.fr;
    G[1] = LB + coef * B - aux.fi;
  }
};

// ---------------------------------------------------------------------------
// The paper's vector TE Maxwell problem in a Kerr medium (App. A, Time-
// Harmonic Maxwell's Equations in Kerr Media), as a real map on the planes
// [Re E_x, Im E_x, Re E_y, Im E_y] = [a, b, c, d]:
//   F = curl curl E - w^2 eps(E) E - i w J,
//   eps(E) = (1 - L i)(1 + chi |E|),  |E| = sqrt(a^2 + b^2 + c^2 + d^2),
// with L = p[2] (the paper's 0.05), w = p[0], chi = p[1], on nodes
// x_i = i hx, hx = 1/(nx - 1) of the unit square whose walls are nodes.
// Central differences: (curl curl E)_x = d2E_y/dxdy - d2E_x/dy2,
// (curl curl E)_y = d2E_x/dxdy - d2E_y/dx2, the mixed derivative on the four
// corner neighbours. Perfect electric conductor walls: the tangential
// component's rows are F = E_t (E_x on the bottom and top walls, E_y on the
// left and right ones); a neighbour beyond a wall is the image across it,
// the tangential component odd and the normal one even (the corner beyond
// two walls takes both signs). |E| = 0 takes a zero derivative.
// ---------------------------------------------------------------------------
struct MaxwellVec2D {
  static constexpr bool PRECOND = true;
  static constexpr int NSRC = 4;
  static constexpr int NF = 4;
  static constexpr bool DIAG = true;
  static constexpr int POLICY = BP_CLAMP;
  static constexpr bool AUX = true;
  template <class T, class V>
  __device__ __forceinline__ static void cell(const ProbDev& P, int i, int j, const Nb<V, 4>& q,
                                              const CellAux<T>& aux, V* M, V* G) {
    const int nx = P.nx, ny = P.ny;
    const bool wx0 = i == 0, wx1 = i == nx - 1, wy0 = j == 0, wy1 = j == ny - 1;
    V W[4], E[4], S[4], N[4], NE[4], NW[4], SE[4], SW[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const T sx = f < 2 ? T(1) : T(-1);   // image across an x wall: E_x even, E_y odd
      const T sy = f < 2 ? T(-1) : T(1);   // across a y wall: E_x odd, E_y even
      W[f] = wx0 ? sx * q.e[f] : q.w[f];
      E[f] = wx1 ? sx * q.w[f] : q.e[f];
      S[f] = wy0 ? sy * q.n[f] : q.s[f];
      N[f] = wy1 ? sy * q.s[f] : q.n[f];
      // a corner beyond a wall is the image of the corner on the other side of that wall
      const V ne = wx1 ? (wy1 ? q.sw[f] : q.nw[f]) : (wy1 ? q.se[f] : q.ne[f]);
      const V nw = wx0 ? (wy1 ? q.se[f] : q.ne[f]) : (wy1 ? q.sw[f] : q.nw[f]);
      const V se = wx1 ? (wy0 ? q.nw[f] : q.sw[f]) : (wy0 ? q.ne[f] : q.se[f]);
      const V sw = wx0 ? (wy0 ? q.ne[f] : q.se[f]) : (wy0 ? q.nw[f] : q.sw[f]);
      NE[f] = (wx1 ? sx : T(1)) * (wy1 ? sy : T(1)) * ne;
      NW[f] = (wx0 ? sx : T(1)) * (wy1 ? sy : T(1)) * nw;
      SE[f] = (wx1 ? sx : T(1)) * (wy0 ? sy : T(1)) * se;
      SW[f] = (wx0 ? sx : T(1)) * (wy0 ? sy : T(1)) * sw;
    }
    const T ihx2 = T(P.invhx2), ihy2 = T(P.invhy2), ixy = T(0.25) * T(P.invhx) * T(P.invhy);
    V cc[4], dyy[4], dxx[4], dxy[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      cc[f] = q.c[f];
      dyy[f] = (N[f] - T(2) * cc[f] + S[f]) * ihy2;
      dxx[f] = (E[f] - T(2) * cc[f] + W[f]) * ihx2;
      dxy[f] = (NE[f] - SE[f] - NW[f] + SW[f]) * ixy;
    }
    const V a = cc[0], b = cc[1], c = cc[2], d = cc[3];
    const V m = sqrt0(a * a + b * b + c * c + d * d);
    const V e = T(1) + T(P.p1) * m;
    const T w = T(P.p0), w2 = w * w, L = T(P.p2);
    V F0 = (dxy[2] - dyy[0]) - w2 * e * (a + L * b) + w * aux.fi;
    V F1 = (dxy[3] - dyy[1]) - w2 * e * (b - L * a) - w * aux.fr;
    V F2 = (dxy[0] - dxx[2]) - w2 * e * (c + L * d) + w * aux.gi;
    V F3 = (dxy[1] - dxx[3]) - w2 * e * (d - L * c) - w * aux.gr;
    if (wy0 || wy1) { F0 = a; F1 = b; }   // PEC: E_x tangential to the bottom and top walls
    if (wx0 || wx1) { F2 = c; F3 = d; }   // PEC: E_y tangential to the left and right walls
    M[0] = a; M[1] = b; M[2] = c; M[3] = d;
    G[0] = F0; G[1] = F1; G[2] = F2; G[3] = F3;
  }
  // The paper's block-diagonal complex-shifted-Laplacian preconditioner (App.
  // A, Preconditioning) at node (i, j) with the field x there: v is replaced
  // by M^-1 v, the x and y components divided by
  //   M_xx = 2/hy^2 - w^2 eps_p,  M_yy = 2/hx^2 - w^2 eps_p,
  //   eps_p = eps(E)(1 - beta i) = (1 - L i)(1 - beta i)(1 + chi |E|),
  // and left alone on the rows of tangential components on the walls (M = 1,
  // those Jacobian rows being the identity).
  template <class T>
  __device__ __forceinline__ static void precond(const ProbDev& P, T beta, int i, int j, const T* x, T* v) {
    const T m = sqrt0(x[0] * x[0] + x[1] * x[1] + x[2] * x[2] + x[3] * x[3]);
    const T e = T(1) + T(P.p1) * m, L = T(P.p2), w2 = T(P.p0) * T(P.p0);
    const T er = e * (T(1) - L * beta), ei = -e * (L + beta);   // eps_p = er + i ei
    const T mi = -w2 * ei;
    const bool pec_x = (j == 0 || j == P.ny - 1), pec_y = (i == 0 || i == P.nx - 1);
    if (!pec_x) {   // (v0 + i v1) / (mxr + i mi)
      const T mr = T(2) * T(P.invhy2) - w2 * er, den = mr * mr + mi * mi;
      const T a = v[0], b = v[1];
      v[0] = (a * mr + b * mi) / den;
      v[1] = (b * mr - a * mi) / den;
    }
    if (!pec_y) {
      const T mr = T(2) * T(P.invhx2) - w2 * er, den = mr * mr + mi * mi;
      const T a = v[2], b = v[3];
      v[2] = (a * mr + b * mi) / den;
      v[3] = (b * mr - a * mi) / den;
    }
  }
};

}  // namespace jfnk
