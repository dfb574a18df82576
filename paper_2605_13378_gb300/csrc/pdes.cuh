// pdes.cuh -- per-cell discrete residuals of the four benchmark PDEs.
//
// Each PDE is a struct with a static `cell` function that, given a loader
// (flat index -> value) and a cell (i, j), returns for every field f the
// "mass" term M_f(x) and the spatial operator G_f(x) at that cell. The value
// type V is a plain float/double (residual, FD quotient) or a Dual (AD JVP):
// the same source computes F(x) and, on dual numbers, J(x) v (Eq. 9).
// Branches test primal values only, so AD differentiates the branch taken.
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
  double thdt;            // theta * dt (1 for the boundary-value problem, unused)
  double c_old;           // (1 - theta) * dt
  double invhx, invhy, invhx2, invhy2;
  double p0, p1, p2, p3;  // PDE parameters (see jfnk_pde)
  int flag;               // Su-Olson: flux limiter on
  int bvp;
  // Su-Olson Marshak wall: q = mq_a - mq_b * E_0
  double mq_a, mq_b;
  // Maxwell first-order absorbing wall: E_ghost = (cr + i ci) E_wall
  double cxr, cxi, cyr, cyi;
  const double* eps64; const float* eps32;   // eps_r plane or null (= 1)
  const double* src64; const float* src32;   // source planes (Re, Im) or null
};

template <class T> __device__ __forceinline__ const T* eps_of(const ProbDev& P);
template <> __device__ __forceinline__ const double* eps_of<double>(const ProbDev& P) { return P.eps64; }
template <> __device__ __forceinline__ const float* eps_of<float>(const ProbDev& P) { return P.eps32; }
template <class T> __device__ __forceinline__ const T* src_of(const ProbDev& P);
template <> __device__ __forceinline__ const double* src_of<double>(const ProbDev& P) { return P.src64; }
template <> __device__ __forceinline__ const float* src_of<float>(const ProbDev& P) { return P.src32; }

// ---------------------------------------------------------------------------
// 1D viscous Burgers, periodic, cells x_i = i/N. Conservative upwind flux
// Phi_{i+1/2} = u_i^2/2 if u_i + u_{i+1} >= 0 else u_{i+1}^2/2 (the Roe flux),
// central second difference for viscosity:
//   G_i = -(Phi_{i+1/2} - Phi_{i-1/2}) / h + nu (u_{i+1} - 2u_i + u_{i-1}) / h^2
// ---------------------------------------------------------------------------
struct Burgers1D {
  static constexpr int NF = 1;
  template <class T, class V, class L>
  __device__ __forceinline__ static void cell(const ProbDev& P, const L& ld, int i, int /*j*/, V* M, V* G) {
    const int n = P.nx;
    const int im = (i == 0) ? n - 1 : i - 1;
    const int ip = (i == n - 1) ? 0 : i + 1;
    V u = ld(i), um = ld(im), up = ld(ip);
    const T half = T(0.5);
    V phip = (primal(u) + primal(up) >= T(0)) ? half * u * u : half * up * up;
    V phim = (primal(um) + primal(u) >= T(0)) ? half * um * um : half * u * u;
    const T invh = T(P.invhx), invh2 = T(P.invhx2), nu = T(P.p0);
    M[0] = u;
    G[0] = (phim - phip) * invh + nu * ((up - T(2) * u + um) * invh2);
  }
};

// ---------------------------------------------------------------------------
// Allen-Cahn u_t = D lap u + c u - u^3 (c = 1; c = 0 is the paper's
// reaction-diffusion sink), periodic unit square, 5-point Laplacian.
// ---------------------------------------------------------------------------
struct AllenCahn2D {
  static constexpr int NF = 1;
  template <class T, class V, class L>
  __device__ __forceinline__ static void cell(const ProbDev& P, const L& ld, int i, int j, V* M, V* G) {
    const int nx = P.nx, ny = P.ny;
    const int ie = (i == nx - 1) ? 0 : i + 1, iw = (i == 0) ? nx - 1 : i - 1;
    const int jn = (j == ny - 1) ? 0 : j + 1, js = (j == 0) ? ny - 1 : j - 1;
    const long long r = (long long)j * nx;
    V u = ld(r + i);
    V ue = ld(r + ie), uw = ld(r + iw);
    V un = ld((long long)jn * nx + i), us = ld((long long)js * nx + i);
    V lap = (ue - T(2) * u + uw) * T(P.invhx2) + (un - T(2) * u + us) * T(P.invhy2);
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
// ---------------------------------------------------------------------------
struct SuOlson2D {
  static constexpr int NF = 2;
  template <class T, class V>
  __device__ __forceinline__ static V face_flux(const ProbDev& P, V gn, V gt, V Ebar) {
    const T three_sigma = T(3) * T(P.p0);
    if (!P.flag) return gn * (T(1) / three_sigma);
    const T rho = T(P.p3);
    V R = dsqrt((gn * gn + gt * gt) / (Ebar * Ebar) + rho * rho);
    return gn / (three_sigma + R);
  }
  template <class T, class V, class L>
  __device__ __forceinline__ static void cell(const ProbDev& P, const L& ld, int i, int j, V* M, V* G) {
    const int nx = P.nx, ny = P.ny;
    const int ic0 = i > 0 ? i - 1 : 0, ic2 = i < nx - 1 ? i + 1 : nx - 1;
    const int jc0 = j > 0 ? j - 1 : 0, jc2 = j < ny - 1 ? j + 1 : ny - 1;
    const long long r0 = (long long)jc0 * nx, r1 = (long long)j * nx, r2 = (long long)jc2 * nx;
    // E(a, b): column ic_a, row jc_b
    V E00 = ld(r0 + ic0), E10 = ld(r0 + i), E20 = ld(r0 + ic2);
    V E01 = ld(r1 + ic0), E11 = ld(r1 + i), E21 = ld(r1 + ic2);
    V E02 = ld(r2 + ic0), E12 = ld(r2 + i), E22 = ld(r2 + ic2);
    V Tc = ld(P.ncell + r1 + i);
    const T ihx = T(P.invhx), ihy = T(P.invhy), q = T(0.25), half = T(0.5);
    V fe, fw, fn, fs;
    if (i < nx - 1) {
      fe = face_flux<T>(P, (E21 - E11) * ihx, ((E12 + E22) - (E10 + E20)) * (q * ihy), half * (E11 + E21));
    } else {
      fe = V(T(0));
    }
    if (i > 0) {
      fw = face_flux<T>(P, (E11 - E01) * ihx, ((E02 + E12) - (E00 + E10)) * (q * ihy), half * (E01 + E11));
    } else {
      fw = E11 * T(P.mq_b) - T(P.mq_a);   // D dE/dx at the wall = -q
    }
    if (j < ny - 1) {
      fn = face_flux<T>(P, (E12 - E11) * ihy, ((E21 + E22) - (E01 + E02)) * (q * ihx), half * (E11 + E12));
    } else {
      fn = V(T(0));
    }
    if (j > 0) {
      fs = face_flux<T>(P, (E11 - E10) * ihy, ((E20 + E21) - (E00 + E01)) * (q * ihx), half * (E10 + E11));
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
  static constexpr int NF = 2;
  template <class T, class V, class L>
  __device__ __forceinline__ static void cell(const ProbDev& P, const L& ld, int i, int j, V* M, V* G) {
    const int nx = P.nx, ny = P.ny;
    const long long n = P.ncell, c = (long long)j * nx + i;
    V A = ld(c), B = ld(n + c);
    const T cxr = T(P.cxr), cxi = T(P.cxi), cyr = T(P.cyr), cyi = T(P.cyi);
    V gxA = cxr * A - cxi * B, gxB = cxr * B + cxi * A;   // ghost beyond an x wall
    V gyA = cyr * A - cyi * B, gyB = cyr * B + cyi * A;   // ghost beyond a y wall
    V Aw, Bw, Ae, Be, As, Bs, An, Bn;
    if (i > 0) { Aw = ld(c - 1); Bw = ld(n + c - 1); } else { Aw = gxA; Bw = gxB; }
    if (i < nx - 1) { Ae = ld(c + 1); Be = ld(n + c + 1); } else { Ae = gxA; Be = gxB; }
    if (j > 0) { As = ld(c - nx); Bs = ld(n + c - nx); } else { As = gyA; Bs = gyB; }
    if (j < ny - 1) { An = ld(c + nx); Bn = ld(n + c + nx); } else { An = gyA; Bn = gyB; }
    const T ihx2 = T(P.invhx2), ihy2 = T(P.invhy2);
    V LA = (Ae - T(2) * A + Aw) * ihx2 + (An - T(2) * A + As) * ihy2;
    V LB = (Be - T(2) * B + Bw) * ihx2 + (Bn - T(2) * B + Bs) * ihy2;
    const T* epsp = eps_of<T>(P);
    const T* srcp = src_of<T>(P);
    const T eps = epsp ? __ldg(epsp + c) : T(1);
    const T fr = srcp ? __ldg(srcp + c) : T(0);
    const T fi = srcp ? __ldg(srcp + n + c) : T(0);
    const T k2 = T(P.p0) * T(P.p0), chi = T(P.p1);
    V coef = k2 * (eps + chi * (A * A + B * B));
    M[0] = A;
    M[1] = B;
    G[0] = LA + coef * A - fr;
    G[1] = LB + coef * B - fi;
  }
};

}  // namespace jfnk
