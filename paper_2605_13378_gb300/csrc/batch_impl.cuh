// batch_impl.cuh -- the batch kernel: every launch advances every unfinished
// solve of a (PDE, precision) group by one phase of Newton-GMRES.
//
// The algorithm per solve is the one of the single-solve driver: Newton on
// F(x) = 0 with a backtracking (Armijo) line search on ||F|| (Sec. 2), the
// Newton step from restarted GMRES(m) with CGS2 Arnoldi and Givens rotations
// (Sec. 3), each Krylov product a JVP by dual numbers (Eq. 9) or by the FD
// quotient (Eq. 7), time steps by the theta method, and for the Maxwell
// problem a Born start (the chi3 = 0 problem solved once first).
//
// Work: a (solve, tile) item list; CTAs take items from an atomic counter.
// A tile is tc consecutive cells (all fields). Per-unit partial sums
// (kBatUnit cells) are written by the tile; the tile that finishes last for
// its solve sums the units in a fixed order and runs the solve's scalar step
// (thread 0), which also chooses the solve's next phase. No CTA ever waits on
// another, so the kernel cannot hang whatever the residency.
#pragma once

#include <type_traits>

#include "batch.h"
#include "jfnk.h"

namespace jfnk {

template <class T> struct BatAcc { typedef float type; };
template <> struct BatAcc<double> { typedef double type; };

template <class T> __device__ __forceinline__ double bat_eps_mach();
template <> __device__ __forceinline__ double bat_eps_mach<double>() { return 2.220446049250313e-16; }
template <> __device__ __forceinline__ double bat_eps_mach<float>() { return 1.1920928955078125e-07; }

__device__ __forceinline__ int bat_nb(int i, int n, int policy) {
  if (i < 0) return policy == BP_WRAP ? i + n : 0;
  if (i >= n) return policy == BP_WRAP ? i - n : n - 1;
  return i;
}

// The residual terms (M, G) of each cell c in [c0, c1), one cell per thread
// per blockDim; ld(f, id) gives the value (plain or dual) of field f at
// cell id, out(c, M, G, centre values) consumes the result.
template <class PDE, class T, class V, class LD, class OUT>
__device__ __forceinline__ void bat_cells(const ProbDev& P, long long c0, long long c1, LD ld, OUT out) {
  constexpr int NF = PDE::NF;
  const int nx = P.nx, ny = P.ny;
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
    const int ie = bat_nb(i + 1, nx, PDE::POLICY), iw = bat_nb(i - 1, nx, PDE::POLICY);
    const int jn = bat_nb(j + 1, ny, PDE::POLICY), js = bat_nb(j - 1, ny, PDE::POLICY);
    const long long rj = (long long)j * nx, rn = (long long)jn * nx, rs = (long long)js * nx;
    Nb<V, NF> q;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      q.c[f] = ld(f, rj + i);
      q.e[f] = ld(f, rj + ie);
      q.w[f] = ld(f, rj + iw);
      q.n[f] = ld(f, rn + i);
      q.s[f] = ld(f, rs + i);
      if constexpr (PDE::DIAG) {
        q.ne[f] = ld(f, rn + ie);
        q.nw[f] = ld(f, rn + iw);
        q.se[f] = ld(f, rs + ie);
        q.sw[f] = ld(f, rs + iw);
      }
    }
    CellAux<T> aux;
    aux.eps = T(1); aux.fr = T(0); aux.fi = T(0); aux.gr = T(0); aux.gi = T(0);
    if constexpr (PDE::AUX) {
      const T* ep = eps_of<T>(P);
      const T* sp = src_of<T>(P);
      if (ep) aux.eps = ep[c];
      if (sp) { aux.fr = sp[c]; aux.fi = sp[P.ncell + c]; }
    }
    V M[NF], G[NF];
    PDE::template cell<T, V>(P, i, j, q, aux, M, G);
    out(c, M, G, q.c);
  }
}

// Sum of K per-thread values over the CTA (fixed order) into dst[0..K).
template <int K>
__device__ __forceinline__ void bat_unit_sum(double (&v)[K], double* dst) {
  __shared__ double red[kBatThreads / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) red[warp][k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][k];
      dst[k] = s;
    }
  }
  __syncthreads();
}

// Maxima of two per-thread values over the CTA into dst[0..2).
__device__ __forceinline__ void bat_unit_max2(double (&v)[2], double* dst) {
  __shared__ double red[kBatThreads / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    double s = v[k];
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane == 0) red[warp][k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w][k]);
      dst[k] = s;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// per-tile work of each phase
// ---------------------------------------------------------------------------
template <class PDE, class TS, class TJ>
struct BatTile {
  typedef typename BatAcc<TJ>::type A;    // Krylov arithmetic
  typedef typename BatAcc<TS>::type AS;   // Newton-step update arithmetic
  static constexpr int NF = PDE::NF;
  static constexpr bool MIXED = !std::is_same<TS, TJ>::value;

  // FD step of Eq. 7 / Eq. 8 from the solve's rule (identical in every tile)
  __device__ static TJ fd_eps(const BatDesc& D, const BatState& S, bool restart) {
    double eps;
    if (D.fd_eps > 0.0) {
      eps = D.fd_eps;
    } else {
      const double sq = sqrt(bat_eps_mach<TJ>());
      const double xn = sqrt(S.xn2[S.cur]);
      if (D.fd_rule == 1) {
        eps = sq * (xn > 1.0 ? xn : 1.0);
      } else {
        const double vn = restart ? sqrt(S.dn2) : 1.0;
        eps = sq * (1.0 + xn) / vn;
      }
    }
    return TJ(eps);
  }

  // F(x + alpha d) over the tile: (FP32 copy), F, ||F||^2, ||x + alpha d||^2 per unit
  __device__ static void residual(const BatDesc& D, const ProbDev& P, const BatState& S, int t, bool trial) {
    const long long nc = P.ncell;
    const TS* x = (const TS*)D.x[S.cur];
    const TS* dd = (const TS*)D.d;
    const TS al = TS(S.alpha);
    const TS* b = P.bvp ? nullptr : (const TS*)D.b;
    const int o = trial ? 1 - S.cur : S.cur;
    TS* Fo = (TS*)D.F[o];
    TS* xo = trial ? (TS*)D.x[o] : nullptr;
    float* x32o = MIXED ? D.x32[o] : nullptr;
    const TS thdt = TS(P.thdt);
    const long long u0 = (long long)t * (D.tc / kBatUnit);
    const long long u1 = min(u0 + D.tc / kBatUnit, (long long)D.nunit);
    for (long long u = u0; u < u1; ++u) {
      const long long c0 = u * kBatUnit, c1 = min(c0 + kBatUnit, nc);
      double acc[2] = {0.0, 0.0};
      auto ld = [&](int f, long long id) -> TS {
        const long long k = f * nc + id;
        return trial ? x[k] + al * dd[k] : x[k];
      };
      auto out = [&](long long c, const TS* M, const TS* G, const TS* xc) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const long long k = f * nc + c;
          TS Fv = P.bvp ? G[f] : M[f] - thdt * G[f];
          if (b) Fv -= b[k];
          Fo[k] = Fv;
          if (xo) xo[k] = xc[f];
          if (x32o) x32o[k] = (float)xc[f];
          acc[0] += (double)Fv * (double)Fv;
          acc[1] += (double)xc[f] * (double)xc[f];
        }
      };
      bat_cells<PDE, TS, TS>(P, c0, c1, ld, out);
      bat_unit_sum<2>(acc, D.part + u * kBatPart);
    }
  }

  // b = M(x^n) + (1 - theta) dt G(x^n)
  __device__ static void rhs(const BatDesc& D, const ProbDev& P, const BatState& S, long long c0, long long c1) {
    const long long nc = P.ncell;
    const TS* x = (const TS*)D.x[S.cur];
    TS* b = (TS*)D.b;
    float* b32 = D.b32;
    const TS co = TS(P.c_old);
    auto ld = [&](int f, long long id) -> TS { return x[f * nc + id]; };
    auto out = [&](long long c, const TS* M, const TS* G, const TS*) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const long long k = f * nc + c;
        const TS v = M[f] + co * G[f];
        b[k] = v;
        if (MIXED) b32[k] = (float)v;
      }
    };
    bat_cells<PDE, TS, TS>(P, c0, c1, ld, out);
  }

  // F(x) in FP32 at the FP32 copy of x (FD quotient of a mixed solve)
  __device__ static void fx32(const BatDesc& D, const ProbDev& P, const BatState& S, long long c0, long long c1) {
    const long long nc = P.ncell;
    const float* x = D.x32[S.cur];
    const float* b = P.bvp ? nullptr : D.b32;
    float* Fo = D.F32;
    const float thdt = float(P.thdt);
    auto ld = [&](int f, long long id) -> float { return x[f * nc + id]; };
    auto out = [&](long long c, const float* M, const float* G, const float*) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const long long k = f * nc + c;
        float Fv = P.bvp ? G[f] : M[f] - thdt * G[f];
        if (b) Fv -= b[k];
        Fo[k] = Fv;
      }
    };
    bat_cells<PDE, float, float>(P, c0, c1, ld, out);
  }

  // Jacobian-vector product in the JVP precision. Arnoldi: w = J (s u_j).
  // Restart: u_0 = rhs - J d with ||u_0||^2 per unit.
  __device__ static void jvp(const BatDesc& D, const ProbDev& P, const BatState& S, int t, bool restart) {
    const long long nc = P.ncell, N = D.N;
    const TJ* xj = MIXED ? (const TJ*)D.x32[S.cur] : (const TJ*)D.x[S.cur];
    const TJ* bj = P.bvp ? nullptr : (MIXED ? (const TJ*)D.b32 : (const TJ*)D.b);
    const TJ* Fx = MIXED ? (const TJ*)D.F32 : (const TJ*)D.F[S.cur];
    const TJ* u = restart ? nullptr : (const TJ*)D.V + (long long)S.j * N;
    const TS* dd = (const TS*)D.d;
    const TJ s = restart ? TJ(1) : TJ(S.g.scale[S.j]);
    const TJ thdt = TJ(P.thdt);
    TJ* w = (TJ*)D.w;
    TJ* u0 = (TJ*)D.V;
    const TJ* rhsv = (const TJ*)D.rhs;
    const bool fd = D.lin == 1;
    const TJ eps = fd ? fd_eps(D, S, restart) : TJ(1);
    const TJ es = eps * s;
    auto dir = [&](long long k) -> TJ { return restart ? (TJ)dd[k] : u[k]; };
    const long long ub0 = (long long)t * (D.tc / kBatUnit);
    const long long ub1 = min(ub0 + D.tc / kBatUnit, (long long)D.nunit);
    for (long long ub = ub0; ub < ub1; ++ub) {
      const long long c0 = ub * kBatUnit, c1 = min(c0 + kBatUnit, nc);
      double acc[1] = {0.0};
      auto emit = [&](long long k, TJ jv) {
        if (restart) {
          TJ o = TJ(-1) * jv;
          o += TJ(1) * rhsv[k];
          u0[k] = o;
          acc[0] += (double)o * (double)o;
        } else {
          w[k] = jv;
        }
      };
      if (!fd) {
        typedef Dual<TJ> DV;
        auto ld = [&](int f, long long id) -> DV {
          const long long k = f * nc + id;
          return DV(xj[k], s * dir(k));
        };
        auto out = [&](long long c, const DV* M, const DV* G, const DV*) {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const DV Fd = P.bvp ? G[f] : M[f] - thdt * G[f];
            emit(f * nc + c, Fd.d);
          }
        };
        bat_cells<PDE, TJ, DV>(P, c0, c1, ld, out);
      } else {
        auto ld = [&](int f, long long id) -> TJ {
          const long long k = f * nc + id;
          return xj[k] + es * dir(k);
        };
        auto out = [&](long long c, const TJ* M, const TJ* G, const TJ*) {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const long long k = f * nc + c;
            TJ Fp = P.bvp ? G[f] : M[f] - thdt * G[f];
            if (bj) Fp -= bj[k];
            emit(k, (Fp - Fx[k]) / eps);
          }
        };
        bat_cells<PDE, TJ, TJ>(P, c0, c1, ld, out);
      }
      if (restart) bat_unit_sum<1>(acc, D.part + ub * kBatPart);
    }
  }

  // per-unit dots u_i . ws (i < k) from the staged tile of w; warp per (unit, i)
  __device__ static void unit_dots(const BatDesc& D, int t, int k, const A* ws, long long c0, long long tcl) {
    const long long nc = D.P.ncell, N = D.N;
    const TJ* V = (const TJ*)D.V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long ub0 = (long long)t * (D.tc / kBatUnit);
    const long long ub1 = min(ub0 + D.tc / kBatUnit, (long long)D.nunit);
    const int pairs = (int)(ub1 - ub0) * k;
    for (int p = warp; p < pairs; p += nw) {
      const long long ub = ub0 + p / k;
      const int i = p % k;
      const long long cu0 = ub * kBatUnit, cu1 = min(cu0 + kBatUnit, nc);
      const TJ* ui = V + (long long)i * N;
      A acc = A(0);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        for (long long c = cu0 + lane; c < cu1; c += 32) acc += (A)ui[f * nc + c] * ws[f * tcl + (c - c0)];
      acc = warp_sum(acc);
      if (lane == 0) D.part[ub * kBatPart + i] = (double)acc;
    }
  }

  // Arnoldi passes over the tile
  __device__ static void arnoldi(const BatDesc& D, const BatState& S, int t, int pass, A* ws) {
    __shared__ A coef[kMaxM + 1];
    const long long nc = D.P.ncell, N = D.N;
    const long long c0 = (long long)t * D.tc, c1 = min(c0 + D.tc, nc), tcl = c1 - c0;
    const int k = S.j + 1;
    TJ* w = (TJ*)D.w;
    const TJ* V = (const TJ*)D.V;
    if (pass >= 2) {
      const double* h = pass == 2 ? S.g.h1 : S.g.h2;
      for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = (A)(h[i] * S.g.scale[i]);
    }
    __syncthreads();
    if (pass == 1) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
        for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) ws[f * tcl + (c - c0)] = (A)w[f * nc + c];
      __syncthreads();
      unit_dots(D, t, k, ws, c0, tcl);
    } else if (pass == 2) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
        for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
          const long long g = f * nc + c;
          A wv = (A)w[g];
          for (int i = 0; i < k; ++i) wv -= coef[i] * (A)V[(long long)i * N + g];
          w[g] = (TJ)wv;
          ws[f * tcl + (c - c0)] = wv;
        }
      __syncthreads();
      unit_dots(D, t, k, ws, c0, tcl);
    } else {
      TJ* un = (TJ*)D.V + (long long)k * N;
      const long long ub0 = (long long)t * (D.tc / kBatUnit);
      const long long ub1 = min(ub0 + D.tc / kBatUnit, (long long)D.nunit);
      for (long long ub = ub0; ub < ub1; ++ub) {
        const long long c = ub * kBatUnit + threadIdx.x;
        double acc[1] = {0.0};
        if (c < nc) {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const long long g = f * nc + c;
            A wv = (A)w[g];
            for (int i = 0; i < k; ++i) wv -= coef[i] * (A)V[(long long)i * N + g];
            un[g] = (TJ)wv;
            acc[0] += (double)wv * (double)wv;
          }
        }
        bat_unit_sum<1>(acc, D.part + ub * kBatPart);
      }
    }
  }

  // d += sum_i y_i u_i (y already scaled), ||d||^2 per unit
  __device__ static void update(const BatDesc& D, const BatState& S, int t) {
    __shared__ AS yc[kMaxM];
    const long long nc = D.P.ncell, N = D.N;
    const int k = S.g.k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) yc[i] = (AS)S.g.y[i];
    __syncthreads();
    TS* d = (TS*)D.d;
    const TJ* V = (const TJ*)D.V;
    const long long ub0 = (long long)t * (D.tc / kBatUnit);
    const long long ub1 = min(ub0 + D.tc / kBatUnit, (long long)D.nunit);
    for (long long ub = ub0; ub < ub1; ++ub) {
      const long long c = ub * kBatUnit + threadIdx.x;
      double acc[1] = {0.0};
      if (c < nc) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const long long g = f * nc + c;
          AS s = AS(0);
          for (int i = 0; i < k; ++i) s += yc[i] * (AS)V[(long long)i * N + g];
          const TS dn = d[g] + (TS)s;
          d[g] = dn;
          acc[0] += (double)dn * (double)dn;
        }
      }
      bat_unit_sum<1>(acc, D.part + ub * kBatPart);
    }
  }

  // Delayed CGS2, dots of step j (Sec. 3; the single-solve form is dcgs_step in
  // ctl.cuh): per unit, q_i . u_j and q_i . w for i <= j (slot j holds the
  // candidate u_j), warp per (unit, i); without w (the last step of a cycle,
  // j = m) the w entries are zero.
  __device__ static void dcgs_dots(const BatDesc& D, const BatState& S, int t) {
    const long long nc = D.P.ncell, N = D.N;
    const int j = S.j, k = j + 1;
    const bool has_w = j < S.g.m;
    const TJ* V = (const TJ*)D.V;
    const TJ* uj = V + (long long)j * N;
    const TJ* w = (const TJ*)D.w;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long ub0 = (long long)t * (D.tc / kBatUnit);
    const long long ub1 = min(ub0 + D.tc / kBatUnit, (long long)D.nunit);
    const int pairs = (int)(ub1 - ub0) * k;
    for (int p = warp; p < pairs; p += nw) {
      const long long ub = ub0 + p / k;
      const int i = p % k;
      const long long cu0 = ub * kBatUnit, cu1 = min(cu0 + kBatUnit, nc);
      const TJ* qi = V + (long long)i * N;
      A au = A(0), aw = A(0);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        for (long long c = cu0 + lane; c < cu1; c += 32) {
          const long long g = f * nc + c;
          const A q = (A)qi[g];
          au += q * (A)uj[g];
          if (has_w) aw += q * (A)w[g];
        }
      au = warp_sum(au);
      aw = warp_sum(aw);
      if (lane == 0) {
        D.part[ub * kBatPart + 2 * i] = (double)au;
        D.part[ub * kBatPart + 2 * i + 1] = (double)aw;
      }
    }
  }

  // Delayed CGS2, update of step j from the step's coefficients:
  // q_j = dgamma u_j - sum_i da_i q_i (over slot j), u_{j+1} = dinvr (w -
  // sum_i dc_i q_i - dc_j q_j) (slot j + 1), ||u_{j+1}||^2 per unit.
  __device__ static void dcgs_update(const BatDesc& D, const BatState& S, int t) {
    __shared__ A ca[kMaxM + 1], cc[kMaxM + 1], s_gi[2];
    const long long nc = D.P.ncell, N = D.N;
    const int j = S.j;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      ca[i] = (A)S.g.da[i];
      cc[i] = (A)S.g.dc[i];
    }
    if (threadIdx.x == 0) { s_gi[0] = (A)S.g.dgamma; s_gi[1] = (A)S.g.dinvr; }
    __syncthreads();
    const A gam = s_gi[0], invr = s_gi[1], cj = cc[j];
    TJ* V = (TJ*)D.V;
    const TJ* w = (const TJ*)D.w;
    const long long ub0 = (long long)t * (D.tc / kBatUnit);
    const long long ub1 = min(ub0 + D.tc / kBatUnit, (long long)D.nunit);
    for (long long ub = ub0; ub < ub1; ++ub) {
      const long long c = ub * kBatUnit + threadIdx.x;
      double acc[1] = {0.0};
      if (c < nc) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const long long g = f * nc + c;
          A q = gam * (A)V[(long long)j * N + g];
          A y = (A)w[g];
          for (int i = 0; i < j; ++i) {
            const A v = (A)V[(long long)i * N + g];
            q -= ca[i] * v;
            y -= cc[i] * v;
          }
          const TJ qs = (TJ)q;
          const TJ ys = (TJ)((y - cj * (A)qs) * invr);
          V[(long long)j * N + g] = qs;
          V[(long long)(j + 1) * N + g] = ys;
          acc[0] += (double)ys * (double)ys;
        }
      }
      bat_unit_sum<1>(acc, D.part + ub * kBatPart);
    }
  }

  // per unit: max|u|, max|v| of the state (a non-finite value counts as +Inf)
  __device__ static void cfl_max(const BatDesc& D, const ProbDev& P, const BatState& S, int t) {
    const long long nc = P.ncell;
    const TS* x = (const TS*)D.x[S.cur];
    const long long u0 = (long long)t * (D.tc / kBatUnit);
    const long long u1 = min(u0 + D.tc / kBatUnit, (long long)D.nunit);
    for (long long u = u0; u < u1; ++u) {
      const long long c = u * kBatUnit + threadIdx.x;
      double m[2] = {0.0, 0.0};
      if (c < nc) {
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const double a = fabs((double)x[f * nc + c]);
          m[f] = a <= 1.7976931348623157e308 ? a : 1.0 / 0.0;
        }
      }
      bat_unit_max2(m, D.part + u * kBatPart);
    }
  }

  __device__ static void work(const BatDesc& D, const BatState& S, int ph, int t, A* ws) {
    ProbDev P = D.P;
    if (D.born && S.stage == 0) P.p1 = 0.0;     // Born stage: the chi3 = 0 problem
    if (P.cfl > 0.0) { P.thdt = S.thdt; P.c_old = S.c_old; }   // adaptive step of this implicit step
    const long long nc = P.ncell;
    const long long c0 = (long long)t * D.tc, c1 = min(c0 + D.tc, nc);
    switch (ph) {
      case PH_IN: {
        TS* x = (TS*)D.x[0];
        const bool zero = D.born && S.stage == 0;
#pragma unroll
        for (int f = 0; f < NF; ++f)
          for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x)
            x[f * nc + c] = zero ? TS(0) : (TS)D.io[f * nc + c];
        break;
      }
      case PH_CFL: if constexpr (PDE::NF == 2) cfl_max(D, P, S, t); break;
      case PH_RHS: rhs(D, P, S, c0, c1); break;
      case PH_RES: residual(D, P, S, t, false); break;
      case PH_LS: residual(D, P, S, t, true); break;
      case PH_FX32: if constexpr (MIXED) fx32(D, P, S, c0, c1); break;
      case PH_GINIT: {
        const TS* F = (const TS*)D.F[S.cur];
        TJ* u0 = (TJ*)D.V;
        TJ* r = (TJ*)D.rhs;
        TS* d = (TS*)D.d;
#pragma unroll
        for (int f = 0; f < NF; ++f)
          for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const long long g = f * nc + c;
            const TS fv = F[g];
            u0[g] = (TJ)(-fv);
            r[g] = (TJ)(-fv);
            d[g] = TS(0);
          }
        break;
      }
      case PH_JVP: jvp(D, P, S, t, false); break;
      case PH_RJVP: jvp(D, P, S, t, true); break;
      case PH_A1: arnoldi(D, S, t, 1, ws); break;
      case PH_A2: arnoldi(D, S, t, 2, ws); break;
      case PH_A3: arnoldi(D, S, t, 3, ws); break;
      case PH_D1: dcgs_dots(D, S, t); break;
      case PH_D2: dcgs_update(D, S, t); break;
      case PH_GUPD: update(D, S, t); break;
      case PH_OUT: {
        const TS* x = (const TS*)D.x[S.cur];
#pragma unroll
        for (int f = 0; f < NF; ++f)
          for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) D.io[f * nc + c] = (double)x[f * nc + c];
        break;
      }
      default: break;
    }
  }
};

// ---------------------------------------------------------------------------
// scalar steps (thread 0 of the CTA that finished the solve's last tile)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bat_end_solve(const BatDesc& D, BatState& S, int ns) {
  S.res_final = S.fnorm;
  if (D.born && S.stage == 0) {
    // the Born solve contributes its Krylov iterations and JVPs only
    S.newton_its = 0; S.ls_backtracks = 0; S.ls_failures = 0; S.krylov_failures = 0;
    S.stage = 1;
    S.newton_it = 0;
    S.fresh = 1;
    S.phase = PH_RES;
    return;
  }
  const bool ok = (S.res0 == 0.0 || S.res_final / S.res0 < 100.0 * D.tol_newton);
  S.status = ns;
  if (ns != 0 && S.first_bad == 0) S.first_bad = ns;
  if (D.P.bvp) {
    S.steps_done = 1;
    S.steps_failed = ok ? 0 : 1;
    S.phase = PH_OUT;
    return;
  }
  S.steps_done += 1;
  if (!ok) S.steps_failed += 1;
  if (ns == JFNK_E_NONFINITE || ns == JFNK_E_BREAKDOWN) { S.phase = PH_OUT; return; }
  S.step += 1;
  S.phase = S.step < D.steps ? (D.P.cfl > 0.0 ? PH_CFL : PH_RHS) : PH_OUT;
}

__device__ __forceinline__ void bat_newton_test(const BatDesc& D, BatState& S) {
  const double fn = S.fnorm, f0 = S.f0;
  const bool linear_once = D.born && S.stage == 0;
  if (!isfinite(fn)) {
    bat_end_solve(D, S, JFNK_E_NONFINITE);
  } else if (f0 == 0.0 || fn / f0 < D.tol_newton) {
    bat_end_solve(D, S, 0);
  } else if (S.newton_it == D.max_newton || (linear_once && S.newton_it == 1)) {
    bat_end_solve(D, S, JFNK_E_NOT_CONVERGED);
  } else {
    S.cycle = 0;
    S.phase = (D.lin == 1 && D.ts != D.tj) ? PH_FX32 : PH_GINIT;
  }
}

__device__ __forceinline__ void bat_after_cycle(const BatDesc& D, BatState& S) {
  GmresCtl& g = S.g;
  if (g.nonfinite) {
    S.krylov_its += g.its;
    bat_end_solve(D, S, JFNK_E_NONFINITE);
  } else if (g.converged || S.cycle == D.max_krylov - 1) {
    S.krylov_its += g.its;
    if (!g.converged) S.krylov_failures += 1;
    S.alpha = 1.0;
    S.phase = PH_LS;
  } else {
    S.cycle += 1;
    S.phase = PH_RJVP;
  }
}

__device__ __forceinline__ void bat_cycle_end(const BatDesc& D, BatState& S) {
  GmresCtl& g = S.g;
  const int k = g.k;
  if (k == 0) { bat_after_cycle(D, S); return; }
  // back substitution H[:k,:k] y = g[:k], then y_t *= scale_t
  double* y = g.y;
  for (int t = 0; t < k; ++t) y[t] = g.g[t];
  for (int i = k - 1; i >= 0; --i) {
    const double* col = g.H + (size_t)i * (kMaxM + 1);
    y[i] = y[i] / col[i];
    const double yi = y[i];
    for (int t = 0; t < i; ++t) y[t] -= col[t] * yi;
  }
  for (int t = 0; t < k; ++t) y[t] *= g.scale[t];
  S.phase = PH_GUPD;
}

__device__ __forceinline__ void bat_control(const BatDesc& D, BatState& S, int ph, const double* sum, bool go) {
  GmresCtl& g = S.g;
  if (S.stage == 2) {   // tile-size probe: the four phases of an Arnoldi step in a loop, fixed j
    S.phase = (ph == PH_A3) ? PH_JVP : ph + 1;
    return;
  }
  switch (ph) {
    case PH_IN:
      S.fresh = 1;
      S.newton_it = 0;
      S.dt = D.P.dt; S.thdt = D.P.thdt; S.c_old = D.P.c_old;
      S.phase = D.P.bvp ? PH_RES : (D.P.cfl > 0.0 ? PH_CFL : PH_RHS);
      break;
    case PH_CFL: {
      const double dt = cfl_rule(sum[0], sum[1], D.P.hx, D.P.hy, D.P.p0, D.P.cfl);
      S.dt = dt;
      if (dt > 0.0 && dt <= 1.7976931348623157e308) {
        S.thdt = D.P.theta * dt;
        S.c_old = (1.0 - D.P.theta) * dt;
        S.phase = PH_RHS;
      } else {
        // non-finite state (NaN) or an undefined rule (+Inf: nu = 0 and the state at rest)
        const int ns = (dt == dt) ? JFNK_E_INVALID : JFNK_E_NONFINITE;
        S.status = ns;
        if (S.first_bad == 0) S.first_bad = ns;
        S.steps_failed += 1;
        S.phase = PH_OUT;
      }
      break;
    }
    case PH_RHS:
      S.fresh = 1;
      S.newton_it = 0;
      S.phase = PH_RES;
      break;
    case PH_RES:
      S.fn2 = sum[0];
      S.fnorm = sqrt(sum[0]);
      S.xn2[S.cur] = sum[1];
      if (S.fresh) { S.f0 = S.fnorm; S.res0 = S.f0; S.fresh = 0; }
      bat_newton_test(D, S);
      break;
    case PH_FX32:
      S.phase = PH_GINIT;
      break;
    case PH_GINIT:
      g.m = D.m;
      g.its = 0;
      g.converged = 0; g.breakdown = 0; g.nonfinite = 0;
      g.host_active = nullptr;
      g.bnorm = sqrt(S.fn2);
      g.target = D.tol_krylov * g.bnorm;
      gmres_cycle_start(&g, S.fn2);
      S.j = 0;
      if (g.active) S.phase = PH_JVP; else bat_after_cycle(D, S);
      break;
    case PH_JVP:
      S.jvp_calls += 1;
      S.phase = D.ortho == JFNK_DCGS2 ? PH_D1 : PH_A1;
      break;
    case PH_D1:   // the coefficient step ran on the whole CTA (k_batch); go: the update pass follows
      if (go) S.phase = PH_D2; else bat_cycle_end(D, S);
      break;
    case PH_D2:
      dcgs_after_update(&g, S.j, sum[0]);
      if (g.nonfinite) {
        bat_after_cycle(D, S);
      } else {
        S.j += 1;   // the next step, or (j = m) the last dots pass of the cycle, which has no w
        S.phase = S.j < g.m ? PH_JVP : PH_D1;
      }
      break;
    case PH_A1:
      for (int i = 0; i <= S.j; ++i) g.h1[i] = sum[i] * g.scale[i];
      S.phase = PH_A2;
      break;
    case PH_A2:
      for (int i = 0; i <= S.j; ++i) g.h2[i] = sum[i] * g.scale[i];
      S.phase = PH_A3;
      break;
    case PH_A3:
      gmres_givens_step(&g, S.j, sum[0]);
      if (g.active) { S.j += 1; S.phase = PH_JVP; } else bat_cycle_end(D, S);
      break;
    case PH_GUPD:
      S.dn2 = sum[0];
      bat_after_cycle(D, S);
      break;
    case PH_RJVP:
      S.jvp_calls += 1;
      gmres_cycle_start(&g, sum[0]);
      S.j = 0;
      if (g.active) S.phase = PH_JVP; else bat_after_cycle(D, S);
      break;
    case PH_LS: {
      const double ft = sqrt(sum[0]);
      bool accept = (D.born && S.stage == 0) || (isfinite(ft) && ft <= (1.0 - D.ls_c1 * S.alpha) * S.fnorm);
      if (!accept) {
        if (S.alpha * 0.5 < D.ls_min_alpha) {
          S.ls_failures += 1;
          accept = true;
        } else {
          S.alpha *= 0.5;
          S.ls_backtracks += 1;
        }
      }
      if (accept) {
        S.cur ^= 1;
        S.fn2 = sum[0];
        S.fnorm = ft;
        S.xn2[S.cur] = sum[1];
        S.newton_it += 1;
        S.newton_its += 1;
        bat_newton_test(D, S);
      }
      break;
    }
    case PH_OUT:
      S.phase = PH_DONE;
      *D.done_flag = 1;
      break;
    default:
      break;
  }
}

__device__ __forceinline__ int bat_nvals(const BatState& S, int ph) {
  switch (ph) {
    case PH_RES: case PH_LS: case PH_CFL: return 2;
    case PH_A1: case PH_A2: return S.j + 1;
    case PH_D1: return 2 * (S.j + 1);
    case PH_A3: case PH_GUPD: case PH_RJVP: case PH_D2: return 1;
    default: return 0;
  }
}

// The delayed-CGS2 coefficient step of a solve (dcgs_step_t, ctl.cuh) on the
// CTA that finished its dots pass, from the unit sums S: the scalars and the
// previous column's first projection and rotations are staged in shared
// memory, the completed Hessenberg columns are read from the solve's state.
__device__ __forceinline__ bool bat_dcgs_step(BatState& S, const double* sum) {
  constexpr int LD = kMaxM + 1;
  __shared__ double sh[5 * LD];
  __shared__ double hcol[LD];
  GmresCtl& g = S.g;
  const int j = S.j, cj = j - 1;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    sh[2 * LD + i] = g.hprev[i];
    if (i < cj) { sh[3 * LD + i] = g.cs[i]; sh[4 * LD + i] = g.sn[i]; }
  }
  const double sigma = g.scale[j], g_prev = j > 0 ? g.g[j - 1] : g.g[0], target = g.target;
  const int m = g.m, active = g.active, its = g.its;
  __syncthreads();
  return dcgs_step_t<BlockTeam, false, double>(&g, j, sum, j < m, sh, hcol, sigma, 1.0 / sigma, g_prev, target, m,
                                               active, its, BlockTeam{}, true, g.da, g.dc, &g.dgamma, &g.dinvr);
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <class PDE, class TS, class TJ>
__global__ void __launch_bounds__(kBatThreads) k_batch(BatLaunch L) {
  typedef BatTile<PDE, TS, TJ> Tile;
  typedef typename Tile::A A;
  extern __shared__ __align__(16) unsigned char bat_smem[];
  __shared__ int s_item, s_phase, s_last;
  __shared__ double s_sum[kBatPart];
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(L.next, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= L.nitems) break;
    const int2 item = L.items[it];
    const BatDesc& D = L.desc[item.x];
    BatState& S = *D.st;
    if (threadIdx.x == 0) s_phase = S.phase;
    __syncthreads();
    const int ph = s_phase;
    if (ph != PH_DONE) {
      Tile::work(D, S, ph, item.y, (A*)bat_smem);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(&S.arrive, 1u) == (unsigned)(D.ntile - 1));
      __syncthreads();
      if (s_last) {
        __threadfence();
        const int nv = bat_nvals(S, ph);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int v = warp; v < nv; v += nw) {
          double s;
          if (ph == PH_CFL) {
            s = 0.0;
            for (int u = lane; u < D.nunit; u += 32) s = fmax(s, D.part[(size_t)u * kBatPart + v]);
            for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
          } else {
            s = lane_strided_sum(D.part + v, kBatPart, D.nunit, lane);
            s = warp_sum(s);
          }
          if (lane == 0) s_sum[v] = s;
        }
        __syncthreads();
        bool go = false;
        if (ph == PH_D1 && S.stage != 2) go = bat_dcgs_step(S, s_sum);   // every thread of the CTA
        if (threadIdx.x == 0) {
          S.arrive = 0u;
          bat_control(D, S, ph, s_sum, go);
          __threadfence();
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(L.ndone, 1u) == gridDim.x - 1) {
      *L.next = 0u;
      *L.ndone = 0u;
      __threadfence();
    }
  }
}

// launch and occupancy of one PDE's kernels (TS, TJ) in {(f64, f64), (f32, f32), (f64, f32)}
template <class PDE>
cudaError_t batch_launch_pde(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st) {
  const size_t smem = (size_t)PDE::NF * 2048 * (tj == VT_F64 ? 8 : 4);
  if (grid < 1) return cudaSuccess;
  if (ts == VT_F64 && tj == VT_F64) k_batch<PDE, double, double><<<grid, kBatThreads, smem, st>>>(L);
  else if (ts == VT_F32 && tj == VT_F32) k_batch<PDE, float, float><<<grid, kBatThreads, smem, st>>>(L);
  else if (ts == VT_F64 && tj == VT_F32) k_batch<PDE, double, float><<<grid, kBatThreads, smem, st>>>(L);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <class PDE>
int batch_occ_pde(int ts, int tj) {
  const size_t smem = (size_t)PDE::NF * 2048 * (tj == VT_F64 ? 8 : 4);
  int n = 0;
  cudaError_t e;
  if (ts == VT_F64 && tj == VT_F64)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<PDE, double, double>, kBatThreads, smem);
  else if (ts == VT_F32 && tj == VT_F32)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<PDE, float, float>, kBatThreads, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<PDE, double, float>, kBatThreads, smem);
  if (e != cudaSuccess) { cudaGetLastError(); return 1; }
  return n > 0 ? n : 1;
}

}  // namespace jfnk
