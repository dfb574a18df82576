// stencil_impl.cuh -- residual, right-hand-side and Jacobian-vector-product sweeps.
//
// The same per-cell residual source (pdes.cuh) is instantiated on plain
// numbers for F(x), the constant part b of an implicit step and the FD
// quotient (Eq. 7), and on dual numbers for the AD product (F(x), J(x) v)
// (Eq. 9). Two launch forms feed it the 3 x 3 neighbourhood of each cell:
//
// * march: each warp owns a strip of 32 * VEC columns (VEC consecutive cells
//   per lane, one 16-byte load per lane per row) and walks down a band of
//   rows, keeping the rows above, at and below the current one in registers
//   and prefetching the row after next; east/west neighbours come from the
//   adjacent lane by warp shuffle. Every input element is read from HBM once
//   (plus the two halo rows of each band, which the neighbouring band has
//   usually just pulled into L2).
// * gather: one thread per cell reads its neighbours directly; used when the
//   row length or the pointers do not allow aligned 16-byte vectors.
#pragma once

#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "kernels.h"
#include "ctl.cuh"
#include "stream.cuh"

namespace jfnk {

enum StencilMode { SM_RESID = 0, SM_RHS = 1, SM_AD = 2, SM_FD = 3, SM_PREC = 4 };

struct StencilArgs {
  const void* x;            // state (T)
  const void* v;            // RESID: direction d (T) or null; AD/FD: direction (TV)
  const double* vscale;     // AD/FD: multiplier s of v (null: 1)
  double alpha;             // RESID: the state is x + alpha d
  const void* b;            // theta-method constant (T) or null
  void* F;                  // RESID, AD: F output (T) or null
  void* out;                // RHS: b output; AD, FD: c_jv Jv + c_add add
  void* xout;               // RESID: x + alpha d (T) or null
  float* x32;               // RESID: (float)(x + alpha d) or null
  const void* Fx;           // FD: F(x) (T)
  double c_jv, c_add;
  const void* add;
  int ndots;                // AD, FD: out . dw[k] (dw[k] null: out . out)
  const void* dw[3];
  double* sums;             // RESID: ||F||^2, ||x + alpha d||^2 when not null
  int post;
  void* post_arg;
  double eps_fixed;
  int eps_rule;
  const double* xn2;
  const double* vn2;
  float* eps_out;
  const int* active;
  LsCtl* ls;                // RESID: a line-search trial, alpha from ls->alpha (see LsCtl)
  unsigned int* err;        // AD, FD: device error word of the staged form's bounded waits (null: march form)
  int pdl;                  // staged form: launched programmatically after the previous kernel, which
                            // must not write x (the staged form starts loading x before its dependency wait)
  int precond;              // AD, FD: the direction is M^-1 v (PDE::precond at each node; gather form)
  double pbeta;             // damping beta of the preconditioner
};

template <class T> struct AccOf { typedef float type; };
template <> struct AccOf<double> { typedef double type; };

template <class T> __device__ __forceinline__ T eps_mach();
template <> __device__ __forceinline__ double eps_mach<double>() { return 2.220446049250313e-16; }
template <> __device__ __forceinline__ float eps_mach<float>() { return 1.1920928955078125e-07f; }

__device__ __forceinline__ float ldv1(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ldv1(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ double ldv1(const double* p, long long i) { return __ldg(p + i); }

// value of the state at which the residual is taken, from x and v entries
template <int MODE, class T> struct Comb;
template <class T> struct Comb<SM_RESID, T> {
  typedef T V;
  T a;
  __device__ __forceinline__ V operator()(T x, T v) const { return x + a * v; }
};
template <class T> struct Comb<SM_RHS, T> {
  typedef T V;
  __device__ __forceinline__ V operator()(T x, T) const { return x; }
};
template <class T> struct Comb<SM_AD, T> {
  typedef Dual<T> V;
  T s;
  __device__ __forceinline__ V operator()(T x, T v) const { return Dual<T>(x, s * v); }
};
template <class T> struct Comb<SM_FD, T> {
  typedef T V;
  T es;
  __device__ __forceinline__ V operator()(T x, T v) const { return x + es * v; }
};

template <int MODE, class T>
__device__ __forceinline__ Comb<MODE, T> make_comb(double alpha, T s, T eps) {
  Comb<MODE, T> cb;
  if constexpr (MODE == SM_RESID) cb.a = T(alpha);
  if constexpr (MODE == SM_AD) cb.s = s;
  if constexpr (MODE == SM_FD) cb.es = eps * s;
  return cb;
}

// --------------------------------------------------------------------------
// per-cell epilogue: write the outputs of cell c and accumulate reductions
// --------------------------------------------------------------------------
template <int MODE, class PDE, class T, class V, class Acc>
__device__ __forceinline__ void emit(const ProbDev& P, const StencilArgs& a, long long c, const V* M, const V* G,
                                     const V* xc, T eps, Acc* acc) {
  constexpr int NF = PDE::NF;
  const T thdt = T(P.thdt);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const long long id = f * P.ncell + c;
    if constexpr (MODE == SM_RHS) {
      ((T*)a.out)[id] = M[f] + T(P.c_old) * G[f];
    } else if constexpr (MODE == SM_RESID) {
      T Fv = P.bvp ? G[f] : M[f] - thdt * G[f];
      if (a.b) Fv -= ((const T*)a.b)[id];
      if (a.F) ((T*)a.F)[id] = Fv;
      const T xv = xc[f];
      if (a.xout) ((T*)a.xout)[id] = xv;
      if (a.x32) a.x32[id] = (float)xv;
      acc[0] += (Acc)Fv * (Acc)Fv;
      acc[1] += (Acc)xv * (Acc)xv;
    } else {
      T jv;
      if constexpr (MODE == SM_AD) {
        const V Fd = P.bvp ? G[f] : M[f] - thdt * G[f];
        jv = Fd.d;
        if (a.F) ((T*)a.F)[id] = a.b ? Fd.v - ((const T*)a.b)[id] : Fd.v;
      } else {
        T Fp = P.bvp ? G[f] : M[f] - thdt * G[f];
        if (a.b) Fp -= ((const T*)a.b)[id];
        jv = (Fp - ((const T*)a.Fx)[id]) / eps;
      }
      T o = T(a.c_jv) * jv;
      if (a.add) o += T(a.c_add) * ((const T*)a.add)[id];
      ((T*)a.out)[id] = o;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (k < a.ndots) {
          const T w = a.dw[k] ? ((const T*)a.dw[k])[id] : o;
          acc[k] += (Acc)o * (Acc)w;
        }
      }
    }
  }
}

// FD step from the rule or the fixed value, computed once per block
template <class T, int MODE>
__device__ __forceinline__ T fd_step(const StencilArgs& a, T s) {
  if constexpr (MODE != SM_FD) {
    return T(0);
  } else {
    __shared__ T s_eps;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double eps;
      if (a.eps_fixed > 0.0) {
        eps = a.eps_fixed;
      } else {
        const double sq = sqrt((double)eps_mach<T>());
        const double xn = sqrt(*a.xn2);
        if (a.eps_rule == 1) {
          eps = sq * (xn > 1.0 ? xn : 1.0);
        } else {
          double vn = a.vn2 ? sqrt(*a.vn2) * (double)s : 1.0;
          if (vn == 0.0) vn = 1.0;   // zero direction: keep the step finite (the quotient is then ~0)
          eps = sq * (1.0 + xn) / vn;
        }
      }
      s_eps = T(eps);
      if (a.eps_out && blockIdx.x == 0 && blockIdx.y == 0) *a.eps_out = (float)eps;
    }
    __syncthreads();
    return s_eps;
  }
}

template <int MODE, class Acc>
__device__ __forceinline__ void finish_reduction(const StencilArgs& a, Acc* acc, int nblocks, int blockLinear,
                                                 RedSite<Acc> red) {
  const int nd = (MODE == SM_RESID) ? (a.sums ? 2 : 0) : (MODE == SM_RHS ? 0 : a.ndots);
  if (nd == 0) return;
  __shared__ Acc sm[8 * 3];
  Acc v3[3] = {acc[0], acc[1], acc[2]};
  double* sums = a.sums;
  const bool last = grid_reduce<Acc, 3>(v3, nd, red, nblocks, blockLinear, sm,
                                        [&](int t, Acc sv) { sums[t] = (double)sv; });
  if constexpr (MODE == SM_RESID) {
    if (last && threadIdx.x == 0 && threadIdx.y == 0 && a.ls) ls_decide(a.ls, sums[0]);
  }
  if constexpr (MODE == SM_AD || MODE == SM_FD) {
    if (last && threadIdx.x == 0 && threadIdx.y == 0 && a.post == POST_GMRES_RESTART)
      gmres_cycle_start((GmresCtl*)a.post_arg, sums[0]);
  }
}

template <class PDE, class T>
__device__ __forceinline__ CellAux<T> load_aux(const ProbDev& P, long long c) {
  CellAux<T> aux;
  aux.eps = T(1); aux.fr = T(0); aux.fi = T(0); aux.gr = T(0); aux.gi = T(0);
  if (PDE::AUX) {
    const T* ep = eps_of<T>(P);
    const T* sp = src_of<T>(P);
    if (ep) aux.eps = __ldg(ep + c);
    if (sp) { aux.fr = __ldg(sp + c); aux.fi = __ldg(sp + P.ncell + c); }
    if (sp && PDE::NSRC >= 4) { aux.gr = __ldg(sp + 2 * P.ncell + c); aux.gi = __ldg(sp + 3 * P.ncell + c); }
  }
  return aux;
}

// --------------------------------------------------------------------------
// gather form: one thread per cell per row it owns
// --------------------------------------------------------------------------
__device__ __forceinline__ int bp_index(int i, int n, int policy) {
  if (i < 0) return policy == BP_WRAP ? i + n : 0;
  if (i >= n) return policy == BP_WRAP ? i - n : n - 1;
  return i;
}

template <class PDE, class T, class TV, int MODE>
__global__ void __launch_bounds__(256) k_gather(ProbDev P, int R, StencilArgs a, RedSite<typename AccOf<T>::type> red) {
  typedef typename AccOf<T>::type Acc;
  typedef Comb<MODE, T> CB;
  typedef typename CB::V V;
  constexpr int NF = PDE::NF;
  if (a.active && *a.active == 0) return;
  if (MODE == SM_RESID && a.ls && a.ls->done) return;
  const T s = (MODE == SM_AD || MODE == SM_FD) ? (a.vscale ? T(*a.vscale) : T(1)) : T(1);
  const T eps = fd_step<T, MODE>(a, s);
  const CB cb = make_comb<MODE, T>((MODE == SM_RESID && a.ls) ? a.ls->alpha : a.alpha, s, eps);
  const T* __restrict__ x = (const T*)a.x;
  const TV* __restrict__ v = (const TV*)a.v;
  Acc acc[3] = {Acc(0), Acc(0), Acc(0)};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int jbase = blockIdx.y * R * blockDim.y + threadIdx.y;
  for (int r = 0; r < R; ++r) {
    const int j = jbase + r * blockDim.y;
    if (i >= P.nx || j >= P.ny) continue;
    const int ie = bp_index(i + 1, P.nx, PDE::POLICY), iw = bp_index(i - 1, P.nx, PDE::POLICY);
    const int jn = bp_index(j + 1, P.ny, PDE::POLICY), js = bp_index(j - 1, P.ny, PDE::POLICY);
    Nb<V, NF> q;
    auto val = [&](long long id) -> V {
      const T xv = __ldg(x + id);
      const T vv = v ? (T)ldv1(v, id) : T(0);
      return cb(xv, vv);
    };
    if constexpr (PDE::PRECOND && (MODE == SM_AD || MODE == SM_FD)) {
      if (a.precond) {
        // every field of a node at once: the direction there becomes M^-1 v before it meets x
        auto node = [&](int ii, int jj, V* dst, int stride) {
          const long long cid = (long long)jj * P.nx + ii;
          T xv[NF], vv[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            xv[f] = __ldg(x + f * P.ncell + cid);
            vv[f] = (T)ldv1(v, f * P.ncell + cid);
          }
          PDE::precond(P, T(a.pbeta), ii, jj, xv, vv);
#pragma unroll
          for (int f = 0; f < NF; ++f) dst[f * stride] = cb(xv[f], vv[f]);
        };
        node(i, j, q.c, 1); node(ie, j, q.e, 1); node(iw, j, q.w, 1); node(i, jn, q.n, 1); node(i, js, q.s, 1);
        if (PDE::DIAG) {
          node(ie, jn, q.ne, 1); node(iw, jn, q.nw, 1); node(ie, js, q.se, 1); node(iw, js, q.sw, 1);
        }
        const long long c = (long long)j * P.nx + i;
        const CellAux<T> aux = load_aux<PDE, T>(P, c);
        V M[NF], G[NF];
        PDE::template cell<T, V>(P, i, j, q, aux, M, G);
        emit<MODE, PDE, T, V, Acc>(P, a, c, M, G, q.c, eps, acc);
        continue;
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long base = f * P.ncell;
      const long long rc = base + (long long)j * P.nx, rn = base + (long long)jn * P.nx,
                      rs = base + (long long)js * P.nx;
      q.c[f] = val(rc + i);
      q.e[f] = val(rc + ie);
      q.w[f] = val(rc + iw);
      q.n[f] = val(rn + i);
      q.s[f] = val(rs + i);
      if (PDE::DIAG) {
        q.ne[f] = val(rn + ie);
        q.nw[f] = val(rn + iw);
        q.se[f] = val(rs + ie);
        q.sw[f] = val(rs + iw);
      }
    }
    const long long c = (long long)j * P.nx + i;
    const CellAux<T> aux = load_aux<PDE, T>(P, c);
    V M[NF], G[NF];
    PDE::template cell<T, V>(P, i, j, q, aux, M, G);
    emit<MODE, PDE, T, V, Acc>(P, a, c, M, G, q.c, eps, acc);
  }
  finish_reduction<MODE, Acc>(a, acc, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x, red);
}

// --------------------------------------------------------------------------
// the right preconditioner alone, node by node: out = M^-1(x) v (out may be
// v itself or null) and, when sums is set, sums[0] = ||M^-1(x) v||^2
// --------------------------------------------------------------------------
template <class PDE, class T>
__global__ void __launch_bounds__(256) k_precond(ProbDev P, StencilArgs a, RedSite<typename AccOf<T>::type> red) {
  typedef typename AccOf<T>::type Acc;
  constexpr int NF = PDE::NF;
  const T* __restrict__ x = (const T*)a.x;
  const T* v = (const T*)a.v;
  T* out = (T*)a.out;
  Acc acc[3] = {Acc(0), Acc(0), Acc(0)};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < P.ncell; c += stride) {
    T xv[NF], vv[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      xv[f] = x[f * P.ncell + c];
      vv[f] = v[f * P.ncell + c];
    }
    if constexpr (PDE::PRECOND) PDE::precond(P, T(a.pbeta), (int)(c % P.nx), (int)(c / P.nx), xv, vv);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (out) out[f * P.ncell + c] = vv[f];
      acc[0] += (Acc)vv[f] * (Acc)vv[f];
    }
  }
  if (a.sums) {
    __shared__ Acc sm[8 * 3];
    Acc v3[3] = {acc[0], Acc(0), Acc(0)};
    double* sums = a.sums;
    grid_reduce<Acc, 3>(v3, 1, red, gridDim.x, blockIdx.x, sm, [&](int, Acc sv) { sums[0] = (double)sv; });
  }
}

// --------------------------------------------------------------------------
// march form
// --------------------------------------------------------------------------
template <class T, int VEC> struct VecOf;
template <> struct VecOf<float, 4> { typedef float4 type; };
template <> struct VecOf<double, 2> { typedef double2 type; };

template <class T, int VEC>
__device__ __forceinline__ void ld_vec(T (&r)[VEC], const T* p) {
  typedef typename VecOf<T, VEC>::type VT;
  const VT q = __ldg((const VT*)p);
  const T* e = (const T*)&q;
#pragma unroll
  for (int k = 0; k < VEC; ++k) r[k] = e[k];
}
__device__ __forceinline__ void ld_vec(float (&r)[4], const __nv_bfloat16* p) {
  const uint2 q = __ldg((const uint2*)p);
  const __nv_bfloat162* h = (const __nv_bfloat162*)&q;
  const float2 a = __bfloat1622float2(h[0]), b = __bfloat1622float2(h[1]);
  r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
}

// One row of one plane as a lane sees it: VEC centre values and, once the
// row is completed, the west neighbour of the first and the east neighbour
// of the last.
template <class T, int VEC>
struct Row {
  T c[VEC];
  T we, ee;
};

template <class T, int VEC, class TS>
__device__ __forceinline__ void row_load(Row<T, VEC>& r, const TS* plane, int rj, int nx, int col, bool act,
                                         int lane, int policy) {
  if (act) {
    ld_vec(r.c, plane + (long long)rj * nx + col);
  } else {
#pragma unroll
    for (int k = 0; k < VEC; ++k) r.c[k] = T(0);
  }
  // lanes at the ends of the strip fetch their outer neighbour themselves
  r.we = T(0);
  r.ee = T(0);
  if (act && lane == 0) r.we = (T)ldv1(plane, (long long)rj * nx + bp_index(col - 1, nx, policy));
  if (act && (lane == 31 || col + VEC >= nx))
    r.ee = (T)ldv1(plane, (long long)rj * nx + bp_index(col + VEC, nx, policy));
}

template <class T, int VEC>
__device__ __forceinline__ void row_complete(Row<T, VEC>& r, int lane, int col, int nx) {
  const T up = __shfl_up_sync(0xffffffffu, r.c[VEC - 1], 1);
  const T dn = __shfl_down_sync(0xffffffffu, r.c[0], 1);
  if (lane != 0) r.we = up;
  if (!(lane == 31 || col + VEC >= nx)) r.ee = dn;
}

template <class T, int VEC>
__device__ __forceinline__ T west_of(const Row<T, VEC>& r, int k) {
  return k > 0 ? r.c[k > 0 ? k - 1 : 0] : r.we;
}
template <class T, int VEC>
__device__ __forceinline__ T east_of(const Row<T, VEC>& r, int k) {
  return k < VEC - 1 ? r.c[k < VEC - 1 ? k + 1 : 0] : r.ee;
}

// Evaluate row j of a band. Slots S0, S1, S2 of the register ring hold rows
// j-1, j, j+1; row j+2 is prefetched into S3 before the arithmetic and
// completed (lane shuffles) after it, so its loads overlap the work on row
// j. The caller rotates the slot names instead of moving registers.
// EPI 0 writes every output through the generic per-cell epilogue; EPI 1 is
// the Krylov product out = J v (AD) or the FD quotient, with one 16-byte
// store per lane and field.
template <class PDE, class T, class TV, int VEC, int MODE, int EPI, int S0, int S1, int S2, int S3>
__device__ __forceinline__ void march_row(const ProbDev& P, const StencilArgs& a, const Comb<MODE, T>& cb, T eps,
                                          Row<T, VEC> (&xr)[PDE::NF][4], Row<T, VEC> (&vr)[PDE::NF][4], int j,
                                          int j1, int col, bool act, int lane, bool usev,
                                          typename AccOf<T>::type* acc) {
  typedef typename Comb<MODE, T>::V V;
  typedef typename AccOf<T>::type Acc;
  constexpr int NF = PDE::NF;
  constexpr int pol = PDE::POLICY;
  const int nx = P.nx, ny = P.ny;
  const T* __restrict__ x = (const T*)a.x;
  const TV* __restrict__ v = (const TV*)a.v;
  const bool pre = (j + 2 <= j1);
  if (pre) {
    const int rj = bp_index(j + 2, ny, pol);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      row_load(xr[f][S3], x + f * P.ncell, rj, nx, col, act, lane, pol);
      if (usev) row_load(vr[f][S3], v + f * P.ncell, rj, nx, col, act, lane, pol);
    }
  }
  const long long crow = (long long)j * nx;
  T jv[NF][VEC];
#pragma unroll
  for (int k = 0; k < VEC; ++k) {
    if (act) {
      const int i = col + k;
      Nb<V, NF> q;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const Row<T, VEC>& xs = xr[f][S0];
        const Row<T, VEC>& xc = xr[f][S1];
        const Row<T, VEC>& xn = xr[f][S2];
        const Row<T, VEC>& vs = vr[f][S0];
        const Row<T, VEC>& vc = vr[f][S1];
        const Row<T, VEC>& vn = vr[f][S2];
        q.c[f] = cb(xc.c[k], vc.c[k]);
        q.w[f] = cb(west_of(xc, k), west_of(vc, k));
        q.e[f] = cb(east_of(xc, k), east_of(vc, k));
        q.n[f] = cb(xn.c[k], vn.c[k]);
        q.s[f] = cb(xs.c[k], vs.c[k]);
        if (PDE::DIAG) {
          q.nw[f] = cb(west_of(xn, k), west_of(vn, k));
          q.ne[f] = cb(east_of(xn, k), east_of(vn, k));
          q.sw[f] = cb(west_of(xs, k), west_of(vs, k));
          q.se[f] = cb(east_of(xs, k), east_of(vs, k));
        }
      }
      const long long c = crow + i;
      const CellAux<T> aux = load_aux<PDE, T>(P, c);
      V M[NF], G[NF];
      PDE::template cell<T, V>(P, i, j, q, aux, M, G);
      if constexpr (EPI == 0) {
        emit<MODE, PDE, T, V, Acc>(P, a, c, M, G, q.c, eps, acc);
      } else {
        const T thdt = T(P.thdt);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if constexpr (MODE == SM_AD) {
            jv[f][k] = P.bvp ? G[f].d : M[f].d - thdt * G[f].d;
          } else {
            jv[f][k] = P.bvp ? primal(G[f]) : primal(M[f]) - thdt * primal(G[f]);   // F(x + eps v) without b
          }
        }
      }
    }
  }
  if constexpr (EPI == 1) {
    if (act) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const long long off = f * P.ncell + crow + col;
        T o[VEC];
        if constexpr (MODE == SM_FD) {
          T fx[VEC], bb[VEC];
          ld_vec(fx, (const T*)a.Fx + off);
          if (a.b) ld_vec(bb, (const T*)a.b + off);
#pragma unroll
          for (int k = 0; k < VEC; ++k) {
            T Fp = jv[f][k];
            if (a.b) Fp -= bb[k];
            o[k] = (Fp - fx[k]) / eps;
          }
        } else {
#pragma unroll
          for (int k = 0; k < VEC; ++k) o[k] = jv[f][k];
        }
        typedef typename VecOf<T, VEC>::type VT;
        *(VT*)((T*)a.out + off) = *(const VT*)o;
      }
    }
  }
  if (pre) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      row_complete(xr[f][S3], lane, col, nx);
      if (usev) row_complete(vr[f][S3], lane, col, nx);
    }
  }
}

template <class PDE, class T, class TV, int VEC, int MODE, int EPI>
__global__ void __launch_bounds__(256) k_march(ProbDev P, int nstrips, int R, StencilArgs a,
                                               RedSite<typename AccOf<T>::type> red) {
  typedef typename AccOf<T>::type Acc;
  typedef Comb<MODE, T> CB;
  constexpr int NF = PDE::NF;
  if (a.active && *a.active == 0) return;
  if (MODE == SM_RESID && a.ls && a.ls->done) return;
  const T s = (MODE == SM_AD || MODE == SM_FD) ? (a.vscale ? T(*a.vscale) : T(1)) : T(1);
  const T eps = fd_step<T, MODE>(a, s);
  const CB cb = make_comb<MODE, T>((MODE == SM_RESID && a.ls) ? a.ls->alpha : a.alpha, s, eps);
  const bool usev = (MODE != SM_RHS) && a.v != nullptr;
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int strip = (int)(gw % nstrips);
  const long long band = gw / nstrips;
  const int nx = P.nx, ny = P.ny;
  Acc acc[3] = {Acc(0), Acc(0), Acc(0)};
  if (band * R < ny) {
    const int j0 = (int)(band * R);
    const int j1 = j0 + R < ny ? j0 + R : ny;
    const int col = strip * 32 * VEC + lane * VEC;
    const bool act = col < nx;
    const T* __restrict__ x = (const T*)a.x;
    const TV* __restrict__ v = (const TV*)a.v;
    constexpr int pol = PDE::POLICY;
    Row<T, VEC> xr[NF][4], vr[NF][4];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (d < 3) {
          const int rj = bp_index(j0 + d - 1, ny, pol);
          row_load(xr[f][d], x + f * P.ncell, rj, nx, col, act, lane, pol);
          row_complete(xr[f][d], lane, col, nx);
        }
        if (d < 3 && usev) {
          const int rj = bp_index(j0 + d - 1, ny, pol);
          row_load(vr[f][d], v + f * P.ncell, rj, nx, col, act, lane, pol);
          row_complete(vr[f][d], lane, col, nx);
        } else {
#pragma unroll
          for (int k = 0; k < VEC; ++k) vr[f][d].c[k] = T(0);
          vr[f][d].we = T(0);
          vr[f][d].ee = T(0);
        }
      }
    }
    for (int j = j0;;) {
      if (j >= j1) break;
      march_row<PDE, T, TV, VEC, MODE, EPI, 0, 1, 2, 3>(P, a, cb, eps, xr, vr, j, j1, col, act, lane, usev, acc);
      if (++j >= j1) break;
      march_row<PDE, T, TV, VEC, MODE, EPI, 1, 2, 3, 0>(P, a, cb, eps, xr, vr, j, j1, col, act, lane, usev, acc);
      if (++j >= j1) break;
      march_row<PDE, T, TV, VEC, MODE, EPI, 2, 3, 0, 1>(P, a, cb, eps, xr, vr, j, j1, col, act, lane, usev, acc);
      if (++j >= j1) break;
      march_row<PDE, T, TV, VEC, MODE, EPI, 3, 0, 1, 2>(P, a, cb, eps, xr, vr, j, j1, col, act, lane, usev, acc);
      ++j;
    }
  }
  if constexpr (EPI == 0) finish_reduction<MODE, Acc>(a, acc, gridDim.x, blockIdx.x, red);
}

}  // namespace jfnk

#include "stencil_stage.cuh"

namespace jfnk {

// --------------------------------------------------------------------------
// geometry and launch
// --------------------------------------------------------------------------
inline int num_sms() {
  static int g_nsm = 0;
  if (g_nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g_nsm <= 0) {
      cudaGetLastError();
      g_nsm = 152;
    }
  }
  return g_nsm;
}

struct MarchGeom {
  int nstrips, R, nbands, nblocks;
};

inline MarchGeom march_geom(const ProbDev& P, int vec) {
  MarchGeom g;
  g.nstrips = (P.nx + 32 * vec - 1) / (32 * vec);
  const long long target_warps = (long long)num_sms() * 24;
  long long nb = (target_warps + g.nstrips - 1) / g.nstrips;
  const long long maxb = (P.ny + 3) / 4;          // at least 4 rows per band
  if (nb > maxb) nb = maxb;
  if (nb < 1) nb = 1;
  g.R = (int)((P.ny + nb - 1) / nb);
  g.nbands = (P.ny + g.R - 1) / g.R;
  const long long warps = (long long)g.nstrips * g.nbands;
  g.nblocks = (int)((warps + 7) / 8);
  return g;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

template <class T, class TV>
static bool march_ok(const ProbDev& P, const StencilArgs& a) {
  if (P.nf > 2) return false;   // four planes: the register rows would spill; the gather form serves them
  if (a.precond) return false;  // the preconditioned direction is formed per node in the gather form
  const int vec = 16 / (int)sizeof(T);
  if (P.nx % vec != 0) return false;
  if (!aligned(a.x, 16)) return false;
  if (a.v && !aligned(a.v, vec * sizeof(TV))) return false;
  const void* e = sizeof(T) == 8 ? (const void*)P.eps64 : (const void*)P.eps32;
  const void* f = sizeof(T) == 8 ? (const void*)P.src64 : (const void*)P.src32;
  return aligned(e, 16) && aligned(f, 16);
}

template <class PDE, class T, class TV, int MODE>
static cudaError_t stencil_launch(const ProbDev& P, const StencilArgs& a, RedWs red, cudaStream_t st) {
  typedef typename AccOf<T>::type Acc;
  RedSite<Acc> rs{(Acc*)red.partials, red.counter, red.max_blocks};
  if constexpr (MODE == SM_PREC) {
    if (!PDE::PRECOND) return cudaErrorInvalidValue;
    k_precond<PDE, T><<<vec_blocks(P.ncell), 256, 0, st>>>(P, a, rs);
  } else {
    if (march_ok<T, TV>(P, a)) {
      constexpr int VEC = 16 / (int)sizeof(T);
      const MarchGeom g = march_geom(P, VEC);
      if constexpr (MODE == SM_AD || MODE == SM_FD) {
        // the plain Krylov product (no F, no addend, no reduction, unit factor) has a vector epilogue
        const bool plain = !a.F && !a.add && a.ndots == 0 && a.c_jv == 1.0 && aligned(a.out, 16) &&
                           (MODE != SM_FD || (aligned(a.Fx, 16) && aligned(a.b, 16)));
        if (plain) {
          // large 2D grids: rows staged in shared memory by bulk copies (stencil_stage.cuh)
          StagePlan sp;
          if (a.err && P.nx >= kStageWarps * 32 * VEC && P.ny >= 64 && aligned(a.v, 16) &&
              stage_plan<T, TV, PDE::NF>(P, num_sms(), &sp)) {
            // opt in once at the per-block limit, so that every later plan (another grid) fits
            static SmemLimit limit_of;
            static SmemOptIn opt_in;
            int limit = 0;
            cudaError_t e = smem_block_limit(k_jvp_stage<PDE, T, TV, MODE>, limit_of, &limit);
            if (e != cudaSuccess) return e;
            if (sp.smem > limit) return cudaErrorInvalidValue;
            e = smem_opt_in(k_jvp_stage<PDE, T, TV, MODE>, opt_in, limit);
            if (e != cudaSuccess) return e;
            e = launch_maybe_pdl(a.pdl != 0, k_jvp_stage<PDE, T, TV, MODE>, dim3(sp.grid), dim3(kStageThreads),
                                 (size_t)sp.smem, st, P, a, sp);
            if (e != cudaSuccess) return e;
            return cudaGetLastError();
          }
          k_march<PDE, T, TV, VEC, MODE, 1><<<g.nblocks, 256, 0, st>>>(P, g.nstrips, g.R, a, rs);
          return cudaGetLastError();
        }
      }
      k_march<PDE, T, TV, VEC, MODE, 0><<<g.nblocks, 256, 0, st>>>(P, g.nstrips, g.R, a, rs);
    } else {
      const StencilGeom g = stencil_geom(P);
      k_gather<PDE, T, TV, MODE><<<g.grid, g.block, 0, st>>>(P, g.rows_per_thread, a, rs);
    }
  }
  return cudaGetLastError();
}

template <class PDE, int MODE>
static cudaError_t stencil_types(const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red, cudaStream_t st) {
  if (t == VT_F64) {
    if (tv != VT_F64) return cudaErrorInvalidValue;
    return stencil_launch<PDE, double, double, MODE>(P, a, red, st);
  }
  if (tv == VT_F32) return stencil_launch<PDE, float, float, MODE>(P, a, red, st);
  if constexpr (MODE == SM_AD || MODE == SM_FD) {
    if (tv == VT_BF16) return stencil_launch<PDE, float, __nv_bfloat16, MODE>(P, a, red, st);
  }
  return cudaErrorInvalidValue;
}

// All launch forms and precisions of one PDE for one mode (instantiated in
// the per-PDE translation units stencil_<pde>.cu).
template <class PDE>
cudaError_t stencil_dispatch(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                             cudaStream_t st) {
  switch (mode) {
    case SM_RESID: return stencil_types<PDE, SM_RESID>(P, t, tv, a, red, st);
    case SM_RHS: return stencil_types<PDE, SM_RHS>(P, t, tv, a, red, st);
    case SM_AD: return stencil_types<PDE, SM_AD>(P, t, tv, a, red, st);
    case SM_FD: return stencil_types<PDE, SM_FD>(P, t, tv, a, red, st);
    case SM_PREC: return stencil_types<PDE, SM_PREC>(P, t, tv, a, red, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t stencil_burgers(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red, cudaStream_t st);
cudaError_t stencil_allen_cahn(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                               cudaStream_t st);
cudaError_t stencil_su_olson(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                             cudaStream_t st);
cudaError_t stencil_maxwell(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                            cudaStream_t st);
cudaError_t stencil_burgers2d(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                              cudaStream_t st);
cudaError_t stencil_maxwell_vec(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                                cudaStream_t st);

}  // namespace jfnk
