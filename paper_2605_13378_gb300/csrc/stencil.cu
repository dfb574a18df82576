// stencil.cu -- residual, right-hand-side and Jacobian-vector-product sweeps.
//
// One thread evaluates one cell per row it owns; a block covers a tile of
// blockDim.x columns by R * blockDim.y rows, thread (tx, ty) taking rows
// ty, ty + blockDim.y, ... so that the rows above and below a cell are read
// by neighbouring threads of the same block at the same time (L1 reuse) and
// every input is streamed from HBM once. The same per-cell residual source
// (pdes.cuh) is instantiated on plain numbers for F(x) and the FD quotient
// (Eq. 7), and on dual numbers for the AD product (F(x), J(x) v) (Eq. 9).
#include "kernels.h"
#include "ctl.cuh"

namespace jfnk {

StencilGeom stencil_geom(const ProbDev& P) {
  StencilGeom g;
  if (P.ny == 1) {
    g.block = dim3(256, 1, 1);
  } else {
    g.block = dim3(32, 8, 1);
  }
  const long long gx = (P.nx + g.block.x - 1) / g.block.x;
  const long long rows = (P.ny + g.block.y - 1) / g.block.y;   // row groups
  // at most ~8 blocks per SM on 152 SMs: fold row groups into R per thread
  long long R = (gx * rows + 1215) / 1216;
  if (R < 1) R = 1;
  const long long gy = (rows + R - 1) / R;
  g.grid = dim3((unsigned)gx, (unsigned)gy, 1);
  g.rows_per_thread = (int)R;
  g.nblocks = (int)(gx * gy);
  return g;
}

// ---------------------------------------------------------------------------
// Loaders: flat index -> value of the state at which the residual is taken.
// ---------------------------------------------------------------------------
template <class T>
struct LoadPlain {            // x + alpha d
  const T* __restrict__ x; const T* __restrict__ d; T alpha;
  __device__ __forceinline__ T operator()(long long i) const {
    T v = __ldg(x + i);
    if (d) v += alpha * __ldg(d + i);
    return v;
  }
};
__device__ __forceinline__ float ldv(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ldv(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ double ldv(const double* p, long long i) { return __ldg(p + i); }

template <class T, class TV>
struct LoadAD {               // dual (x, s v)
  const T* __restrict__ x; const TV* __restrict__ v; T s;
  __device__ __forceinline__ Dual<T> operator()(long long i) const {
    return Dual<T>(__ldg(x + i), s * (T)ldv(v, i));
  }
};
template <class T, class TV>
struct LoadFD {               // x + (eps s) v
  const T* __restrict__ x; const TV* __restrict__ v; T es;
  __device__ __forceinline__ T operator()(long long i) const {
    return __ldg(x + i) + es * (T)ldv(v, i);
  }
};

template <class T> struct AccOf { typedef float type; };
template <> struct AccOf<double> { typedef double type; };

template <class T> __device__ __forceinline__ T eps_mach();
template <> __device__ __forceinline__ double eps_mach<double>() { return 2.220446049250313e-16; }
template <> __device__ __forceinline__ float eps_mach<float>() { return 1.1920928955078125e-07f; }

#define JFNK_CELL_LOOP_BEGIN                                                        \
  const int i = blockIdx.x * blockDim.x + threadIdx.x;                              \
  const int jbase = blockIdx.y * R * blockDim.y + threadIdx.y;                      \
  for (int r = 0; r < R; ++r) {                                                     \
    const int j = jbase + r * blockDim.y;                                           \
    if (i < P.nx && j < P.ny) {
#define JFNK_CELL_LOOP_END \
    }                      \
  }

// ---------------------------------------------------------------------------
// F = M(x + a d) - theta dt G(x + a d) - b (or G for the boundary-value
// problem), optional copies of x + a d in T and FP32, and ||F||^2, ||x+ad||^2.
// ---------------------------------------------------------------------------
template <class PDE, class T>
__global__ void __launch_bounds__(256) k_residual(ProbDev P, int R, const T* __restrict__ x, const T* __restrict__ d,
                                                  T alpha, const T* __restrict__ b, T* __restrict__ F,
                                                  T* __restrict__ xout, float* __restrict__ x32,
                                                  RedSite<double> red, double* sums) {
  constexpr int NF = PDE::NF;
  LoadPlain<T> ld{x, d, alpha};
  double acc[2] = {0.0, 0.0};
  const T thdt = T(P.thdt);
  JFNK_CELL_LOOP_BEGIN
    T M[NF], G[NF];
    PDE::template cell<T, T>(P, ld, i, j, M, G);
    const long long c = (long long)j * P.nx + i;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long id = f * P.ncell + c;
      T Fv = P.bvp ? G[f] : (M[f] - thdt * G[f]);
      if (b) Fv -= b[id];
      if (F) F[id] = Fv;
      const T xv = ld(id);
      if (xout) xout[id] = xv;
      if (x32) x32[id] = (float)xv;
      acc[0] += (double)Fv * (double)Fv;
      acc[1] += (double)xv * (double)xv;
    }
  JFNK_CELL_LOOP_END
  if (sums) {
    __shared__ double sm[8 * 2];
    grid_reduce<double, 2>(acc, 2, red, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x, sm,
                           [&](int t, double s) { sums[t] = s; });
  }
}

// b = M(xn) + (1 - theta) dt G(xn)
template <class PDE, class T>
__global__ void __launch_bounds__(256) k_rhs(ProbDev P, int R, const T* __restrict__ xn, T* __restrict__ b) {
  constexpr int NF = PDE::NF;
  LoadPlain<T> ld{xn, nullptr, T(0)};
  const T cold = T(P.c_old);
  JFNK_CELL_LOOP_BEGIN
    T M[NF], G[NF];
    PDE::template cell<T, T>(P, ld, i, j, M, G);
    const long long c = (long long)j * P.nx + i;
#pragma unroll
    for (int f = 0; f < NF; ++f) b[f * P.ncell + c] = M[f] + cold * G[f];
  JFNK_CELL_LOOP_END
}

// ---------------------------------------------------------------------------
// Jacobian-vector product: AD (one dual sweep) or FD (one perturbed sweep).
// ---------------------------------------------------------------------------
struct JvpDev {
  const void* x; const void* v; const double* vscale;
  const void* b; void* F; const void* Fx;
  void* out; double c_jv; const void* add; double c_add;
  int ndots; const void* dw[3]; double* sums;
  int post; void* post_arg;
  double eps_fixed; int eps_rule; const double* xn2; const double* vn2;
  float* eps_out;
  const int* active;
};

template <class PDE, class T, class TV, int LIN>
__global__ void __launch_bounds__(256) k_jvp(ProbDev P, int R, JvpDev a, RedSite<typename AccOf<T>::type> red) {
  typedef typename AccOf<T>::type Acc;
  constexpr int NF = PDE::NF;
  if (a.active && *a.active == 0) return;
  const T* __restrict__ x = (const T*)a.x;
  const TV* __restrict__ v = (const TV*)a.v;
  const T* __restrict__ b = (const T*)a.b;
  T* __restrict__ out = (T*)a.out;
  const T* __restrict__ add = (const T*)a.add;
  const T s = a.vscale ? T(*a.vscale) : T(1);
  const T thdt = T(P.thdt);
  const T cjv = T(a.c_jv), cadd = T(a.c_add);
  Acc acc[3] = {Acc(0), Acc(0), Acc(0)};
  __shared__ T s_eps;
  if (LIN == 1) {
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
          const double vn = a.vn2 ? sqrt(*a.vn2) * (double)s : 1.0;
          eps = sq * (1.0 + xn) / vn;
        }
      }
      s_eps = T(eps);
      if (a.eps_out && blockIdx.x == 0 && blockIdx.y == 0) *a.eps_out = (float)eps;
    }
    __syncthreads();
  }
  JFNK_CELL_LOOP_BEGIN
    const long long c = (long long)j * P.nx + i;
    T jv[NF];
    if (LIN == 0) {
      LoadAD<T, TV> ld{x, v, s};
      Dual<T> M[NF], G[NF];
      PDE::template cell<T, Dual<T> >(P, ld, i, j, M, G);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Dual<T> Fd = P.bvp ? G[f] : (M[f] - thdt * G[f]);
        jv[f] = Fd.d;
        if (a.F) ((T*)a.F)[f * P.ncell + c] = b ? Fd.v - b[f * P.ncell + c] : Fd.v;
      }
    } else {
      const T eps = s_eps;
      LoadFD<T, TV> ld{x, v, eps * s};
      T M[NF], G[NF];
      PDE::template cell<T, T>(P, ld, i, j, M, G);
      const T* __restrict__ Fx = (const T*)a.Fx;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const long long id = f * P.ncell + c;
        T Fp = P.bvp ? G[f] : (M[f] - thdt * G[f]);
        if (b) Fp -= b[id];
        jv[f] = (Fp - Fx[id]) / eps;
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const long long id = f * P.ncell + c;
      T o = cjv * jv[f];
      if (add) o += cadd * add[id];
      out[id] = o;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (k < a.ndots) {
          const T w = a.dw[k] ? ((const T*)a.dw[k])[id] : o;
          acc[k] += (Acc)o * (Acc)w;
        }
      }
    }
  JFNK_CELL_LOOP_END
  if (a.ndots > 0) {
    __shared__ Acc sm[8 * 3];
    double* sums = a.sums;
    const int post = a.post;
    void* parg = a.post_arg;
    const bool last = grid_reduce<Acc, 3>(acc, a.ndots, red, gridDim.x * gridDim.y,
                                          blockIdx.y * gridDim.x + blockIdx.x, sm,
                                          [&](int t, Acc sv) { sums[t] = (double)sv; });
    if (last && threadIdx.x == 0 && threadIdx.y == 0 && post == POST_GMRES_RESTART)
      gmres_cycle_start((GmresCtl*)parg, sums[0]);
  }
}

// ---------------------------------------------------------------------------
// Host launchers: dispatch on PDE and precision.
// ---------------------------------------------------------------------------
template <class PDE>
static cudaError_t residual_pde(const ProbDev& P, int t, const void* x, const void* d, double alpha,
                                const void* b, void* F, void* xout, float* x32, RedWs red, double* sums,
                                cudaStream_t st) {
  const StencilGeom g = stencil_geom(P);
  if (t == VT_F64) {
    RedSite<double> rs{(double*)red.partials, red.counter};
    k_residual<PDE, double><<<g.grid, g.block, 0, st>>>(P, g.rows_per_thread, (const double*)x, (const double*)d,
                                                        alpha, (const double*)b, (double*)F, (double*)xout, x32,
                                                        rs, sums);
  } else {
    RedSite<double> rs{(double*)red.partials, red.counter};
    k_residual<PDE, float><<<g.grid, g.block, 0, st>>>(P, g.rows_per_thread, (const float*)x, (const float*)d,
                                                       (float)alpha, (const float*)b, (float*)F, (float*)xout, x32,
                                                       rs, sums);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual(const ProbDev& P, int t, const void* x, const void* d, double alpha, const void* b,
                            void* F, void* xout, float* x32, RedWs red, double* sums, cudaStream_t st) {
  switch (P.pde) {
    case 0: return residual_pde<Burgers1D>(P, t, x, d, alpha, b, F, xout, x32, red, sums, st);
    case 1: return residual_pde<AllenCahn2D>(P, t, x, d, alpha, b, F, xout, x32, red, sums, st);
    case 2: return residual_pde<SuOlson2D>(P, t, x, d, alpha, b, F, xout, x32, red, sums, st);
    case 3: return residual_pde<MaxwellTE2D>(P, t, x, d, alpha, b, F, xout, x32, red, sums, st);
  }
  return cudaErrorInvalidValue;
}

template <class PDE>
static cudaError_t rhs_pde(const ProbDev& P, int t, const void* xn, void* b, cudaStream_t st) {
  const StencilGeom g = stencil_geom(P);
  if (t == VT_F64)
    k_rhs<PDE, double><<<g.grid, g.block, 0, st>>>(P, g.rows_per_thread, (const double*)xn, (double*)b);
  else
    k_rhs<PDE, float><<<g.grid, g.block, 0, st>>>(P, g.rows_per_thread, (const float*)xn, (float*)b);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const ProbDev& P, int t, const void* xn, void* b, cudaStream_t st) {
  switch (P.pde) {
    case 0: return rhs_pde<Burgers1D>(P, t, xn, b, st);
    case 1: return rhs_pde<AllenCahn2D>(P, t, xn, b, st);
    case 2: return rhs_pde<SuOlson2D>(P, t, xn, b, st);
    case 3: return rhs_pde<MaxwellTE2D>(P, t, xn, b, st);
  }
  return cudaErrorInvalidValue;
}

template <class PDE, class T, class TV>
static void jvp_lin(const ProbDev& P, const StencilGeom& g, int lin, const JvpDev& a,
                    RedSite<typename AccOf<T>::type> rs, cudaStream_t st) {
  if (lin == 0)
    k_jvp<PDE, T, TV, 0><<<g.grid, g.block, 0, st>>>(P, g.rows_per_thread, a, rs);
  else
    k_jvp<PDE, T, TV, 1><<<g.grid, g.block, 0, st>>>(P, g.rows_per_thread, a, rs);
}

template <class PDE>
static cudaError_t jvp_pde(const ProbDev& P, const JvpArgs& in, RedWs red, cudaStream_t st) {
  const StencilGeom g = stencil_geom(P);
  JvpDev a;
  a.x = in.x; a.v = in.v; a.vscale = in.vscale; a.b = in.b; a.F = in.F; a.Fx = in.Fx;
  a.out = in.out; a.c_jv = in.c_jv; a.add = in.add; a.c_add = in.c_add;
  a.ndots = in.ndots; a.dw[0] = in.dw[0]; a.dw[1] = in.dw[1]; a.dw[2] = in.dw[2]; a.sums = in.sums;
  a.post = in.post; a.post_arg = in.post_arg;
  a.eps_fixed = in.eps_fixed; a.eps_rule = in.eps_rule; a.xn2 = in.xn2; a.vn2 = in.vn2; a.eps_out = in.eps_out;
  a.active = in.active;
  if (in.t == VT_F64) {
    if (in.tv != VT_F64) return cudaErrorInvalidValue;
    jvp_lin<PDE, double, double>(P, g, in.lin, a, RedSite<double>{(double*)red.partials, red.counter}, st);
  } else {
    RedSite<float> rs{(float*)red.partials, red.counter};
    if (in.tv == VT_F32)
      jvp_lin<PDE, float, float>(P, g, in.lin, a, rs, st);
    else if (in.tv == VT_BF16)
      jvp_lin<PDE, float, __nv_bfloat16>(P, g, in.lin, a, rs, st);
    else
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_jvp(const ProbDev& P, const JvpArgs& a, RedWs red, cudaStream_t st) {
  switch (P.pde) {
    case 0: return jvp_pde<Burgers1D>(P, a, red, st);
    case 1: return jvp_pde<AllenCahn2D>(P, a, red, st);
    case 2: return jvp_pde<SuOlson2D>(P, a, red, st);
    case 3: return jvp_pde<MaxwellTE2D>(P, a, red, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace jfnk
