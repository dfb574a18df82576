// krylov.cu -- flat-vector kernels of the Krylov solvers.
//
// Restarted GMRES(m) (Sec. 2; Saad and Schultz) with classical Gram-Schmidt
// applied twice, as three fused passes over the basis per Arnoldi step:
//   pass 1  h1 = V^T w                         (dots)
//   pass 2  w <- w - V h1,   h2 = V^T w        (update + dots)
//   pass 3  u <- w - V h2,   ||u||^2, Givens   (update + norm + rotation)
// The basis is stored unnormalised (v_t = scale[t] u_t), which removes the
// normalisation sweep; the scale is folded into the coefficients. Every
// reduction accumulates in the Krylov precision inside a thread and follows a
// fixed tree over a grid that depends only on the vector length, so results
// are reproducible run to run and independent of what else is on the GPU.
// BiCGSTAB (van der Vorst) and CG (Hestenes-Stiefel) scalar updates follow
// the textbook recurrences with device-side breakdown tests.
#include "kernels.h"
#include "krylov.h"
#include "ctl.cuh"

namespace jfnk {

template <class T> struct AccK { typedef float type; };
template <> struct AccK<double> { typedef double type; };

__device__ __forceinline__ float ldb(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ldb(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ double ldb(const double* p, long long i) { return __ldg(p + i); }
// basis loads inside a kernel that also writes the basis (no read-only path)
__device__ __forceinline__ float ldbw(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ldbw(const float* p, long long i) { return p[i]; }
__device__ __forceinline__ double ldbw(const double* p, long long i) { return p[i]; }

#define VEC_LOOP(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
                            i += (long long)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// Start of a GMRES solve of J d = -F: u_0 = -F (basis precision), the
// Krylov right-hand side rhs = -F (JVP precision), d = 0, and the control
// block (beta = ||F||, target = tol ||F||) from sums[0] = ||F||^2.
// ---------------------------------------------------------------------------
template <class TS, class TJ, class TB, class TD>
__global__ void k_gmres_init(long long n, const TS* __restrict__ F, TB* __restrict__ u0, TJ* __restrict__ rhs,
                             TD* __restrict__ d, GmresCtl* ctl, const double* sums, double tol, int m) {
  VEC_LOOP(i, n) {
    const TS f = F[i];
    u0[i] = store_as<TB>::cvt(-f);
    rhs[i] = (TJ)(-f);
    d[i] = TD(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double f2 = sums[0];
    ctl->m = m;
    ctl->its = 0;
    ctl->converged = 0;
    ctl->breakdown = 0;
    ctl->nonfinite = 0;
    ctl->bnorm = sqrt(f2);
    ctl->target = tol * ctl->bnorm;
    gmres_cycle_start(ctl, f2);
  }
}

// pass 1: h1[t] = scale[t] * sum_i u_t[i] w[i], t < k
template <class TB, class TJ, int KMAX>
__global__ void __launch_bounds__(256) k_arnoldi_dots(long long n, const TB* __restrict__ V, long long ldv, int k,
                                                      const TJ* __restrict__ w, GmresCtl* ctl,
                                                      RedSite<typename AccK<TJ>::type> red) {
  typedef typename AccK<TJ>::type A;
  if (!ctl->active) return;
  A acc[KMAX];
#pragma unroll
  for (int t = 0; t < KMAX; ++t) acc[t] = A(0);
  VEC_LOOP(i, n) {
    const A wi = (A)__ldg(w + i);
#pragma unroll
    for (int t = 0; t < KMAX; ++t)
      if (t < k) acc[t] += (A)ldb(V, t * ldv + i) * wi;
  }
  __shared__ A sm[8 * KMAX];
  grid_reduce<A, KMAX>(acc, k, red, gridDim.x, blockIdx.x, sm,
                       [&](int t, A s) { ctl->h1[t] = (double)s * ctl->scale[t]; });
}

// pass 2: w <- w - sum_t h1[t] v_t;  h2[t] = v_t . w
template <class TB, class TJ, int KMAX>
__global__ void __launch_bounds__(256) k_arnoldi_update_dots(long long n, const TB* __restrict__ V, long long ldv,
                                                             int k, TJ* __restrict__ w, GmresCtl* ctl,
                                                             RedSite<typename AccK<TJ>::type> red) {
  typedef typename AccK<TJ>::type A;
  if (!ctl->active) return;
  __shared__ A coef[KMAX];
  for (int t = threadIdx.x; t < k; t += blockDim.x) coef[t] = (A)(ctl->h1[t] * ctl->scale[t]);
  __syncthreads();
  A acc[KMAX];
#pragma unroll
  for (int t = 0; t < KMAX; ++t) acc[t] = A(0);
  VEC_LOOP(i, n) {
    A ub[KMAX];
    A wi = (A)w[i];
#pragma unroll
    for (int t = 0; t < KMAX; ++t)
      if (t < k) { ub[t] = (A)ldb(V, t * ldv + i); wi -= coef[t] * ub[t]; }
    w[i] = (TJ)wi;
    const A wr = (A)(TJ)wi;
#pragma unroll
    for (int t = 0; t < KMAX; ++t)
      if (t < k) acc[t] += ub[t] * wr;
  }
  __shared__ A sm[8 * KMAX];
  grid_reduce<A, KMAX>(acc, k, red, gridDim.x, blockIdx.x, sm,
                       [&](int t, A s) { ctl->h2[t] = (double)s * ctl->scale[t]; });
}

// pass 3: u_{j+1} = w - sum_t h2[t] v_t (stored in the basis precision),
// ||u_{j+1}||^2 of the stored values, then the Givens step on the last block.
template <class TB, class TJ, int KMAX>
__global__ void __launch_bounds__(256) k_arnoldi_update_norm(long long n, TB* __restrict__ V, long long ldv, int k,
                                                             const TJ* __restrict__ w, GmresCtl* ctl,
                                                             RedSite<typename AccK<TJ>::type> red) {
  typedef typename AccK<TJ>::type A;
  if (!ctl->active) return;
  __shared__ A coef[KMAX];
  for (int t = threadIdx.x; t < k; t += blockDim.x) coef[t] = (A)(ctl->h2[t] * ctl->scale[t]);
  __syncthreads();
  A acc[1] = {A(0)};
  TB* __restrict__ unew = V + (long long)k * ldv;
  VEC_LOOP(i, n) {
    A wi = (A)__ldg(w + i);
#pragma unroll
    for (int t = 0; t < KMAX; ++t)
      if (t < k) wi -= coef[t] * (A)ldbw(V, t * ldv + i);
    const TB st = store_as<TB>::cvt(wi);
    unew[i] = st;
    const A sv = (A)to_f(st);
    acc[0] += sv * sv;
  }
  __shared__ A sm[8];
  __shared__ double s_n2;
  const bool last = grid_reduce<A, 1>(acc, 1, red, gridDim.x, blockIdx.x, sm, [&](int, A s) { s_n2 = (double)s; });
  if (last && threadIdx.x == 0) gmres_givens_step(ctl, k - 1, s_n2);
}

bool stream_supported(long long n) { return n % 8 == 0 && n >= 8; }

cudaError_t launch_basis_stream(int mode, int tb, int tj, int td, long long n, const void* V, int k, int kmax,
                                void* w, void* d, GmresCtl* ctl, RedWs red, unsigned int* err, int nsm,
                                cudaStream_t st) {
  if (!stream_supported(n) || k > kMaxM || kmax > kMaxM) return cudaErrorInvalidValue;
  if (tb == VT_F64 && tj == VT_F64 && td == VT_F64)
    return basis_stream_f64(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  if (tb == VT_F32 && tj == VT_F32 && (td == VT_F32 || td == VT_F64))
    return basis_stream_f32(mode, td, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  if (tb == VT_BF16 && tj == VT_F32 && td == VT_F64)
    return basis_stream_bf16(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_dcgs(int pass, int tb, int tj, long long n, void* V, int j, const void* w, GmresCtl* ctl,
                        RedWs red, unsigned int* err, int nsm, cudaStream_t st, bool pdl, bool defer) {
  if (!stream_supported(n) || j < 0 || j > kMaxM || (pass != 1 && pass != 2)) return cudaErrorInvalidValue;
  if (tb == VT_F64 && tj == VT_F64) return dcgs_f64(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  if (tb == VT_F32 && tj == VT_F32) return dcgs_f32(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  if (tb == VT_BF16 && tj == VT_F32) return dcgs_bf16(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  return cudaErrorInvalidValue;
}

// back substitution H[:k,:k] y = g[:k] by one warp, column oriented
__global__ void k_gmres_backsolve(GmresCtl* ctl) {
  const int k = ctl->k;
  const int lane = threadIdx.x;
  __shared__ double y[kMaxM];
  for (int t = lane; t < k; t += 32) y[t] = ctl->g[t];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    const double* col = ctl->H + (size_t)i * (kMaxM + 1);
    double yi = 0.0;
    if (lane == 0) y[i] = y[i] / col[i];
    __syncwarp();
    yi = y[i];
    for (int t = lane; t < i; t += 32) y[t] -= col[t] * yi;
    __syncwarp();
  }
  for (int t = lane; t < k; t += 32) ctl->y[t] = y[t] * ctl->scale[t];
}

// d += sum_{t<k} y_t v_t (y already multiplied by scale)
template <class TB, class TD, int KMAX>
__global__ void __launch_bounds__(256) k_gmres_update(long long n, const TB* __restrict__ V, long long ldv,
                                                      TD* __restrict__ d, const GmresCtl* ctl) {
  typedef typename AccK<TD>::type A;
  const int k = ctl->k;
  if (k == 0) return;
  __shared__ A coef[KMAX];
  for (int t = threadIdx.x; t < KMAX; t += blockDim.x) coef[t] = t < k ? (A)ctl->y[t] : A(0);
  __syncthreads();
  VEC_LOOP(i, n) {
    A s = A(0);
#pragma unroll
    for (int t = 0; t < KMAX; ++t)
      if (t < k) s += coef[t] * (A)ldb(V, t * ldv + i);
    d[i] = d[i] + (TD)s;
  }
}

// y = (TO) (c x)
template <class TI, class TO>
__global__ void k_cast(long long n, const TI* __restrict__ x, TO* __restrict__ y, double c) {
  VEC_LOOP(i, n) y[i] = store_as<TO>::cvt((typename AccK<TI>::type)c * (typename AccK<TI>::type)to_d(x[i]));
}

// sums[q] = a_q . b_q for q < nd (b_q null: a_q . a_q), reduced in Acc.
template <class T>
__global__ void __launch_bounds__(256) k_vdots(long long n, int nd, const T* a0, const T* b0, const T* a1,
                                               const T* b1, const T* a2, const T* b2, double* sums,
                                               RedSite<typename AccK<T>::type> red, const int* active) {
  typedef typename AccK<T>::type A;
  if (active && *active == 0) return;
  A acc[3] = {A(0), A(0), A(0)};
  const T* as[3] = {a0, a1, a2};
  const T* bs[3] = {b0, b1, b2};
  VEC_LOOP(i, n) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q < nd) {
        const A x = (A)as[q][i];
        const A y = bs[q] ? (A)bs[q][i] : x;
        acc[q] += x * y;
      }
    }
  }
  __shared__ A sm[8 * 3];
  grid_reduce<A, 3>(acc, nd, red, gridDim.x, blockIdx.x, sm, [&](int q, A s) { sums[q] = (double)s; });
}

// ---------------------------------------------------------------------------
// BiCGSTAB phases (r_hat = r_0 = b, x_0 = 0). Scalars live in BicgCtl;
// every phase first checks `active`.
// ---------------------------------------------------------------------------
// init: r = rhat = b = -F (TJ), p = v = 0, x = 0; rho_old = alpha = omega = 1
template <class TS, class TJ, class TD>
__global__ void k_bicg_init(long long n, const TS* __restrict__ F, TJ* r, TJ* rhat, TJ* p, TJ* v, TD* d,
                            BicgCtl* c, const double* sums, double tol) {
  VEC_LOOP(i, n) {
    const TJ b = (TJ)(-F[i]);
    r[i] = b; rhat[i] = b; p[i] = TJ(0); v[i] = TJ(0); d[i] = TD(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double bn = sqrt(sums[0]);
    c->bnorm = bn;
    c->target = tol * bn;
    c->rho_old = 1.0; c->alpha = 1.0; c->omega = 1.0;
    c->rho = sums[0];          // rhat . r = ||b||^2 for the first iteration
    c->its = 0; c->converged = 0; c->breakdown = 0; c->nonfinite = 0; c->flag_half = 0;
    c->resid = bn;
    c->active = (bn > 0.0 && isfinite(bn)) ? 1 : 0;
    if (bn == 0.0) c->converged = 1;
    if (!isfinite(bn)) c->nonfinite = 1;
    mirror_active(c->host_active, c->active);
  }
}

// p = r + beta (p - omega v), beta = (rho / rho_old)(alpha / omega); ||p||^2 for FD
template <class TJ>
__global__ void __launch_bounds__(256) k_bicg_p(long long n, const TJ* __restrict__ r, TJ* __restrict__ p,
                                                const TJ* __restrict__ v, BicgCtl* c, double* pn2,
                                                RedSite<typename AccK<TJ>::type> red) {
  typedef typename AccK<TJ>::type A;
  if (!c->active) return;
  const double rho = c->rho;
  const A beta = (A)((rho / c->rho_old) * (c->alpha / c->omega));
  const A om = (A)c->omega;
  A acc[1] = {A(0)};
  VEC_LOOP(i, n) {
    const A pi = (A)r[i] + beta * ((A)p[i] - om * (A)v[i]);
    p[i] = (TJ)pi;
    acc[0] += pi * pi;
  }
  if (pn2) {
    __shared__ A sm[8];
    grid_reduce<A, 1>(acc, 1, red, gridDim.x, blockIdx.x, sm, [&](int, A s) { *pn2 = (double)s; });
  }
}

// after v = J p and sums[0] = rhat . v: alpha = rho / (rhat . v); s = r - alpha v, ||s||^2;
// converged on ||s|| <= target (then x += alpha p)
template <class TJ, class TD>
__global__ void __launch_bounds__(256) k_bicg_s(long long n, const TJ* __restrict__ r, const TJ* __restrict__ v,
                                                TJ* __restrict__ s, BicgCtl* c, double* sn2,
                                                RedSite<typename AccK<TJ>::type> red, int it) {
  typedef typename AccK<TJ>::type A;
  if (!c->active) return;
  const double rv = c->sums[0];
  const double alpha = c->rho / rv;
  const A al = (A)alpha;
  A acc[1] = {A(0)};
  VEC_LOOP(i, n) {
    const A si = (A)r[i] - al * (A)v[i];
    s[i] = (TJ)si;
    acc[0] += si * si;
  }
  __shared__ A sm[8];
  __shared__ double s_n2;
  const bool last = grid_reduce<A, 1>(acc, 1, red, gridDim.x, blockIdx.x, sm, [&](int, A q) { s_n2 = (double)q; });
  if (last && threadIdx.x == 0) {
    if (sn2) *sn2 = s_n2;
    if (rv == 0.0 || !isfinite(rv)) {
      c->breakdown = 1; c->active = 0; c->its = it + 1;
    } else {
      c->alpha = alpha;
      const double sn = sqrt(s_n2);
      c->resid = sn;
      if (!isfinite(sn)) { c->nonfinite = 1; c->active = 0; c->its = it + 1; }
      else if (sn <= c->target) { c->converged = 1; c->active = 0; c->flag_half = it + 1; c->its = it + 1; }
    }
    mirror_active(c->host_active, c->active);
  }
}

// half-step convergence of iteration `it`: x += alpha p (once)
template <class TJ, class TD>
__global__ void k_bicg_half(long long n, const TJ* __restrict__ p, TD* __restrict__ d, BicgCtl* c, int it) {
  if (c->flag_half != it + 1) return;
  const double al = c->alpha;
  VEC_LOOP(i, n) d[i] = d[i] + (TD)(al * (double)p[i]);
}

// after t = J s with sums[0] = t.s, sums[1] = t.t: omega = (t.s)/(t.t);
// x += alpha p + omega s; r = s - omega t; ||r||^2 and rhat . r (next rho)
template <class TJ, class TD>
__global__ void __launch_bounds__(256) k_bicg_x(long long n, const TJ* __restrict__ p, const TJ* __restrict__ s,
                                                const TJ* __restrict__ t, TJ* __restrict__ r,
                                                const TJ* __restrict__ rhat, TD* __restrict__ d, BicgCtl* c,
                                                RedSite<typename AccK<TJ>::type> red, int it) {
  typedef typename AccK<TJ>::type A;
  if (!c->active) return;
  const double ts = c->sums[0], tt = c->sums[1];
  const bool bad = (tt == 0.0 || !isfinite(tt) || !isfinite(ts));
  const double omega = bad ? 0.0 : ts / tt;
  const A al = (A)c->alpha, om = (A)omega;
  A acc[2] = {A(0), A(0)};
  if (!bad) {
    VEC_LOOP(i, n) {
      const A si = (A)s[i];
      d[i] = d[i] + (TD)(al * (A)p[i] + om * si);
      const A ri = si - om * (A)t[i];
      r[i] = (TJ)ri;
      acc[0] += ri * ri;
      acc[1] += (A)rhat[i] * ri;
    }
  }
  __shared__ A sm[8 * 2];
  __shared__ double s_r2, s_rr;
  const bool last = grid_reduce<A, 2>(acc, 2, red, gridDim.x, blockIdx.x, sm, [&](int q, A v) {
    if (q == 0) s_r2 = (double)v; else s_rr = (double)v; });
  if (last && threadIdx.x == 0) {
    c->its = it + 1;
    if (bad) {
      c->breakdown = 1; c->active = 0;
    } else {
      c->omega = omega;
      const double rn = sqrt(s_r2);
      c->resid = rn;
      c->rho_old = c->rho;
      c->rho = s_rr;
      if (!isfinite(rn)) { c->nonfinite = 1; c->active = 0; }
      else if (rn <= c->target) { c->converged = 1; c->active = 0; }
      else if (omega == 0.0 || s_rr == 0.0 || !isfinite(s_rr)) { c->breakdown = 1; c->active = 0; }
    }
    mirror_active(c->host_active, c->active);
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <class TB, class TJ, int KMAX>
static void arnoldi_step_k(long long n, void* V, int k, void* w, GmresCtl* ctl, RedWs red, cudaStream_t st,
                           int pass) {
  typedef typename AccK<TJ>::type A;
  RedSite<A> rs{(A*)red.partials, red.counter, red.max_blocks};
  const int nb = vec_blocks(n);
  if (pass == 1)
    k_arnoldi_dots<TB, TJ, KMAX><<<nb, kVecThreads, 0, st>>>(n, (const TB*)V, n, k, (const TJ*)w, ctl, rs);
  else if (pass == 2)
    k_arnoldi_update_dots<TB, TJ, KMAX><<<nb, kVecThreads, 0, st>>>(n, (const TB*)V, n, k, (TJ*)w, ctl, rs);
  else
    k_arnoldi_update_norm<TB, TJ, KMAX><<<nb, kVecThreads, 0, st>>>(n, (TB*)V, n, k, (const TJ*)w, ctl, rs);
}

template <class TB, class TJ>
static void arnoldi_step_t(long long n, void* V, int k, void* w, GmresCtl* ctl, RedWs red, cudaStream_t st,
                           int pass) {
  if (k <= 8) arnoldi_step_k<TB, TJ, 8>(n, V, k, w, ctl, red, st, pass);
  else if (k <= 16) arnoldi_step_k<TB, TJ, 16>(n, V, k, w, ctl, red, st, pass);
  else if (k <= 32) arnoldi_step_k<TB, TJ, 32>(n, V, k, w, ctl, red, st, pass);
  else arnoldi_step_k<TB, TJ, 64>(n, V, k, w, ctl, red, st, pass);
}

cudaError_t launch_arnoldi_pass(int pass, int tb, int tj, long long n, void* V, int k, void* w, GmresCtl* ctl,
                                RedWs red, cudaStream_t st) {
  if (k < 1 || k > kMaxM) return cudaErrorInvalidValue;
  if (tb == VT_F64 && tj == VT_F64) arnoldi_step_t<double, double>(n, V, k, w, ctl, red, st, pass);
  else if (tb == VT_F32 && tj == VT_F32) arnoldi_step_t<float, float>(n, V, k, w, ctl, red, st, pass);
  else if (tb == VT_BF16 && tj == VT_F32) arnoldi_step_t<__nv_bfloat16, float>(n, V, k, w, ctl, red, st, pass);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_gmres_init(int ts, int tj, int tb, int td, long long n, const void* F, void* u0, void* rhs,
                              void* d, GmresCtl* ctl, const double* sums, double tol, int m, cudaStream_t st) {
  const int nb = vec_blocks(n);
#define GI(TS_, TJ_, TB_, TD_) k_gmres_init<TS_, TJ_, TB_, TD_><<<nb, kVecThreads, 0, st>>>( \
    n, (const TS_*)F, (TB_*)u0, (TJ_*)rhs, (TD_*)d, ctl, sums, tol, m)
  if (ts == VT_F64 && tj == VT_F64 && tb == VT_F64 && td == VT_F64) GI(double, double, double, double);
  else if (ts == VT_F32 && tj == VT_F32 && tb == VT_F32 && td == VT_F32) GI(float, float, float, float);
  else if (ts == VT_F64 && tj == VT_F32 && tb == VT_F32 && td == VT_F64) GI(double, float, float, double);
  else if (ts == VT_F64 && tj == VT_F32 && tb == VT_BF16 && td == VT_F64) GI(double, float, __nv_bfloat16, double);
  else return cudaErrorInvalidValue;
#undef GI
  return cudaGetLastError();
}

cudaError_t launch_gmres_finish(int tb, int td, long long n, const void* V, void* d, GmresCtl* ctl, int kmax,
                                cudaStream_t st, int streamed, unsigned int* err, int nsm) {
  k_gmres_backsolve<<<1, 32, 0, st>>>(ctl);
  if (streamed) {
    const int tj = (tb == VT_F64) ? VT_F64 : VT_F32;
    return launch_basis_stream(4, tb, tj, td, n, V, 0, kmax, nullptr, d, ctl, RedWs{nullptr, nullptr, 0}, err, nsm,
                               st);
  }
  const int nb = vec_blocks(n);
#define GU(TB_, TD_, K_) k_gmres_update<TB_, TD_, K_><<<nb, kVecThreads, 0, st>>>(n, (const TB_*)V, n, (TD_*)d, ctl)
#define GUK(TB_, TD_) do { if (kmax <= 8) GU(TB_, TD_, 8); else if (kmax <= 16) GU(TB_, TD_, 16); \
                           else if (kmax <= 32) GU(TB_, TD_, 32); else GU(TB_, TD_, 64); } while (0)
  if (tb == VT_F64 && td == VT_F64) GUK(double, double);
  else if (tb == VT_F32 && td == VT_F32) GUK(float, float);
  else if (tb == VT_F32 && td == VT_F64) GUK(float, double);
  else if (tb == VT_BF16 && td == VT_F64) GUK(__nv_bfloat16, double);
  else return cudaErrorInvalidValue;
#undef GUK
#undef GU
  return cudaGetLastError();
}

// Start of the line search of one Newton step: trial alpha = 1 from the merit fnorm = ||F(x_k)||.
__global__ void k_ls_begin(LsCtl* c, double fnorm, double c1, double min_alpha, int accept_first) {
  c->fnorm = fnorm;
  c->alpha = 1.0;
  c->c1 = c1;
  c->min_alpha = min_alpha;
  c->ft = 0.0;
  c->alpha_acc = 0.0;
  c->done = 0;
  c->backtracks = 0;
  c->failures = 0;
  c->accept_first = accept_first;
}

cudaError_t launch_ls_begin(LsCtl* c, double fnorm, double c1, double min_alpha, int accept_first, cudaStream_t st) {
  k_ls_begin<<<1, 1, 0, st>>>(c, fnorm, c1, min_alpha, accept_first);
  return cudaGetLastError();
}

cudaError_t launch_cast(int ti, int to, long long n, const void* x, void* y, double c, cudaStream_t st) {
  const int nb = vec_blocks(n);
#define CA(TI_, TO_) k_cast<TI_, TO_><<<nb, kVecThreads, 0, st>>>(n, (const TI_*)x, (TO_*)y, c)
  if (ti == VT_F64 && to == VT_F64) CA(double, double);
  else if (ti == VT_F64 && to == VT_F32) CA(double, float);
  else if (ti == VT_F32 && to == VT_F64) CA(float, double);
  else if (ti == VT_F32 && to == VT_F32) CA(float, float);
  else if (ti == VT_F32 && to == VT_BF16) CA(float, __nv_bfloat16);
  else return cudaErrorInvalidValue;
#undef CA
  return cudaGetLastError();
}

cudaError_t launch_vdots(int t, long long n, int nd, const void* const* a, const void* const* b, double* sums,
                         RedWs red, const int* active, cudaStream_t st) {
  const int nb = vec_blocks(n);
  if (t == VT_F64)
    k_vdots<double><<<nb, kVecThreads, 0, st>>>(n, nd, (const double*)a[0], (const double*)b[0], (const double*)a[1],
                                                (const double*)b[1], (const double*)a[2], (const double*)b[2], sums,
                                                RedSite<double>{(double*)red.partials, red.counter, red.max_blocks}, active);
  else
    k_vdots<float><<<nb, kVecThreads, 0, st>>>(n, nd, (const float*)a[0], (const float*)b[0], (const float*)a[1],
                                               (const float*)b[1], (const float*)a[2], (const float*)b[2], sums,
                                               RedSite<float>{(float*)red.partials, red.counter, red.max_blocks}, active);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conjugate gradients (Hestenes-Stiefel) for symmetric positive definite
// Jacobians, x_0 = 0. Scalars live in BicgCtl: rho = r.r, alpha, beta;
// sums[0] = p.q from the JVP's fused dot. Every phase first checks `active`.
// ---------------------------------------------------------------------------
// init: r = p = b = -F (TJ), d = 0; rho = ||b||^2 (= ||p||^2 for the FD step)
template <class TS, class TJ, class TD>
__global__ void k_cg_init(long long n, const TS* __restrict__ F, TJ* r, TJ* p, TD* d, BicgCtl* c,
                          const double* sums, double* pn2, double tol) {
  VEC_LOOP(i, n) {
    const TJ b = (TJ)(-F[i]);
    r[i] = b; p[i] = b; d[i] = TD(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double bn = sqrt(sums[0]);
    c->bnorm = bn;
    c->target = tol * bn;
    c->rho = sums[0];
    c->beta = 0.0;
    c->its = 0; c->converged = 0; c->breakdown = 0; c->nonfinite = 0; c->flag_half = 0;
    c->resid = bn;
    c->active = (bn > 0.0 && isfinite(bn)) ? 1 : 0;
    if (bn == 0.0) c->converged = 1;
    if (!isfinite(bn)) c->nonfinite = 1;
    if (pn2) *pn2 = sums[0];
    mirror_active(c->host_active, c->active);
  }
}

// p = r + beta p (iterations after the first); ||p||^2 for the FD step
template <class TJ>
__global__ void __launch_bounds__(256) k_cg_p(long long n, const TJ* __restrict__ r, TJ* __restrict__ p, BicgCtl* c,
                                              double* pn2, RedSite<typename AccK<TJ>::type> red) {
  typedef typename AccK<TJ>::type A;
  if (!c->active) return;
  const A beta = (A)c->beta;
  A acc[1] = {A(0)};
  VEC_LOOP(i, n) {
    const A pi = (A)r[i] + beta * (A)p[i];
    p[i] = (TJ)pi;
    acc[0] += pi * pi;
  }
  if (pn2) {
    __shared__ A sm[8];
    grid_reduce<A, 1>(acc, 1, red, gridDim.x, blockIdx.x, sm, [&](int, A s) { *pn2 = (double)s; });
  }
}

// after q = J p with sums[0] = p.q: alpha = rho / (p.q); d += alpha p; r -= alpha q;
// rho' = r.r; converged on ||r|| <= target, else beta = rho' / rho
template <class TJ, class TD>
__global__ void __launch_bounds__(256) k_cg_x(long long n, const TJ* __restrict__ p, const TJ* __restrict__ q,
                                              TJ* __restrict__ r, TD* __restrict__ d, BicgCtl* c,
                                              RedSite<typename AccK<TJ>::type> red, int it) {
  typedef typename AccK<TJ>::type A;
  if (!c->active) return;
  const double pq = c->sums[0];
  const bool bad = !(pq > 0.0) || !isfinite(pq);   // J not positive definite along p
  const double alpha = bad ? 0.0 : c->rho / pq;
  const A al = (A)alpha;
  A acc[1] = {A(0)};
  if (!bad) {
    VEC_LOOP(i, n) {
      d[i] = d[i] + (TD)(al * (A)p[i]);
      const A ri = (A)r[i] - al * (A)q[i];
      r[i] = (TJ)ri;
      acc[0] += ri * ri;
    }
  }
  __shared__ A sm[8];
  __shared__ double s_r2;
  const bool last = grid_reduce<A, 1>(acc, 1, red, gridDim.x, blockIdx.x, sm, [&](int, A v) { s_r2 = (double)v; });
  if (last && threadIdx.x == 0) {
    c->its = it + 1;
    if (bad) {
      c->breakdown = 1; c->active = 0;
    } else {
      c->alpha = alpha;
      const double rn = sqrt(s_r2);
      c->resid = rn;
      if (!isfinite(rn)) { c->nonfinite = 1; c->active = 0; }
      else if (rn <= c->target) { c->converged = 1; c->active = 0; }
      else { c->beta = s_r2 / c->rho; c->rho = s_r2; }
    }
    mirror_active(c->host_active, c->active);
  }
}

cudaError_t launch_cg(int phase, int ts, int tj, int td, long long n, const BicgVecs& vv, BicgCtl* c, RedWs red,
                      int it, double tol, cudaStream_t st) {
  const int nb = vec_blocks(n);
#define CGK(TS_, TJ_, TD_)                                                                                  \
  do {                                                                                                      \
    typedef typename AccK<TJ_>::type A;                                                                     \
    RedSite<A> rs{(A*)red.partials, red.counter, red.max_blocks};                                           \
    switch (phase) {                                                                                        \
      case 0: k_cg_init<TS_, TJ_, TD_><<<nb, kVecThreads, 0, st>>>(n, (const TS_*)vv.F, (TJ_*)vv.r,         \
                  (TJ_*)vv.p, (TD_*)vv.d, c, vv.sums, vv.pn2, tol); break;                                  \
      case 1: k_cg_p<TJ_><<<nb, kVecThreads, 0, st>>>(n, (const TJ_*)vv.r, (TJ_*)vv.p, c, vv.pn2, rs);      \
              break;                                                                                        \
      case 2: k_cg_x<TJ_, TD_><<<nb, kVecThreads, 0, st>>>(n, (const TJ_*)vv.p, (const TJ_*)vv.v,           \
                  (TJ_*)vv.r, (TD_*)vv.d, c, rs, it); break;                                                \
    }                                                                                                       \
  } while (0)
  if (ts == VT_F64 && tj == VT_F64 && td == VT_F64) CGK(double, double, double);
  else if (ts == VT_F32 && tj == VT_F32 && td == VT_F32) CGK(float, float, float);
  else if (ts == VT_F64 && tj == VT_F32 && td == VT_F64) CGK(double, float, double);
  else return cudaErrorInvalidValue;
#undef CGK
  return cudaGetLastError();
}

cudaError_t launch_bicg(int phase, int ts, int tj, int td, long long n, const BicgVecs& vv, BicgCtl* c,
                        RedWs red, int it, double tol, cudaStream_t st) {
  const int nb = vec_blocks(n);
#define BI(TS_, TJ_, TD_)                                                                                   \
  do {                                                                                                      \
    typedef typename AccK<TJ_>::type A;                                                                     \
    RedSite<A> rs{(A*)red.partials, red.counter, red.max_blocks};                                                           \
    switch (phase) {                                                                                        \
      case 0: k_bicg_init<TS_, TJ_, TD_><<<nb, kVecThreads, 0, st>>>(n, (const TS_*)vv.F, (TJ_*)vv.r,       \
                  (TJ_*)vv.rhat, (TJ_*)vv.p, (TJ_*)vv.v, (TD_*)vv.d, c, vv.sums, tol); break;               \
      case 1: k_bicg_p<TJ_><<<nb, kVecThreads, 0, st>>>(n, (const TJ_*)vv.r, (TJ_*)vv.p, (const TJ_*)vv.v, c, \
                  vv.pn2, rs); break;                                                                       \
      case 2: k_bicg_s<TJ_, TD_><<<nb, kVecThreads, 0, st>>>(n, (const TJ_*)vv.r, (const TJ_*)vv.v,         \
                  (TJ_*)vv.s, c, vv.sn2, rs, it); break;                                                    \
      case 3: k_bicg_half<TJ_, TD_><<<nb, kVecThreads, 0, st>>>(n, (const TJ_*)vv.p, (TD_*)vv.d, c, it);    \
              break;                                                                                        \
      case 4: k_bicg_x<TJ_, TD_><<<nb, kVecThreads, 0, st>>>(n, (const TJ_*)vv.p, (const TJ_*)vv.s,         \
                  (const TJ_*)vv.t, (TJ_*)vv.r, (const TJ_*)vv.rhat, (TD_*)vv.d, c, rs, it); break;         \
    }                                                                                                       \
  } while (0)
  if (ts == VT_F64 && tj == VT_F64 && td == VT_F64) BI(double, double, double);
  else if (ts == VT_F32 && tj == VT_F32 && td == VT_F32) BI(float, float, float);
  else if (ts == VT_F64 && tj == VT_F32 && td == VT_F64) BI(double, float, double);
  else return cudaErrorInvalidValue;
#undef BI
  return cudaGetLastError();
}

}  // namespace jfnk
