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
#include "stream.cuh"

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

// ---------------------------------------------------------------------------
// Streaming form of the basis passes. Persistent CTAs (one per SM) walk the
// super-chunks they own: 8 KB of every vector. For each super-chunk a
// producer warp streams the w chunk and then the basis vectors in groups of
// eight (64 KB per group) through a shared-memory ring filled by bulk copies;
// eight consumer warps keep the w chunk (and the updated w) in registers and
// fold each group into it. Long contiguous runs and few concurrent streams
// keep HBM rows open, and each pass reads each basis vector once; the
// update-and-dots pass streams the groups a second time, straight from L2.
//   MODE 1  h1[t] = scale[t] sum u_t w                      (dots)
//   MODE 2  w -= sum_t h1[t] v_t ;  h2[t] = v_t . w          (update + dots)
//   MODE 3  u_k = w - sum_t h2[t] v_t ; ||u_k||^2 ; Givens   (update + norm)
//   MODE 4  d += sum_t y_t v_t                               (solution update)
// Requires n % 8 == 0 (every copy and every vector access is 16-byte sized
// and aligned).
// ---------------------------------------------------------------------------
template <class A, class T> __device__ __forceinline__ A as_arith(T x) { return (A)x; }
template <> __device__ __forceinline__ float as_arith<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ double as_arith<double, __nv_bfloat16>(__nv_bfloat16 x) {
  return (double)__bfloat162float(x);
}

constexpr int kSuperBytes = 8192;   // bytes of one vector per super-chunk
constexpr int kGroup = 8;           // basis vectors per ring stage
constexpr int kStages = 3;

// VW consecutive elements of a 16-byte slice, converted to A
template <class A, class T, int VW>
__device__ __forceinline__ void ld_slice(A (&r)[VW], const T* p) {
  const uint4 q = *(const uint4*)p;
  const T* e = (const T*)&q;
#pragma unroll
  for (int i = 0; i < VW; ++i) r[i] = as_arith<A>(e[i]);
}
// slices of TJ elements that are wider than 16 bytes (w for a BF16 basis)
template <class A, class T, int VW>
__device__ __forceinline__ void ld_any(A (&r)[VW], const T* p) {
  constexpr int PER = 16 / (int)sizeof(T);
#pragma unroll
  for (int b = 0; b < VW; b += PER) {
    const uint4 q = *(const uint4*)(p + b);
    const T* e = (const T*)&q;
#pragma unroll
    for (int i = 0; i < PER && b + i < VW; ++i) r[b + i] = as_arith<A>(e[i]);
  }
}
template <class A, class T, int VW>
__device__ __forceinline__ void st_any(T* p, const A (&r)[VW]) {
  constexpr int PER = 16 / (int)sizeof(T);
#pragma unroll
  for (int b = 0; b < VW; b += PER) {
    uint4 q;
    T* e = (T*)&q;
#pragma unroll
    for (int i = 0; i < PER; ++i) e[i] = store_as<T>::cvt(r[b + i]);
    *(uint4*)(p + b) = q;
  }
}

template <class TB, class TJ, class TD, int KMAX, int MODE>
__global__ void __launch_bounds__(kStreamThreads + 32, 1)
    k_basis_stream(long long n, const TB* __restrict__ V, long long ldv, int k, TJ* __restrict__ w,
                   TD* __restrict__ d, GmresCtl* ctl, RedSite<typename AccK<TJ>::type> red, int stage_bytes,
                   unsigned int* err) {
  typedef typename AccK<TJ>::type A;
  constexpr int CE = kSuperBytes / (int)sizeof(TB);   // elements per super-chunk
  constexpr int VW = 16 / (int)sizeof(TB);            // elements per 16-byte slice
  constexpr int R = CE / (kStreamThreads * VW);       // slices per consumer thread
  constexpr int EPT = R * VW;
  constexpr int NACC = MODE <= 2 ? KMAX : 1;
  constexpr int NGMAX = (KMAX + kGroup - 1) / kGroup;
  if (MODE != 4 && !ctl->active) return;
  if (MODE == 4) {
    k = ctl->k;
    if (k == 0) return;
  }
  extern __shared__ __align__(128) unsigned char sring[];
  uint64_t* full = (uint64_t*)(sring + (size_t)kStages * stage_bytes);
  uint64_t* empty = full + kStages;
  __shared__ A coef[kMaxM + 1];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStreamThreads / 32);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  for (int t = tid; t < k; t += blockDim.x) {
    if (MODE == 2) coef[t] = (A)(ctl->h1[t] * ctl->scale[t]);
    if (MODE == 3) coef[t] = (A)(ctl->h2[t] * ctl->scale[t]);
    if (MODE == 4) coef[t] = (A)ctl->y[t];
  }
  __syncthreads();
  const int ng = (k + kGroup - 1) / kGroup;
  const int has_w = MODE <= 3 ? 1 : 0;
  const int per_sc = has_w + ng * (MODE == 2 ? 2 : 1);    // ring items per super-chunk
  const long long nsc = (n + CE - 1) / CE;
  const long long G = gridDim.x;
  const int my_sc = ((long long)blockIdx.x < nsc) ? (int)((nsc - 1 - blockIdx.x) / G + 1) : 0;
  const int nitems = my_sc * per_sc;
  A acc[NACC];
#pragma unroll
  for (int q = 0; q < NACC; ++q) acc[q] = A(0);
  if (warp == 0) {
    // ---------------- producer ----------------
    int it = 0;
    for (; it < nitems; ++it) {
      const int sidx = it % kStages;
      if (it >= kStages && !mbar_wait_bounded(&empty[sidx], (uint32_t)(((it / kStages) - 1) & 1), kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
        break;
      }
      if (s_abort) break;
      const int sc = it / per_sc, r = it % per_sc;
      const long long e0 = ((long long)blockIdx.x + (long long)sc * G) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      unsigned char* st = sring + (size_t)sidx * stage_bytes;
      if (has_w && r == 0) {
        const uint32_t wb = (uint32_t)cnt * sizeof(TJ);
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[sidx], wb);
          bulk_g2s(st, w + e0, wb, &full[sidx]);
        }
      } else {
        const int g = (r - has_w) % ng;
        const int t0 = g * kGroup;
        const int nv = (k - t0) < kGroup ? (k - t0) : kGroup;
        const uint32_t vb = (uint32_t)cnt * sizeof(TB);
        if (lane == 0) mbar_arrive_expect_tx(&full[sidx], (uint32_t)nv * vb);
        __syncwarp();
        if (lane < nv) bulk_g2s(st + (size_t)lane * kSuperBytes, V + (t0 + lane) * ldv + e0, vb, &full[sidx]);
      }
      __syncwarp();
    }
    if (s_abort && lane == 0) {
      for (int q = (it - kStages > 0 ? it - kStages : 0); q < it; ++q)
        mbar_wait_bounded(&full[q % kStages], (uint32_t)((q / kStages) & 1), kWaitLimitNs);
    }
  } else {
    // ---------------- consumers ----------------
    const int ctid = tid - 32;
    A wr[EPT];            // w, then the updated w (modes 1-3); the sum y_t v_t (mode 4)
#pragma unroll
    for (int e = 0; e < EPT; ++e) wr[e] = A(0);
    for (int it = 0; it < nitems; ++it) {
      const int sidx = it % kStages;
      if (!mbar_wait_bounded(&full[sidx], (uint32_t)((it / kStages) & 1), kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
        break;
      }
      if (s_abort) break;
      const int sc = it / per_sc, r = it % per_sc;
      const long long e0 = ((long long)blockIdx.x + (long long)sc * G) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      const unsigned char* st = sring + (size_t)sidx * stage_bytes;
      if (has_w && r == 0) {
        const TJ* ws = (const TJ*)st;
#pragma unroll
        for (int sl = 0; sl < R; ++sl) {
          const int e = sl * kStreamThreads * VW + ctid * VW;
          A tmp[VW];
          if (e < cnt) ld_any<A, TJ, VW>(tmp, ws + e);
          else for (int i = 0; i < VW; ++i) tmp[i] = A(0);
#pragma unroll
          for (int i = 0; i < VW; ++i) wr[sl * VW + i] = tmp[i];
        }
      } else {
        const int rr = r - has_w;
        const bool pass_b = (MODE == 2) && rr >= ng;
        const int g = rr % ng;
        // group g holds vectors 8g .. 8g+7: unrolled over the possible g so that t is a compile-time index
#pragma unroll
        for (int gg = 0; gg < NGMAX; ++gg) {
          if (gg != g) continue;
#pragma unroll
          for (int q = 0; q < kGroup; ++q) {
            const int t = gg * kGroup + q;
            if (t < KMAX && t < k) {
              const TB* vs = (const TB*)(st + (size_t)q * kSuperBytes);
#pragma unroll
              for (int sl = 0; sl < R; ++sl) {
                const int e = sl * kStreamThreads * VW + ctid * VW;
                if (e < cnt) {
                  A vv[VW];
                  ld_slice<A, TB, VW>(vv, vs + e);
#pragma unroll
                  for (int i = 0; i < VW; ++i) {
                    if (MODE == 1 || (MODE == 2 && pass_b)) acc[t < NACC ? t : 0] += vv[i] * wr[sl * VW + i];
                    else if (MODE == 4) wr[sl * VW + i] += coef[t] * vv[i];
                    else wr[sl * VW + i] -= coef[t] * vv[i];
                  }
                }
              }
            }
          }
        }
        const bool end_a = (rr == ng - 1);
        if (end_a && MODE == 2) {
          // updated w: store it and round to its storage precision before the dots
#pragma unroll
          for (int sl = 0; sl < R; ++sl) {
            const int e = sl * kStreamThreads * VW + ctid * VW;
            if (e < cnt) {
              A tmp[VW];
#pragma unroll
              for (int i = 0; i < VW; ++i) { tmp[i] = (A)(TJ)wr[sl * VW + i]; wr[sl * VW + i] = tmp[i]; }
              st_any<A, TJ, VW>(w + e0 + e, tmp);
            }
          }
        }
        if (end_a && MODE == 3) {
#pragma unroll
          for (int sl = 0; sl < R; ++sl) {
            const int e = sl * kStreamThreads * VW + ctid * VW;
            if (e < cnt) {
              A tmp[VW];
#pragma unroll
              for (int i = 0; i < VW; ++i) {
                tmp[i] = as_arith<A>(store_as<TB>::cvt(wr[sl * VW + i]));
                acc[0] += tmp[i] * tmp[i];
              }
              st_any<A, TB, VW>((TB*)V + (long long)k * ldv + e0 + e, tmp);
            }
          }
        }
        if (end_a && MODE == 4) {
#pragma unroll
          for (int sl = 0; sl < R; ++sl) {
            const int e = sl * kStreamThreads * VW + ctid * VW;
            if (e < cnt) {
#pragma unroll
              for (int i = 0; i < VW; ++i) {
                TD* dp = d + e0 + e + i;
                *dp = *dp + (TD)wr[sl * VW + i];
                wr[sl * VW + i] = A(0);
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sidx]);
    }
  }
  __syncthreads();
  if (s_abort || MODE == 4) return;
  __shared__ A sm[9 * NACC];
  if (MODE <= 2) {
    grid_reduce<A, NACC>(acc, k, red, gridDim.x, blockIdx.x, sm, [&](int t, A sv) {
      if (MODE == 1) ctl->h1[t] = (double)sv * ctl->scale[t];
      else ctl->h2[t] = (double)sv * ctl->scale[t];
    });
  } else {
    __shared__ double s_n2;
    const bool last = grid_reduce<A, NACC>(acc, 1, red, gridDim.x, blockIdx.x, sm,
                                           [&](int, A sv) { s_n2 = (double)sv; });
    if (last && tid == 0) gmres_givens_step(ctl, k - 1, s_n2);
  }
}

template <class TB, class TJ, class TD, int KMAX, int MODE>
static cudaError_t stream_launch(long long n, const void* V, int k, int kmax, void* w, void* d, GmresCtl* ctl,
                                 RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  typedef typename AccK<TJ>::type A;
  (void)kmax;
  constexpr int CE = kSuperBytes / (int)sizeof(TB);
  int stage = kGroup * kSuperBytes;
  const int wbytes = CE * (int)sizeof(TJ);
  if (wbytes > stage) stage = wbytes;
  const size_t smem = (size_t)kStages * stage + (size_t)kStages * 16;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_basis_stream<TB, TJ, TD, KMAX, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_basis_stream<TB, TJ, TD, KMAX, MODE><<<nsm, kStreamThreads + 32, smem, st>>>(
      n, (const TB*)V, n, k, (TJ*)w, (TD*)d, ctl, RedSite<A>{(A*)red.partials, red.counter, red.max_blocks}, stage,
      err);
  return cudaGetLastError();
}

template <class TB, class TJ, class TD, int MODE>
static cudaError_t stream_k(long long n, const void* V, int k, int kmax, void* w, void* d, GmresCtl* ctl,
                            RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  const int kk = (MODE == 4) ? kmax : k;
  if (kk <= 8) return stream_launch<TB, TJ, TD, 8, MODE>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  if (kk <= 16) return stream_launch<TB, TJ, TD, 16, MODE>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  if (kk <= 32) return stream_launch<TB, TJ, TD, 32, MODE>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  return stream_launch<TB, TJ, TD, 64, MODE>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
}

template <class TB, class TJ, class TD>
static cudaError_t stream_mode(int mode, long long n, const void* V, int k, int kmax, void* w, void* d,
                               GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  switch (mode) {
    case 1: return stream_k<TB, TJ, TD, 1>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
    case 2: return stream_k<TB, TJ, TD, 2>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
    case 3: return stream_k<TB, TJ, TD, 3>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
    case 4: return stream_k<TB, TJ, TD, 4>(n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  }
  return cudaErrorInvalidValue;
}

bool stream_supported(long long n) { return n % 8 == 0 && n >= 8; }

cudaError_t launch_basis_stream(int mode, int tb, int tj, int td, long long n, const void* V, int k, int kmax,
                                void* w, void* d, GmresCtl* ctl, RedWs red, unsigned int* err, int nsm,
                                cudaStream_t st) {
  if (!stream_supported(n) || k > kMaxM || kmax > kMaxM) return cudaErrorInvalidValue;
  if (tb == VT_F64 && tj == VT_F64 && td == VT_F64)
    return stream_mode<double, double, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  if (tb == VT_F32 && tj == VT_F32 && td == VT_F32)
    return stream_mode<float, float, float>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  if (tb == VT_F32 && tj == VT_F32 && td == VT_F64)
    return stream_mode<float, float, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  if (tb == VT_BF16 && tj == VT_F32 && td == VT_F64)
    return stream_mode<__nv_bfloat16, float, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
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
