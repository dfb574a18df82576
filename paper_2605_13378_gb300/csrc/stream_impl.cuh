// stream_impl.cuh -- the bulk-copy streaming kernel of the GMRES basis passes
// (instantiated per basis precision in stream_f64.cu, stream_f32.cu and
// stream_bf16.cu).
#pragma once

#include "kernels.h"
#include "krylov.h"
#include "ctl.cuh"
#include "stream.cuh"

namespace jfnk {

template <class T> struct AccS { typedef float type; };
template <> struct AccS<double> { typedef double type; };

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
                   TD* __restrict__ d, GmresCtl* ctl, RedSite<typename AccS<TJ>::type> red, int stage_bytes,
                   unsigned int* err) {
  typedef typename AccS<TJ>::type A;
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
  // Ring item `it` -> (kind, super-chunk, group); kind 0 = w chunk, 1 = pass A group, 2 = pass B group.
  // Per super-chunk: [W, A.0 .. A.(ng-1)] and, for MODE 2, then [B.0 .. B.(ng-1)] while the chunk is hot in L2.
  auto item_of = [&](int it, int& kind, int& sc, int& g) {
    sc = it / per_sc;
    const int r = it % per_sc;
    if (has_w && r == 0) { kind = 0; g = 0; return; }
    const int rr = r - has_w;
    kind = rr < ng ? 1 : 2;
    g = rr % ng;
  };
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
      int kind, sc, g;
      item_of(it, kind, sc, g);
      const long long e0 = ((long long)blockIdx.x + (long long)sc * G) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      unsigned char* st = sring + (size_t)sidx * stage_bytes;
      if (kind == 0) {
        const uint32_t wb = (uint32_t)cnt * sizeof(TJ);
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[sidx], wb);
          bulk_g2s(st, w + e0, wb, &full[sidx]);
        }
      } else {
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
      const uint64_t deadline = global_timer_ns() + kWaitLimitNs;
      for (int q = (it - kStages > 0 ? it - kStages : 0); q < it; ++q)
        mbar_wait_until(&full[q % kStages], (uint32_t)((q / kStages) & 1), deadline);
    }
  } else {
    // ---------------- consumers ----------------
    const int ctid = tid - 32;
    // w, then the updated w (modes 1-3); the sum y_t v_t (mode 4)
    A w0[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) w0[e] = A(0);
    for (int it = 0; it < nitems; ++it) {
      const int sidx = it % kStages;
      if (!mbar_wait_bounded(&full[sidx], (uint32_t)((it / kStages) & 1), kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
        break;
      }
      if (s_abort) break;
      int kind, sc, g;
      item_of(it, kind, sc, g);
      const long long e0 = ((long long)blockIdx.x + (long long)sc * G) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      const unsigned char* st = sring + (size_t)sidx * stage_bytes;
      auto handle = [&](A (&wr)[EPT]) {
        if (kind == 0) {
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
          return;
        }
        const bool pass_b = (MODE == 2) && kind == 2;
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
        const bool end_a = (kind == 1) && (g == ng - 1);
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
      };
      handle(w0);
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
    if (last) gmres_givens_step_block(ctl, k - 1, s_n2);
  }
}

// ---------------------------------------------------------------------------
// Update-and-dots pass (MODE 2) with the whole super-chunk resident: the
// super-chunk is small enough (1-4 KB per vector) that all k basis vectors
// and the w chunk fit one stage of a two-stage ring, so the update and the
// dots both read shared memory and each vector crosses HBM and the copy
// engine once.
// ---------------------------------------------------------------------------
constexpr int kResStages = 2;
constexpr int kResBudget = 100 * 1024;   // bytes per stage

template <class TB, class TJ, int KMAX>
__global__ void __launch_bounds__(kStreamThreads + 32, 1)
    k_basis_resident2(long long n, const TB* __restrict__ V, long long ldv, int k, TJ* __restrict__ w, GmresCtl* ctl,
                      RedSite<typename AccS<TJ>::type> red, int scb, int stage_bytes, unsigned int* err) {
  typedef typename AccS<TJ>::type A;
  constexpr int VW = 16 / (int)sizeof(TB);
  if (!ctl->active) return;
  extern __shared__ __align__(128) unsigned char sring[];
  uint64_t* full = (uint64_t*)(sring + (size_t)kResStages * stage_bytes);
  uint64_t* empty = full + kResStages;
  __shared__ A coef[kMaxM + 1];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < kResStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStreamThreads / 32);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  for (int t = tid; t < k; t += blockDim.x) coef[t] = (A)(ctl->h1[t] * ctl->scale[t]);
  __syncthreads();
  const int CE = scb / (int)sizeof(TB);
  const long long nsc = (n + CE - 1) / CE;
  const long long G = gridDim.x;
  const int my = ((long long)blockIdx.x < nsc) ? (int)((nsc - 1 - blockIdx.x) / G + 1) : 0;
  A acc[KMAX];
#pragma unroll
  for (int q = 0; q < KMAX; ++q) acc[q] = A(0);
  if (warp == 0) {
    int it = 0;
    for (; it < my; ++it) {
      const int sidx = it % kResStages;
      if (it >= kResStages &&
          !mbar_wait_bounded(&empty[sidx], (uint32_t)(((it / kResStages) - 1) & 1), kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
        break;
      }
      if (s_abort) break;
      const long long e0 = ((long long)blockIdx.x + (long long)it * G) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      const uint32_t vb = (uint32_t)cnt * sizeof(TB), wb = (uint32_t)cnt * sizeof(TJ);
      unsigned char* st = sring + (size_t)sidx * stage_bytes;
      if (lane == 0) mbar_arrive_expect_tx(&full[sidx], (uint32_t)k * vb + wb);
      __syncwarp();
      for (int t = lane; t <= k; t += 32) {
        if (t < k) bulk_g2s(st + (size_t)t * scb, V + t * ldv + e0, vb, &full[sidx]);
        else bulk_g2s(st + (size_t)k * scb, w + e0, wb, &full[sidx]);
      }
      __syncwarp();
    }
    if (s_abort && lane == 0) {
      const uint64_t deadline = global_timer_ns() + kWaitLimitNs;
      for (int q = (it - kResStages > 0 ? it - kResStages : 0); q < it; ++q)
        mbar_wait_until(&full[q % kResStages], (uint32_t)((q / kResStages) & 1), deadline);
    }
  } else {
    const int ctid = tid - 32;
    const int e = ctid * VW;   // this thread's slice of every chunk
    for (int it = 0; it < my; ++it) {
      const int sidx = it % kResStages;
      if (!mbar_wait_bounded(&full[sidx], (uint32_t)((it / kResStages) & 1), kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
        break;
      }
      if (s_abort) break;
      const long long e0 = ((long long)blockIdx.x + (long long)it * G) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      const unsigned char* st = sring + (size_t)sidx * stage_bytes;
      if (e < cnt) {
        A wr[VW];
        ld_any<A, TJ, VW>(wr, (const TJ*)(st + (size_t)k * scb) + e);
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
          if (t < k) {
            A vv[VW];
            ld_slice<A, TB, VW>(vv, (const TB*)(st + (size_t)t * scb) + e);
#pragma unroll
            for (int i = 0; i < VW; ++i) wr[i] -= coef[t] * vv[i];
          }
        }
#pragma unroll
        for (int i = 0; i < VW; ++i) wr[i] = (A)(TJ)wr[i];
        st_any<A, TJ, VW>(w + e0 + e, wr);
        __syncwarp(__activemask());   // re-read the chunk rather than keep k slices in registers
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
          if (t < k) {
            A vv[VW];
            ld_slice<A, TB, VW>(vv, (const TB*)(st + (size_t)t * scb) + e);
#pragma unroll
            for (int i = 0; i < VW; ++i) acc[t] += vv[i] * wr[i];
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sidx]);
    }
  }
  __syncthreads();
  if (s_abort) return;
  __shared__ A sm[9 * KMAX];
  grid_reduce<A, KMAX>(acc, k, red, gridDim.x, blockIdx.x, sm,
                       [&](int t, A sv) { ctl->h2[t] = (double)sv * ctl->scale[t]; });
}

// Chunk bytes per vector for the resident form, or 0 when k vectors do not fit.
template <class TB, class TJ>
static int resident_scb(int k, int* stage) {
  for (int scb = 4096; scb >= 1024; scb >>= 1) {
    const int ce = scb / (int)sizeof(TB);
    if (ce < 16 / (int)sizeof(TB) * 32) break;
    if (ce > kStreamThreads * (16 / (int)sizeof(TB))) continue;   // one 16-byte slice per consumer thread
    int st = k * scb + ce * (int)sizeof(TJ);
    st = (st + 127) / 128 * 128;
    if (st <= kResBudget) { *stage = st; return scb; }
  }
  return 0;
}

template <class TB, class TJ, int KMAX>
static cudaError_t resident2_launch(long long n, const void* V, int k, void* w, GmresCtl* ctl, RedWs red,
                                    unsigned int* err, int nsm, cudaStream_t st, bool* used) {
  typedef typename AccS<TJ>::type A;
  int stage = 0;
  const int scb = resident_scb<TB, TJ>(k, &stage);
  *used = scb > 0;
  if (!*used) return cudaSuccess;
  const size_t smem = (size_t)kResStages * stage + (size_t)kResStages * 16;
  static SmemOptIn opt_in;
  cudaError_t e = smem_opt_in(k_basis_resident2<TB, TJ, KMAX>, opt_in, kResStages * kResBudget + 64);
  if (e != cudaSuccess) return e;
  k_basis_resident2<TB, TJ, KMAX><<<nsm, kStreamThreads + 32, smem, st>>>(
      n, (const TB*)V, n, k, (TJ*)w, ctl, RedSite<A>{(A*)red.partials, red.counter, red.max_blocks}, scb, stage, err);
  return cudaGetLastError();
}

template <class TB, class TJ, class TD, int KMAX, int MODE>
static cudaError_t stream_launch(long long n, const void* V, int k, int kmax, void* w, void* d, GmresCtl* ctl,
                                 RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  typedef typename AccS<TJ>::type A;
  (void)kmax;
  constexpr int CE = kSuperBytes / (int)sizeof(TB);
  int stage = kGroup * kSuperBytes;
  const int wbytes = CE * (int)sizeof(TJ);
  if (wbytes > stage) stage = wbytes;
  const size_t smem = (size_t)kStages * stage + (size_t)kStages * 16;
  static SmemOptIn opt_in;
  cudaError_t e = smem_opt_in(k_basis_stream<TB, TJ, TD, KMAX, MODE>, opt_in, (int)smem);
  if (e != cudaSuccess) return e;
  k_basis_stream<TB, TJ, TD, KMAX, MODE><<<nsm, kStreamThreads + 32, smem, st>>>(
      n, (const TB*)V, n, k, (TJ*)w, (TD*)d, ctl, RedSite<A>{(A*)red.partials, red.counter, red.max_blocks}, stage,
      err);
  return cudaGetLastError();
}

template <class TB, class TJ, class TD, int MODE>
static cudaError_t stream_k(long long n, const void* V, int k, int kmax, void* w, void* d, GmresCtl* ctl,
                            RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  const int kk = (MODE == 4) ? kmax : k;
  if (MODE == 2 && sizeof(TB) <= 4) {   // FP64 is ALU-bound: keep every consumer thread busy (grouped form)
    bool used = false;
    cudaError_t e;
    if (kk <= 8) e = resident2_launch<TB, TJ, 8>(n, V, k, w, ctl, red, err, nsm, st, &used);
    else if (kk <= 16) e = resident2_launch<TB, TJ, 16>(n, V, k, w, ctl, red, err, nsm, st, &used);
    else if (kk <= 32) e = resident2_launch<TB, TJ, 32>(n, V, k, w, ctl, red, err, nsm, st, &used);
    else e = resident2_launch<TB, TJ, 64>(n, V, k, w, ctl, red, err, nsm, st, &used);
    if (used || e != cudaSuccess) return e;
  }
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

}  // namespace jfnk
