// dcgs_impl.cuh -- the two fused basis passes of delayed CGS2 (see dcgs_step in
// ctl.cuh), instantiated per basis precision in stream_f64.cu, stream_f32.cu
// and stream_bf16.cu:
//   dots    q_i . u_j and q_i . w for i <= j (slot j holds u_j itself, so
//           i = j gives u_j . u_j and u_j . w), then the step's scalar work
//   update  q_j = dgamma u_j - sum_i da_i q_i (written over slot j),
//           u_{j+1} = dinvr (w - sum_i dc_i q_i - dc_j q_j) (slot j + 1) and
//           ||u_{j+1}||^2
// Each reads basis slots 0..j and w once, against three passes of CGS2.
// Resident form: one super-chunk of every vector involved fills one entry of
// a shared-memory ring (bulk copies by producer warp 0, eight consumer warps);
// the ring has as many entries as fit the device's per-block limit (227 KB on
// GB300, less the kernel's static shared memory), so that short passes keep
// more than one entry in flight while the consumers read another. The update
// pass takes each block's super-chunks in reverse order, so that it starts on
// the chunks the dots pass read last, which the 129 MB L2 may still hold.
// Requires n % 8 == 0, like the other streaming passes.
#pragma once

#include <type_traits>

#include "stream_impl.cuh"

namespace jfnk {

constexpr int kDcgsBudget = 100 * 1024;   // largest entry: two entries always fit
constexpr int kDcgsMaxStages = 32;

// bytes per vector of a super-chunk holding nv basis slots (+ the w chunk):
// the largest candidate up to 32 KB whose entry fits the budget (larger bulk
// copies stream faster; chunks shrink only as the basis grows). The update
// pass (pass 2) also takes 3 KB between 4 and 2 KB: there, fewer bulk copies
// per byte paid off, while the dots pass streamed faster with 2 KB chunks and
// a deeper ring. Every candidate is a multiple of 16 bytes (bulk-copy
// granule), and the passes take any number of slices per chunk.
template <class TB, class TJ>
static int dcgs_scb(int pass, int nv, bool has_w, int* stage) {
  constexpr int kCand[] = {32768, 16384, 8192, 4096, 3072, 2048, 1024, 512};
  for (int scb : kCand) {
    if (scb == 3072 && pass != 2) continue;
    const int ce = scb / (int)sizeof(TB);
    int st = nv * scb + (has_w ? ce * (int)sizeof(TJ) : 0);
    st = (st + 127) / 128 * 128;
    if (st <= kDcgsBudget) { *stage = st; return scb; }
  }
  return 0;
}

// producer: slots 0..nv-1 of this block's super-chunk `c`, then (w not null)
// the w chunk, into ring entry it % nst (`it` counts the entries filled)
template <class TB, class TJ>
__device__ __forceinline__ bool dcgs_produce(int it, int c, long long n, const TB* V, const TJ* w, int nv, int CE,
                                             int scb, int stage_bytes, int nst, unsigned char* sring, uint64_t* full,
                                             uint64_t* empty, unsigned int* err, int* s_abort) {
  const int lane = threadIdx.x & 31;
  const int sidx = it % nst;
  if (it >= nst &&
      !mbar_wait_bounded(&empty[sidx], (uint32_t)(((it / nst) - 1) & 1), kWaitLimitNs)) {
    if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); *s_abort = 1; }
    return false;
  }
  if (*s_abort) return false;
  const long long e0 = ((long long)blockIdx.x + (long long)c * gridDim.x) * CE;
  const long long rem = n - e0;
  const int cnt = rem < CE ? (int)rem : CE;
  const uint32_t vb = (uint32_t)cnt * sizeof(TB), wb = (uint32_t)cnt * sizeof(TJ);
  unsigned char* st = sring + (size_t)sidx * stage_bytes;
  if (lane == 0) mbar_arrive_expect_tx(&full[sidx], (uint32_t)nv * vb + (w ? wb : 0u));
  __syncwarp();
  for (int t = lane; t <= nv; t += 32) {
    if (t < nv) bulk_g2s(st + (size_t)t * scb, V + (long long)t * n + e0, vb, &full[sidx]);
    else if (w) bulk_g2s(st + (size_t)nv * scb, w + e0, wb, &full[sidx]);
  }
  __syncwarp();
  return true;
}

// Dots pass. FP32 accumulators and at most 24 basis slots (kJoint): every
// consumer thread owns slices sl = t, t + 256, ... of every chunk and keeps
// two accumulators per basis slot, q_i . u_j and q_i . w, so each basis slice
// is read from shared memory once (FP32 bases keep chunks of at least 4 KB,
// 256 slices, up to 24 slots; a BF16 basis drops to 128 slices at j = 23).
// Otherwise (FP64 accumulators, or longer bases, whose 2 KB chunks hold 128
// slices) warps 1-4 accumulate q_i . u_j and warps 5-8 q_i . w, each of the
// 128 threads of a group owning slices sl = t, t + 128, ...
// The last block to finish sums the block partials and runs dcgs_step; in the
// deferred form (defer, with w) the pass ends when every block has stored its
// partials, value-major after the first gridDim.x kMaxK doubles
// (partials[G kMaxK + v G + b]), and every block of the update pass sums them
// and runs the step itself.
template <class TB, class TJ, int KMAX>
__global__ void __launch_bounds__(kStreamThreads + 32, 1)
    k_dcgs_dots(long long n, const TB* __restrict__ V, int j, const TJ* __restrict__ w, GmresCtl* ctl,
                double* partials, unsigned int* counter, int cap, int scb, int stage_bytes, int nst, int defer,
                unsigned int* err) {
  typedef typename AccS<TJ>::type A;
  constexpr int VW = 16 / (int)sizeof(TB);
  constexpr int NA = KMAX + 1;                 // accumulators: basis slots 0..j, j <= KMAX
  constexpr int GT = kStreamThreads / 2;       // threads per group (split form)
  constexpr bool kJoint = sizeof(A) == 4 && KMAX <= 24;   // chunks of at least 256 slices: every thread busy
  constexpr int NW = kJoint ? NA : 1;          // w accumulators of the joint form
  grid_dep_wait();      // the JVP that wrote w has completed (programmatic launch)
  grid_dep_trigger();
  const bool dfr = defer && w != nullptr;
  // host sizing error: never write past the partials
  if (!ctl->active || (dfr ? 2 : 1) * (int)gridDim.x > cap) return;
  extern __shared__ __align__(128) unsigned char sring[];
  uint64_t* full = (uint64_t*)(sring + (size_t)nst * stage_bytes);
  uint64_t* empty = full + nst;
  __shared__ int s_abort;
  __shared__ unsigned int s_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < nst; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStreamThreads / 32);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  const int nv = j + 1;
  const bool has_w = w != nullptr;
  const int CE = scb / (int)sizeof(TB);
  const long long nsc = (n + CE - 1) / CE;
  const int my = ((long long)blockIdx.x < nsc) ? (int)((nsc - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int role = (warp - 1) >> 2;            // split form: 0 dots with u_j, 1 dots with w
  const int gt = ((warp - 1) & 3) * 32 + lane;
  A acc[NA], accw[NW];
#pragma unroll
  for (int t = 0; t < NA; ++t) acc[t] = A(0);
#pragma unroll
  for (int t = 0; t < NW; ++t) accw[t] = A(0);
  if (warp == 0) {
    int it = 0;
    for (; it < my; ++it)
      if (!dcgs_produce<TB, TJ>(it, it, n, V, w, nv, CE, scb, stage_bytes, nst, sring, full, empty, err, &s_abort)) break;
    if (s_abort && lane == 0) {
      const uint64_t deadline = global_timer_ns() + kWaitLimitNs;
      for (int q = (it - nst > 0 ? it - nst : 0); q < it; ++q)
        mbar_wait_until(&full[q % nst], (uint32_t)((q / nst) & 1), deadline);
    }
  } else {
    for (int it = 0; it < my; ++it) {
      const int sidx = it % nst;
      if (!mbar_wait_bounded(&full[sidx], (uint32_t)((it / nst) & 1), kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
        break;
      }
      if (s_abort) break;
      const long long e0 = ((long long)blockIdx.x + (long long)it * gridDim.x) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      const int nsl = cnt / VW;
      const unsigned char* st = sring + (size_t)sidx * stage_bytes;
      if constexpr (kJoint) {
        const TB* uj = (const TB*)(st + (size_t)j * scb);
        if (has_w) {
          const TJ* ws = (const TJ*)(st + (size_t)nv * scb);
          for (int sl = tid - 32; sl < nsl; sl += kStreamThreads) {
            A x[VW], y[VW];
            ld_slice<A, TB, VW>(x, uj + sl * VW);
            ld_any<A, TJ, VW>(y, ws + sl * VW);
#pragma unroll
            for (int t = 0; t < NA; ++t) {
              if (t <= j) {
                A q[VW];
                ld_slice<A, TB, VW>(q, (const TB*)(st + (size_t)t * scb) + sl * VW);
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                  acc[t] += q[e] * x[e];
                  accw[t] += q[e] * y[e];
                }
              }
            }
          }
        } else {
          for (int sl = tid - 32; sl < nsl; sl += kStreamThreads) {
            A x[VW];
            ld_slice<A, TB, VW>(x, uj + sl * VW);
#pragma unroll
            for (int t = 0; t < NA; ++t) {
              if (t <= j) {
                A q[VW];
                ld_slice<A, TB, VW>(q, (const TB*)(st + (size_t)t * scb) + sl * VW);
#pragma unroll
                for (int e = 0; e < VW; ++e) acc[t] += q[e] * x[e];
              }
            }
          }
        }
      } else if (role == 0 || has_w) {
        for (int sl = gt; sl < nsl; sl += GT) {
          A x[VW];
          if (role == 0) ld_slice<A, TB, VW>(x, (const TB*)(st + (size_t)j * scb) + sl * VW);
          else ld_any<A, TJ, VW>(x, (const TJ*)(st + (size_t)nv * scb) + sl * VW);
#pragma unroll
          for (int t = 0; t < NA; ++t) {
            if (t <= j) {
              A q[VW];
              ld_slice<A, TB, VW>(q, (const TB*)(st + (size_t)t * scb) + sl * VW);
#pragma unroll
              for (int e = 0; e < VW; ++e) acc[t] += q[e] * x[e];
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sidx]);
    }
  }
  __syncthreads();
  if (s_abort) return;
  // block partials: warp butterflies, then the warps in order (all eight in the
  // joint form, the four of each group in the split form); FP32 partials as
  // float-float pairs (the cross-block sums then stay in FP32 arithmetic)
  constexpr bool kFF = std::is_same<A, float>::value;
  const int G = (int)gridDim.x;
  double* const pdst = dfr ? partials + (size_t)G * kMaxK + blockIdx.x : partials + (size_t)blockIdx.x * kMaxK;
  const int pstr = dfr ? G : 1;   // value stride of this block's partials
  if constexpr (kJoint) {
    __shared__ float redj[kStreamThreads / 32][2 * NA];
    if (warp >= 1) {
#pragma unroll
      for (int t = 0; t < NA; ++t) {
        if (t <= j) {
          const float su = warp_sum(acc[t]), sw = warp_sum(accw[t]);
          if (lane == 0) { redj[warp - 1][2 * t] = su; redj[warp - 1][2 * t + 1] = sw; }
        }
      }
    }
    __syncthreads();
    for (int v = tid; v < 2 * nv; v += blockDim.x) {
      FF sum{redj[0][v], 0.0f};
#pragma unroll
      for (int q = 1; q < kStreamThreads / 32; ++q) sum = ff_add(sum, FF{redj[q][v], 0.0f});
      ff_store(&pdst[(size_t)v * pstr], sum);
    }
  } else {
    __shared__ double red[kStreamThreads / 32][NA];
    if (warp >= 1) {
#pragma unroll
      for (int t = 0; t < NA; ++t) {
        if (t <= j) {
          const A sv = warp_sum(acc[t]);
          if (lane == 0) red[warp - 1][t] = (double)sv;
        }
      }
    }
    __syncthreads();
    for (int v = tid; v < 2 * nv; v += blockDim.x) {
      const int r = v & 1, t = v >> 1;
      if constexpr (kFF) {
        FF sum{(float)red[4 * r][t], 0.0f};
#pragma unroll
        for (int q = 1; q < 4; ++q) sum = ff_add(sum, FF{(float)red[4 * r + q][t], 0.0f});
        ff_store(&pdst[(size_t)v * pstr], sum);
      } else {
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) sum += red[4 * r + q][t];
        pdst[(size_t)v * pstr] = sum;
      }
    }
  }
  if (dfr) return;   // the update pass sums the partials (the kernel boundary orders them)
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double S[2 * (kMaxM + 1)];
  __shared__ double sh[5 * (kMaxM + 1)];
  __shared__ double s_ctl[4];
  __shared__ float s_fhi[2 * (kMaxM + 1)], s_flo[2 * (kMaxM + 1)];
  __shared__ int s_m, s_active, s_its;
  // one round of loads: every block's partials into the drained ring (when
  // they fit beside the completed Hessenberg columns), the control state into
  // shared memory
  const int nval = 2 * nv;
  const size_t ring = (size_t)nst * stage_bytes;
  // partials staged value-major with a padded row, [nval][G + 1], so that the
  // lanes of a warp summing one value read consecutive banks
  const bool staged = ((size_t)(G + 1) * nval + (size_t)j * (kMaxM + 1)) * sizeof(double) <= ring;
  double* hs = (double*)sring;                       // completed Hessenberg columns
  double* pr = hs + (size_t)j * (kMaxM + 1);         // [nval][G + 1]
  // every load of the tail is issued before any store: the completed
  // Hessenberg columns and the control state (what dcgs_stage stages), then
  // the partials, 24 per thread (e = b nval + v advanced without divisions)
  constexpr int LD = kMaxM + 1;
  const int T = (int)blockDim.x, cj = j - 1, ne = (j > 0 ? cj : 0) * LD;
  double hv[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = tid + q * T;
    hv[q] = e < ne ? __ldcg(&ctl->Hraw[e]) : 0.0;
  }
  double hp = 0.0, hc = 0.0, hn = 0.0;
  if (tid < j) {
    hp = __ldcg(&ctl->hprev[tid]);
    if (tid < cj) { hc = __ldcg(&ctl->cs[tid]); hn = __ldcg(&ctl->sn[tid]); }
  }
  double c0 = 0.0, c1 = 0.0, c2 = 0.0;
  int cm = 0, cact = 0, cits = 0;
  if (tid == 0) {
    c0 = ctl->scale[j];
    c1 = j > 0 ? ctl->g[j - 1] : ctl->g[0];
    c2 = ctl->target;
    cm = ctl->m;
    cact = ctl->active;
    cits = ctl->its;
  }
  if (staged) {
    const int total = G * nval, db = T / nval, dvv = T - db * nval;
    int b = tid / nval, v = tid - (tid / nval) * nval;
    for (int e0 = tid; e0 < total; e0 += 24 * T) {
      double val[24];
      int bq = b, vq = v;
#pragma unroll
      for (int q = 0; q < 24; ++q) {
        const int e = e0 + q * T;
        val[q] = e < total ? __ldcg(&partials[(size_t)bq * kMaxK + vq]) : 0.0;
        vq += dvv;
        bq += db;
        if (vq >= nval) { vq -= nval; ++bq; }
      }
      bq = b;
      vq = v;
#pragma unroll
      for (int q = 0; q < 24; ++q) {
        const int e = e0 + q * T;
        if (e < total) pr[(size_t)vq * (G + 1) + bq] = val[q];
        vq += dvv;
        bq += db;
        if (vq >= nval) { vq -= nval; ++bq; }
      }
      b = bq;
      v = vq;
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = tid + q * T;
    if (e < ne) hs[e] = hv[q];
  }
  if (tid < j) {
    sh[2 * LD + tid] = hp;
    if (tid < cj) { sh[3 * LD + tid] = hc; sh[4 * LD + tid] = hn; }
  }
  if (tid == 0) {
    s_ctl[0] = c0;
    s_ctl[1] = c1;
    s_ctl[2] = c2;
    s_ctl[3] = 1.0 / c0;
    s_m = cm;
    s_active = cact;
    s_its = cits;
  }
  __syncthreads();
  // warp per value, lanes over blocks in a fixed order, then the butterfly;
  // four values of a warp at once so that their dependent adds interleave
  const int nw = (int)(blockDim.x >> 5);
  for (int v0 = warp; v0 < nval; v0 += 4 * nw) {
    if constexpr (kFF) {
      FF sum[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
      // five blocks per lane and value loaded ahead of the dependent adds
      for (int b0 = lane; b0 < G; b0 += 5 * 32) {
        FF x[4][5];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            const int b = b0 + 32 * k;
            x[u][k] = FF{0.0f, 0.0f};
            if (v < nval && b < G) x[u][k] = staged ? ff_load(&pr[(size_t)v * (G + 1) + b])
                                                    : ff_load(&partials[(size_t)b * kMaxK + v]);
          }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (b0 + 32 * k < G) sum[u] = ff_add(sum[u], x[u][k]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) sum[u] = warp_sum_ff(sum[u]);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
          if (v < nval) { s_fhi[v] = sum[u].hi; s_flo[v] = sum[u].lo; }
        }
      }
    } else {
      double sum[4] = {0.0, 0.0, 0.0, 0.0};
      if (staged) {
        for (int b = lane; b < G; b += 32) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int v = v0 + u * nw;
            if (v < nval) sum[u] += pr[(size_t)v * (G + 1) + b];
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
          if (v < nval) sum[u] = lane_strided_sum(partials + v, kMaxK, G, lane);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) sum[u] = warp_sum(sum[u]);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
          if (v < nval) S[v] = sum[u];
        }
      }
    }
  }
  __syncthreads();
  if constexpr (kFF) {
    // the float-float sums to FP64, one value per thread (the conversions run on the
    // FP64 pipe, so they are spread over the block rather than left to lane 0 of each warp)
    if (tid < nval) S[tid] = (double)s_fhi[tid] + (double)s_flo[tid];
    __syncthreads();
  }
  dcgs_step(ctl, j, S, has_w, sh, hs, s_ctl[0], s_ctl[3], s_ctl[1], s_ctl[2], s_m, s_active, s_its);
  __syncthreads();
  if (tid == 0) *counter = 0u;
}

// Start of the update pass in the deferred form, run by the consumer warps
// while warp 0 fills the ring: the sums of the dots pass's block partials
// (each value by one warp over the blocks in a fixed order, so that every
// block forms the same bits), then dcgs_step_t with block 0 as the only
// writer of the control state. The step's inputs that block 0 overwrites are
// read from this step's parity slot; the completed Hessenberg columns are read
// from global memory (no shared memory taken from the ring). The coefficients
// go to ca, cc (cc[j] the coefficient of q_j), s_gamma, s_invr.
template <class A>
__device__ __forceinline__ bool dcgs_deferred_step(GmresCtl* ctl, int j, const double* __restrict__ dpart, int G,
                                                   A* ca, A* cc, A* s_gamma, A* s_invr) {
  constexpr int LD = kMaxM + 1;
  constexpr bool kFF = std::is_same<A, float>::value;
  __shared__ double S[2 * LD];
  __shared__ double sh[5 * LD];
  __shared__ double hcol[LD];
  const ConsumerTeam tm;
  const int r = tm.rank(), T = tm.size(), lane = r & 31, warp = r >> 5, nw = T >> 5;
  const int nval = 2 * (j + 1), cj = j - 1, p = j & 1;
  for (int i = r; i < j; i += T) {
    sh[2 * LD + i] = __ldcg(&ctl->hprev_p[p][i]);
    if (i < cj) { sh[3 * LD + i] = __ldcg(&ctl->cs[i]); sh[4 * LD + i] = __ldcg(&ctl->sn[i]); }
  }
  const double sigma = __ldcg(&ctl->scale[j]), g_prev = __ldcg(&ctl->gprev_p[p]), target = __ldcg(&ctl->target);
  const int m = __ldcg(&ctl->m), its0 = __ldcg(&ctl->its_p[p]);
  // four values per warp at once, five blocks per lane and value loaded ahead
  // of the dependent adds (value-major partials: the lanes read adjacent words)
  for (int v0 = warp; v0 < nval; v0 += 4 * nw) {
    if constexpr (kFF) {
      FF sum[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
      for (int b0 = lane; b0 < G; b0 += 5 * 32) {
        FF x[4][5];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            const int b = b0 + 32 * k;
            x[u][k] = (v < nval && b < G) ? ff_load(&dpart[(size_t)v * G + b]) : FF{0.0f, 0.0f};
          }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (b0 + 32 * k < G) sum[u] = ff_add(sum[u], x[u][k]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) sum[u] = warp_sum_ff(sum[u]);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
          if (v < nval) S[v] = (double)sum[u].hi + (double)sum[u].lo;
        }
      }
    } else {
      double sum[4] = {0.0, 0.0, 0.0, 0.0};
      for (int b = lane; b < G; b += 32) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
          if (v < nval) sum[u] += __ldcg(&dpart[(size_t)v * G + b]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) sum[u] = warp_sum(sum[u]);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + u * nw;
          if (v < nval) S[v] = sum[u];
        }
      }
    }
  }
  tm.sync();
  // the pass runs only while the cycle is active (checked at its entry), so active0 = 1
  return dcgs_step_t<ConsumerTeam, false, A>(ctl, j, S, true, sh, hcol, sigma, 1.0 / sigma, g_prev, target, m, 1,
                                             its0, tm, blockIdx.x == 0, ca, cc, s_gamma, s_invr);
}

// Update pass. Deferred form (dpart, the dots pass's value-major partials):
// warp 0 fills the free ring entries while the consumer warps run the step,
// then both wait on named barrier 2 for its decision; when the step ends the
// cycle the pass streams nothing (every block reaches the same decision) and
// waits for its fills before it returns.
template <class TB, class TJ, int KMAX>
__global__ void __launch_bounds__(kStreamThreads + 32, 1)
    k_dcgs_update(long long n, TB* __restrict__ V, int j, const TJ* __restrict__ w, GmresCtl* ctl,
                  RedSite<typename AccS<TJ>::type> red, const double* __restrict__ dpart, int scb, int stage_bytes,
                  int nst, unsigned int* err) {
  typedef typename AccS<TJ>::type A;
  constexpr int VW = 16 / (int)sizeof(TB);
  grid_dep_wait();      // the dots pass has completed
  grid_dep_trigger();
  if (!ctl->active) return;
  extern __shared__ __align__(128) unsigned char sring[];
  uint64_t* full = (uint64_t*)(sring + (size_t)nst * stage_bytes);
  uint64_t* empty = full + nst;
  __shared__ A ca[kMaxM + 1], cc[kMaxM + 1];
  __shared__ A s_gamma, s_invr;
  __shared__ int s_abort, s_go;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool deferred = dpart != nullptr;
  if (tid == 0) {
    for (int q = 0; q < nst; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStreamThreads / 32);
    }
    fence_mbar_init();
    s_abort = 0;
    s_go = 1;
    if (!deferred) {
      s_gamma = (A)ctl->dgamma;
      s_invr = (A)ctl->dinvr;
      cc[j] = (A)ctl->dc[j];
    }
  }
  if (!deferred)
    for (int t = tid; t < j; t += blockDim.x) {
      ca[t] = (A)ctl->da[t];
      cc[t] = (A)ctl->dc[t];
    }
  __syncthreads();
  const int nv = j + 1;
  const int CE = scb / (int)sizeof(TB);
  const long long nsc = (n + CE - 1) / CE;
  const int my = ((long long)blockIdx.x < nsc) ? (int)((nsc - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  A acc[1] = {A(0)};
  if (warp == 0) {
    int it = 0;
    const int pre = deferred ? (my < nst ? my : nst) : my;   // before the decision: the free entries only
    for (; it < pre; ++it)
      if (!dcgs_produce<TB, TJ>(it, my - 1 - it, n, V, w, nv, CE, scb, stage_bytes, nst, sring, full, empty, err,
                                &s_abort))
        break;
    if (deferred) {
      named_sync(2, blockDim.x);   // the step's decision
      if (s_go && !s_abort)
        for (; it < my; ++it)
          if (!dcgs_produce<TB, TJ>(it, my - 1 - it, n, V, w, nv, CE, scb, stage_bytes, nst, sring, full, empty,
                                    err, &s_abort))
            break;
    }
    if ((s_abort || !s_go) && lane == 0) {   // wait for the fills in flight before returning
      const uint64_t deadline = global_timer_ns() + kWaitLimitNs;
      for (int q = (it - nst > 0 ? it - nst : 0); q < it; ++q)
        mbar_wait_until(&full[q % nst], (uint32_t)((q / nst) & 1), deadline);
    }
  } else {
    if (deferred) {
      const bool go = dcgs_deferred_step<A>(ctl, j, dpart, (int)gridDim.x, ca, cc, &s_gamma, &s_invr);
      if (tid == 32) s_go = go;
      named_sync(2, blockDim.x);
    }
    const A gam = s_gamma, cj = cc[j], invr = s_invr;
    for (int it = 0; s_go && it < my; ++it) {
      const int sidx = it % nst;
      if (!mbar_wait_bounded(&full[sidx], (uint32_t)((it / nst) & 1), kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
        break;
      }
      if (s_abort) break;
      const long long e0 = ((long long)blockIdx.x + (long long)(my - 1 - it) * gridDim.x) * CE;
      const long long rem = n - e0;
      const int cnt = rem < CE ? (int)rem : CE;
      const unsigned char* st = sring + (size_t)sidx * stage_bytes;
      for (int e = (tid - 32) * VW; e < cnt; e += kStreamThreads * VW) {   // this thread's slices of the chunk
        A q[VW], y[VW];
        ld_slice<A, TB, VW>(q, (const TB*)(st + (size_t)j * scb) + e);
        ld_any<A, TJ, VW>(y, (const TJ*)(st + (size_t)nv * scb) + e);
#pragma unroll
        for (int i = 0; i < VW; ++i) q[i] *= gam;
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
          if (t < j) {
            A v[VW];
            ld_slice<A, TB, VW>(v, (const TB*)(st + (size_t)t * scb) + e);
            const A a = ca[t], c = cc[t];
#pragma unroll
            for (int i = 0; i < VW; ++i) {
              q[i] -= a * v[i];
              y[i] -= c * v[i];
            }
          }
        }
        // q_j as stored, then u_{j+1} from it
#pragma unroll
        for (int i = 0; i < VW; ++i) {
          q[i] = as_arith<A>(store_as<TB>::cvt(q[i]));
          y[i] = as_arith<A>(store_as<TB>::cvt((y[i] - cj * q[i]) * invr));
          acc[0] += y[i] * y[i];
        }
        st_any<A, TB, VW>(V + (long long)j * n + e0 + e, q);
        st_any<A, TB, VW>(V + (long long)(j + 1) * n + e0 + e, y);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sidx]);
    }
  }
  __syncthreads();
  if (s_abort || !s_go) return;
  __shared__ A sm[9];
  __shared__ double s_n2;
  const bool last = grid_reduce<A, 1>(acc, 1, red, gridDim.x, blockIdx.x, sm, [&](int, A sv) { s_n2 = (double)sv; });
  if (last && tid == 0) dcgs_after_update(ctl, j, s_n2);
}

template <class TB, class TJ, int KMAX>
static cudaError_t dcgs_launch_k(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                                 unsigned int* err, int nsm, cudaStream_t st, bool pdl, bool defer) {
  typedef typename AccS<TJ>::type A;
  if (defer && (w == nullptr || red.max_blocks < 2 * nsm)) return cudaErrorInvalidValue;
  int stage = 0;
  const int scb = dcgs_scb<TB, TJ>(pass, j + 1, w != nullptr, &stage);
  if (scb == 0) return cudaErrorInvalidValue;
  // as many ring entries (and their two barriers) as the per-block limit holds
  static SmemLimit limit_of[2];
  static SmemOptIn opt_in[2];
  int limit = 0;
  cudaError_t e = pass == 1 ? smem_block_limit(k_dcgs_dots<TB, TJ, KMAX>, limit_of[0], &limit)
                            : smem_block_limit(k_dcgs_update<TB, TJ, KMAX>, limit_of[1], &limit);
  if (e != cudaSuccess) return e;
  int nst = limit / (stage + 16);
  if (nst > kDcgsMaxStages) nst = kDcgsMaxStages;
  if (nst < 2) return cudaErrorInvalidValue;               // two entries always fit on GB300 (kDcgsBudget)
  const size_t smem = (size_t)nst * stage + (size_t)nst * 16;
  e = pass == 1 ? smem_opt_in(k_dcgs_dots<TB, TJ, KMAX>, opt_in[0], limit)
                : smem_opt_in(k_dcgs_update<TB, TJ, KMAX>, opt_in[1], limit);
  if (e != cudaSuccess) return e;
  if (pass == 1)
    e = launch_maybe_pdl(pdl, k_dcgs_dots<TB, TJ, KMAX>, dim3(nsm), dim3(kStreamThreads + 32), smem, st, n,
                         (const TB*)V, j, (const TJ*)w, ctl, (double*)red.partials, red.counter, red.max_blocks, scb,
                         stage, nst, defer ? 1 : 0, err);
  else
    e = launch_maybe_pdl(pdl, k_dcgs_update<TB, TJ, KMAX>, dim3(nsm), dim3(kStreamThreads + 32), smem, st, n, (TB*)V,
                         j, (const TJ*)w, ctl, RedSite<A>{(A*)red.partials, red.counter, red.max_blocks},
                         defer ? (const double*)red.partials + (size_t)nsm * kMaxK : (const double*)nullptr, scb,
                         stage, nst, err);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// pass 1: dots of step j (w null: the last step of a cycle); pass 2: update of step j.
// defer (w not null, partials for at least 2 nsm blocks): the step runs at the start of
// the update pass instead of the end of the dots pass; both passes of a step take the same value.
template <class TB, class TJ>
static cudaError_t dcgs_dispatch(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                                 unsigned int* err, int nsm, cudaStream_t st, bool pdl, bool defer) {
  if (j < 8) return dcgs_launch_k<TB, TJ, 8>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  if (j < 16) return dcgs_launch_k<TB, TJ, 16>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  if (j < 24) return dcgs_launch_k<TB, TJ, 24>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  if (j < 32) return dcgs_launch_k<TB, TJ, 32>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  // buckets of eight up to 48: the slot loops are unrolled to KMAX, so a wide bucket spends issue
  // slots on predicated-off slots (and registers on their accumulators)
  if (j < 40) return dcgs_launch_k<TB, TJ, 40>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  if (j < 48) return dcgs_launch_k<TB, TJ, 48>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
  return dcgs_launch_k<TB, TJ, 64>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
}

}  // namespace jfnk
