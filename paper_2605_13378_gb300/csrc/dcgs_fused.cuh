// dcgs_fused.cuh -- one pass per delayed-CGS2 Arnoldi step with the AD
// Jacobian-vector product inside it: the update of step j, the JVP of the
// new candidate u_{j+1} and the dots of step j + 1 share one read of the
// basis (FP32 basis and JVP: the mixed-precision and FP32 forms).
//
// The two-pass form (dcgs_impl.cuh) reads basis slots 0..j twice per step:
// for the dots Q^T [u_j, w] and for the update that forms q_j and u_{j+1},
// with the JVP of u_{j+1} in between. The JVP of a cell needs u_{j+1} only on
// the cell and its four face neighbours, so a CTA that forms u_{j+1} row by
// row over a strip of columns can apply the Jacobian one row behind and take
// that row's dots while its basis row is still in shared memory. Each CTA
// owns a contiguous run of (column strip, row) pairs and also forms u_{j+1}
// on the halo just outside its run (one row above and below, one column left
// and right); the halo costs a few percent of extra reads and keeps CTAs
// independent of each other.
//
// Buffers (no buffer is both read and written by the pass):
//   V      basis; slots 0..j-1 hold q_0..q_{j-1}, slot j receives q_j
//   U_in   u_j;  U_out receives u_{j+1}
//   W_in   w_j = J u_j unscaled, used as wmul w_j with wmul = sigma_j (at
//          j = 0 it holds J(sigma_0 u_0) and wmul = 1)
//   W_out  receives J u_{j+1} unscaled
//   X      the state in FP32 (the JVP's linearisation point)
// Block partials: q_i . u_{j+1} and q_i . J u_{j+1} for i <= j, then
// u_{j+1} . u_{j+1} and u_{j+1} . J u_{j+1}. The last CTA sets
// sigma_{j+1} = 1 / ||u_{j+1}|| (dcgs_after_update), scales the J u dots by
// it (J (sigma u) = sigma J u) and runs dcgs_step for step j + 1.
// Requires nx % 4 == 0 (16-byte row starts for the bulk copies), ny >= 3.
//
// Shared memory holds three rows of every vector involved plus the rows in
// flight, so a strip is at most 252 columns and each consumer thread takes
// one column: per basis slot and element the pass issues two shared loads
// and four FMAs, against one 16-byte load per four elements in the
// streaming passes. On GB300 that makes it issue- and latency-bound (about
// 1.4 TB/s of its own algorithmic bytes on the 2048^2 Allen-Cahn workload,
// against 3.8 and 5.5 TB/s for the dots and update passes), so it is
// selected only on request (opts.ortho = JFNK_DCGS2_FUSED).
#pragma once

#include "dcgs_impl.cuh"

namespace jfnk {

constexpr int kFusedMaxStages = 16;
constexpr int kFusedBudget = 200 * 1024;   // dynamic shared memory: stages + row rings + barriers

struct FusedGeom {
  int tiles_x;       // column strips
  int sw;            // elements per (vector, field) row in a stage
  int nvec;          // vectors per stage: slots 0..j-1, U_in, W_in (and X)
  int nstage, stage_bytes, ring_bytes, smem;
  int grid;
  long long total;   // tiles_x * ny (strip, row) pairs
};

struct FusedArgs {
  long long n, ncell;
  int nx, ny, j, has_w, wmul_one;
  float* V;
  const float* U_in; float* U_out;
  const float* W_in; float* W_out;
  const float* X;
  GmresCtl* ctl;
  double* partials; unsigned int* counter; int cap;
  unsigned int* err;
  FusedGeom g;
};

// Shared-memory plan for step j: the widest strip (252, 124 or 60 columns)
// whose stage leaves room for at least five stages (rows k - 2 .. k resident,
// two in flight); false when none does. Strips are at most 252 columns, so a
// row of a strip with its two halo columns fits the 256 consumer threads.
inline bool fused_geom(int nx, int ny, int nf, int j, bool has_w, int nsm, FusedGeom* G) {
  if (nx % 4 != 0 || ny < 3 || nx < 4) return false;
  const int widths[3] = {252, 124, 60};
  for (int wi = 0; wi < 3; ++wi) {
    const int tx = (nx + widths[wi] - 1) / widths[wi];
    const int maxw = (nx + tx - 1) / tx;
    const int sw = (maxw + 16 + 3) / 4 * 4;
    const int nvec = j + 2 + (has_w ? 1 : 0);
    const int stage = (nvec * nf * sw * 4 + 127) / 128 * 128;
    const int ring = 12 * nf * sw * 4;
    int S = (kFusedBudget - ring - 2 * kFusedMaxStages * 8) / stage;
    if (S > kFusedMaxStages) S = kFusedMaxStages;
    if (S < 5) continue;                               // three rows resident, two in flight
    G->tiles_x = tx;
    G->sw = sw;
    G->nvec = nvec;
    G->nstage = S;
    G->stage_bytes = stage;
    G->ring_bytes = ring;
    G->smem = S * stage + ring + 2 * kFusedMaxStages * 8;
    G->total = (long long)tx * ny;
    long long grid = nsm > 0 ? nsm : 1;
    const long long by_rows = G->total / 16;          // at least 16 rows per CTA: halo rows stay cheap
    if (grid > by_rows) grid = by_rows > 0 ? by_rows : 1;
    G->grid = (int)grid;
    return true;
  }
  return false;
}

// Named barrier 1 over the consumer warps with an OR of v: every consumer
// gets the same answer, so they leave the row loop together.
__device__ __forceinline__ bool fz_bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kStreamThreads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ int fz_bp(int i, int n, int policy) {
  if (i < 0) return policy == BP_WRAP ? i + n : 0;
  if (i >= n) return policy == BP_WRAP ? i - n : n - 1;
  return i;
}

// Shared-memory offset of column c in a strip row whose main chunk starts at
// column a0: wrap halos come from the 4-element blocks at sw - 8 (columns
// nx - 4 .. nx - 1) and sw - 4 (columns 0 .. 3); clamp halos repeat the wall.
__device__ __forceinline__ int fz_off(int c, int a0, int nx, int sw, int policy) {
  if (c < 0) return policy == BP_WRAP ? sw - 8 + 3 : -a0;
  if (c >= nx) return policy == BP_WRAP ? sw - 4 : nx - 1 - a0;
  return c - a0;
}

// The CTA's run of (strip, row) pairs, cut into segments of one strip each.
struct FzRun {
  long long L, L1;
  int ny, tiles_x, nx;
  __device__ bool next(int* s, int* c0, int* c1, int* ra, int* rb) {
    if (L >= L1) return false;
    *s = (int)(L / ny);
    *ra = (int)(L - (long long)(*s) * ny);
    const long long left = L1 - L;
    *rb = (int)((long long)(*ra) + left < ny ? (long long)(*ra) + left : ny);
    *c0 = (int)((long long)(*s) * nx / tiles_x);
    *c1 = (int)((long long)(*s + 1) * nx / tiles_x);
    L += *rb - *ra;
    return true;
  }
};

template <class PDE, int KMAX>
__global__ void __launch_bounds__(kStreamThreads + 32, 1) k_dcgs_fused(FusedArgs a, ProbDev P) {
  constexpr int NF = PDE::NF;
  constexpr int NC = kStreamThreads;                 // consumer threads
  constexpr int NA = KMAX;                           // accumulators of slots 0..j-1 (j < KMAX)
  if (!a.ctl->active || (int)gridDim.x > a.cap) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const FusedGeom& G = a.g;
  const int S = G.nstage, sw = G.sw, nx = a.nx, ny = a.ny, j = a.j;
  const bool has_w = a.has_w != 0;
  float* uring = (float*)(smem + (size_t)S * G.stage_bytes);     // u_{j+1}: [4][NF][sw]
  float* xring = uring + 4 * NF * sw;                              // x: [3][NF][sw], then J u: [2][NF][sw]
  float* qring = xring + 5 * NF * sw;                              // q_j: [3][NF][sw]
  uint64_t* full = (uint64_t*)(smem + (size_t)S * G.stage_bytes + G.ring_bytes);
  uint64_t* empty = full + kFusedMaxStages;
  __shared__ float ca[kMaxM + 1], cc[kMaxM + 1];
  __shared__ float s_gam, s_cj, s_invr, s_wmul;
  __shared__ int s_abort;
  __shared__ unsigned int s_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], NC / 32);
    }
    fence_mbar_init();
    s_abort = 0;
    s_gam = (float)a.ctl->dgamma;
    s_cj = (float)a.ctl->dc[j];
    s_invr = (float)a.ctl->dinvr;
    s_wmul = a.wmul_one ? 1.0f : (float)a.ctl->scale[j];
  }
  for (int t = tid; t < j; t += blockDim.x) {
    ca[t] = (float)a.ctl->da[t];
    cc[t] = (float)a.ctl->dc[t];
  }
  __syncthreads();
  const long long L0 = (long long)blockIdx.x * G.total / gridDim.x;
  const long long L1 = (long long)(blockIdx.x + 1) * G.total / gridDim.x;
  const long long N = a.n, nc = a.ncell;
  float au[NA], aw[NA];
#pragma unroll
  for (int t = 0; t < NA; ++t) { au[t] = 0.0f; aw[t] = 0.0f; }
  float qu = 0.0f, qw = 0.0f, uu = 0.0f, uw = 0.0f;   // slot j (q_j) and u_{j+1} itself

  if (warp == 0) {
    // ---- producer: one stage per row step, rows ra - 1 .. rb of each segment
    FzRun run{L0, L1, ny, G.tiles_x, nx};
    int s, c0, c1, ra, rb;
    int idx = 0;
    bool ok = true;
    while (ok && run.next(&s, &c0, &c1, &ra, &rb)) {
      const int a0 = (c0 - 1 > 0 ? c0 - 1 : 0) / 4 * 4;
      const int a1 = (c1 + 1 + 3) / 4 * 4 < nx ? (c1 + 1 + 3) / 4 * 4 : nx;
      const uint32_t len = (uint32_t)(a1 - a0) * 4u;
      const bool needL = PDE::POLICY == BP_WRAP && c0 == 0, needR = PDE::POLICY == BP_WRAP && c1 == nx;
      const uint32_t per = len + (needL ? 16u : 0u) + (needR ? 16u : 0u);
      for (int k = ra - 1; k <= rb; ++k, ++idx) {
        const int sidx = idx % S;
        int good = 1;
        if (lane == 0) {
          if (idx >= S && !mbar_wait_bounded(&empty[sidx], (uint32_t)(((idx / S) - 1) & 1), kWaitLimitNs)) {
            atomicExch(a.err, (unsigned)STREAM_TIMEOUT);
            s_abort = 1;
          }
          good = *(volatile int*)&s_abort == 0;
        }
        good = __shfl_sync(0xffffffffu, good, 0);    // one decision for the whole warp
        if (!good) { ok = false; break; }
        const int rr = fz_bp(k, ny, PDE::POLICY);
        unsigned char* st = smem + (size_t)sidx * G.stage_bytes;
        if (lane == 0) mbar_arrive_expect_tx(&full[sidx], (uint32_t)(G.nvec * NF) * per);
        __syncwarp();
        for (int vf = lane; vf < G.nvec * NF; vf += 32) {
          const int v = vf / NF, f = vf - v * NF;
          const float* src;
          if (v < j) src = a.V + (long long)v * N;
          else if (v == j) src = a.U_in;
          else if (v == j + 1) src = a.W_in;
          else src = a.X;
          src += (long long)f * nc + (long long)rr * nx;
          float* dst = (float*)(st + (size_t)vf * sw * 4);
          bulk_g2s(dst, src + a0, len, &full[sidx]);
          if (needL) bulk_g2s(dst + sw - 8, src + nx - 4, 16u, &full[sidx]);
          if (needR) bulk_g2s(dst + sw - 4, src, 16u, &full[sidx]);
        }
        __syncwarp();
      }
    }
    if (!ok && lane == 0) {
      // drain the copies still in flight (bounded) before the CTA leaves
      const uint64_t deadline = global_timer_ns() + kWaitLimitNs;
      for (int q = (idx - S > 0 ? idx - S : 0); q < idx; ++q)
        mbar_wait_until(&full[q % S], (uint32_t)((q / S) & 1), deadline);
    }
  } else {
    // ---- consumers, one column position each. Step k (rows ra - 1 .. rb,
    // then one trailing step): one loop over the basis slots forms q_j and
    // u_{j+1} on row k and accumulates the dots of row k - 2, whose J u_{j+1}
    // was applied in the previous step; then the Jacobian is applied on row
    // k - 1 (its north neighbour, row k, now exists).
    const int ct = tid - 32;
    const float gam = s_gam, cj = s_cj, invr = s_invr, wmul = s_wmul;
    const float thdt = (float)P.thdt;
    const int vs = NF * sw;                         // stage stride between basis slots
    FzRun run{L0, L1, ny, G.tiles_x, nx};
    int s, c0, c1, ra, rb;
    int idx = 0;
    bool ok = true;
    while (ok && run.next(&s, &c0, &c1, &ra, &rb)) {
      const int a0 = (c0 - 1 > 0 ? c0 - 1 : 0) / 4 * 4;
      const int W2 = c1 - c0 + 2;                   // positions: columns c0 - 1 .. c1
      const int p = ct;
      const bool act = p < W2, inner = p >= 1 && p <= W2 - 2;
      const int c = c0 - 1 + p;
      const int off = act ? fz_off(c, a0, nx, sw, PDE::POLICY) : 0;
      const int base = idx;                          // stage index of row ra - 1
      const int nrow = rb - ra + 2;                  // rows with a stage: ra - 1 .. rb
      for (int ls = 0; ls <= nrow; ++ls) {           // ls = nrow: the trailing step
        const int k = ra - 1 + ls;
        const bool load = ls < nrow;
        const bool halo = ls == 0 || ls == nrow - 1;
        const bool dots = ls >= 3;                   // dots of row k - 2 (interior rows ra .. rb - 1)
        const int sk = base + ls, sd = base + ls - 2;
        if (!load && !dots) continue;                // a one-row segment: nothing trails (uniform across consumers)
        if (load && !mbar_wait_bounded(&full[sk % S], (uint32_t)((sk / S) & 1), kWaitLimitNs) && lane == 0) {
          // recorded; the step is computed from whatever the stage holds (in-bounds reads,
          // result discarded) and every consumer leaves the loop together at its end
          atomicExch(a.err, (unsigned)STREAM_TIMEOUT);
          s_abort = 1;
        }
        const float* stk = (const float*)(smem + (size_t)((load ? sk : sd) % S) * G.stage_bytes);
        const float* std_ = (const float*)(smem + (size_t)((dots ? sd : sk) % S) * G.stage_bytes);
        const int rr = fz_bp(k, ny, PDE::POLICY);
        if (act) {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const float u = stk[(j * NF + f) * sw + off];
            const float w = stk[((j + 1) * NF + f) * sw + off] * wmul;
            float q = gam * u, y = w;
            const bool dm = dots && inner;
            const float ud = dm ? uring[(((ls - 2) & 3) * NF + f) * sw + p] : 0.0f;
            const float vd = dm ? xring[(3 * NF + ((ls - 2) & 1) * NF + f) * sw + p] : 0.0f;   // J u, row k - 2
            const float* pk = stk + f * sw + off;
            const float* pd = std_ + f * sw + off;
#pragma unroll
            for (int t = 0; t < KMAX; ++t) {
              if (t >= j) break;                     // registers need static indices: unrolled, left early
              const float qa = pk[t * vs], qb = pd[t * vs];
              q -= ca[t] * qa;
              y -= cc[t] * qa;
              au[t] += qb * ud;
              aw[t] += qb * vd;
            }
            if (dm) {
              const float qj = qring[((ls - 2) % 3 * NF + f) * sw + p];
              qu += qj * ud;
              qw += qj * vd;
              uu += ud * ud;
              uw += ud * vd;
            }
            if (load) {
              y = (y - cj * q) * invr;
              uring[((ls & 3) * NF + f) * sw + p] = y;
              qring[(ls % 3 * NF + f) * sw + p] = q;
              if (has_w) xring[(ls % 3 * NF + f) * sw + p] = stk[((j + 2) * NF + f) * sw + off];
              if (!halo && inner) {
                const long long g = (long long)f * nc + (long long)rr * nx + c;
                a.V[(long long)j * N + g] = q;
                a.U_out[g] = y;
              }
            }
          }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
        if (has_w && ls >= 2 && load && inner) {
          // J u_{j+1} on row r = k - 1 from rows k - 2, k - 1, k of u_{j+1} and x
          const int r = k - 1;                       // interior row: no wrap
          const int us = (ls - 2) & 3, uc = (ls - 1) & 3, un = ls & 3;
          const int xs = (ls - 2) % 3, xc = (ls - 1) % 3, xn = ls % 3;
          Nb<Dual<float>, NF> qn;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            qn.c[f] = Dual<float>(xring[(xc * NF + f) * sw + p], uring[(uc * NF + f) * sw + p]);
            qn.e[f] = Dual<float>(xring[(xc * NF + f) * sw + p + 1], uring[(uc * NF + f) * sw + p + 1]);
            qn.w[f] = Dual<float>(xring[(xc * NF + f) * sw + p - 1], uring[(uc * NF + f) * sw + p - 1]);
            qn.n[f] = Dual<float>(xring[(xn * NF + f) * sw + p], uring[(un * NF + f) * sw + p]);
            qn.s[f] = Dual<float>(xring[(xs * NF + f) * sw + p], uring[(us * NF + f) * sw + p]);
          }
          CellAux<float> aux;
          aux.eps = 1.0f; aux.fr = 0.0f; aux.fi = 0.0f; aux.gr = 0.0f; aux.gi = 0.0f;
          if constexpr (PDE::AUX) {
            const float* ep = P.eps32;
            if (ep) aux.eps = ep[(long long)r * nx + c];
          }
          Dual<float> M[NF], Gd[NF];
          PDE::template cell<float, Dual<float>>(P, c, r, qn, aux, M, Gd);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const float jv = P.bvp ? Gd[f].d : M[f].d - thdt * Gd[f].d;
            xring[(3 * NF + ((ls - 1) & 1) * NF + f) * sw + p] = jv;
            a.W_out[(long long)f * nc + (long long)r * nx + c] = jv;
          }
        }
        const bool stop = fz_bar_or(*(volatile int*)&s_abort != 0);
        if (lane == 0) {
          if (load && halo) mbar_arrive(&empty[sk % S]);
          if (dots) mbar_arrive(&empty[sd % S]);
        }
        if (stop) { ok = false; break; }
      }
      idx = base + nrow;
    }
  }
  __syncthreads();
  if (s_abort) return;
  // ---- block partials: warp butterflies, then the consumer warps in order
  const int nval = 2 * (j + 2);
  __shared__ double red[kStreamThreads / 32][2 * (NA + 2)];
  if (warp >= 1) {
#pragma unroll
    for (int t = 0; t < NA; ++t) {
      if (t < j) {
        const float su = warp_sum(au[t]), sv = warp_sum(aw[t]);
        if (lane == 0) { red[warp - 1][2 * t] = (double)su; red[warp - 1][2 * t + 1] = (double)sv; }
      }
    }
    const float s0 = warp_sum(qu), s1 = warp_sum(qw), s2 = warp_sum(uu), s3 = warp_sum(uw);
    if (lane == 0) {
      red[warp - 1][2 * j] = (double)s0;
      red[warp - 1][2 * j + 1] = (double)s1;
      red[warp - 1][2 * j + 2] = (double)s2;
      red[warp - 1][2 * j + 3] = (double)s3;
    }
  }
  __syncthreads();
  for (int v = tid; v < nval; v += blockDim.x) {
    double sum = 0.0;
    for (int q = 0; q < kStreamThreads / 32; ++q) sum += red[q][v];
    a.partials[(size_t)blockIdx.x * kMaxK + v] = sum;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // ---- last CTA: the step's scalar work, as in the dots pass, for step j + 1
  const int jj = j + 1;
  __shared__ double Sd[2 * (kMaxM + 1)];
  __shared__ double sh[5 * (kMaxM + 1)];
  __shared__ double s_ctl[4];
  __shared__ int s_m, s_active, s_its;
  const int GB = (int)gridDim.x;
  const size_t ringb = (size_t)S * G.stage_bytes;
  const bool staged = ((size_t)GB * nval + (size_t)jj * (kMaxM + 1)) * sizeof(double) <= ringb;
  double* hs = (double*)smem;
  double* pr = hs + (size_t)jj * (kMaxM + 1);
  for (int e0 = tid; staged && e0 < GB * nval; e0 += 8 * (int)blockDim.x) {
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * (int)blockDim.x;
      v[q] = e < GB * nval ? __ldcg(&a.partials[(size_t)(e / nval) * kMaxK + (e % nval)]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * (int)blockDim.x;
      if (e < GB * nval) pr[e] = v[q];
    }
  }
  __syncthreads();
  for (int v = warp; v < nval; v += (int)(blockDim.x >> 5)) {
    double sum;
    if (staged) {
      sum = 0.0;
      for (int b = lane; b < GB; b += 32) sum += pr[(size_t)b * nval + v];
    } else {
      sum = lane_strided_sum(a.partials + v, kMaxK, GB, lane);
    }
    sum = warp_sum(sum);
    if (lane == 0) Sd[v] = sum;
  }
  __syncthreads();
  if (tid == 0) {
    dcgs_after_update(a.ctl, j, Sd[2 * jj]);         // scale[j] = 1, sigma_{j+1} = 1 / ||u_{j+1}||
    s_ctl[0] = a.ctl->scale[jj];
    s_ctl[3] = 1.0 / s_ctl[0];
    s_ctl[1] = a.ctl->g[j];
    s_ctl[2] = a.ctl->target;
    s_m = a.ctl->m;
    s_active = a.ctl->active;
    s_its = a.ctl->its;
  }
  __syncthreads();
  if (!s_active) {
    if (tid == 0) *a.counter = 0u;
    return;
  }
  const double sigma = s_ctl[0];
  for (int i = tid; i <= jj; i += blockDim.x) Sd[2 * i + 1] *= sigma;   // dots with J (sigma u_{j+1})
  dcgs_stage(a.ctl, jj, sh, hs);
  __syncthreads();
  dcgs_step(a.ctl, jj, Sd, has_w, sh, hs, sigma, s_ctl[3], s_ctl[1], s_ctl[2], s_m, s_active, s_its);
  __syncthreads();
  if (tid == 0) *a.counter = 0u;
}

template <class PDE, int KMAX>
static cudaError_t dcgs_fused_k(const FusedArgs& a, const ProbDev& P, cudaStream_t st) {
  static SmemOptIn opt_in;
  cudaError_t e = smem_opt_in(k_dcgs_fused<PDE, KMAX>, opt_in, kFusedBudget);
  if (e != cudaSuccess) return e;
  k_dcgs_fused<PDE, KMAX><<<a.g.grid, kStreamThreads + 32, a.g.smem, st>>>(a, P);
  return cudaGetLastError();
}

// accumulator buckets of 8: the unrolled dots loop leaves at t = j
template <class PDE>
static cudaError_t dcgs_fused_dispatch(const FusedArgs& a, const ProbDev& P, cudaStream_t st) {
  switch (a.j >> 3) {
    case 0: return dcgs_fused_k<PDE, 8>(a, P, st);
    case 1: return dcgs_fused_k<PDE, 16>(a, P, st);
    case 2: return dcgs_fused_k<PDE, 24>(a, P, st);
    case 3: return dcgs_fused_k<PDE, 32>(a, P, st);
    case 4: return dcgs_fused_k<PDE, 40>(a, P, st);
    case 5: return dcgs_fused_k<PDE, 48>(a, P, st);
    case 6: return dcgs_fused_k<PDE, 56>(a, P, st);
    default: return dcgs_fused_k<PDE, 64>(a, P, st);
  }
}

cudaError_t dcgs_fused_allen_cahn(const FusedArgs& a, const ProbDev& P, cudaStream_t st);
cudaError_t dcgs_fused_maxwell(const FusedArgs& a, const ProbDev& P, cudaStream_t st);
cudaError_t dcgs_fused_burgers2d(const FusedArgs& a, const ProbDev& P, cudaStream_t st);

}  // namespace jfnk
