// stencil_stage.cuh -- the Krylov product out = J(x) v (AD, Eq. 9) or the FD
// quotient (F(x + eps v) - F(x)) / eps (Eq. 7) with the rows of x and v
// staged in shared memory by bulk copies.
//
// The march form (stencil_impl.cuh) keeps one row of prefetch per warp in
// registers, so the bytes it has in flight are bounded by the register file
// (about 24 KB per SM at three blocks of eight warps), well short of what HBM3e
// needs to stream at full rate. Here each CTA owns one unit of the grid -- a
// strip of W columns (W = 8 warps x 32 lanes x one 16-byte vector, or the
// row length when shorter) by a band of R rows -- and a producer warp copies
// the band's rows j0 - 1 .. j1 of every field of x and v, each with a 16-byte
// halo on both sides (the wrapped or clamped columns beyond the strip), into
// a ring of shared-memory slots with cp.async.bulk, up to ~96 KB ahead of the
// consumers. Eight consumer warps evaluate row j from the slots of rows
// j - 1, j, j + 1 (one 16-byte vector of cells per thread, neighbours from the
// same slots) and release the slot of row j - 1. The per-cell residual is the
// one in pdes.cuh, on dual numbers (AD) or plain numbers (FD). Every wait is
// bounded by the global timer; on expiry the CTA records STREAM_TIMEOUT in the
// error word (StencilArgs::err) and stops after draining its copies.
// Included by stencil_impl.cuh after the definitions it uses (Comb, Row,
// VecOf, load_aux, fd_step, bp_index).
#pragma once

#include "stream.cuh"

namespace jfnk {

constexpr int kStageWarps = 8;                        // consumer warps (warp 0 produces)
constexpr int kStageThreads = 32 * (kStageWarps + 1);
constexpr int kStageMaxSlots = 24;
constexpr int kStageRingBytes3 = 64 * 1024;           // ring per CTA at three CTAs per SM ...
constexpr int kStageRingBytes2 = 96 * 1024;           // ... or at two, when 64 KB holds fewer than 6 slots
constexpr int kStageMinRows = 4;                      // shortest band (two halo rows per band)

// Launch plan of the staged sweep, computed on the host.
struct StagePlan {
  int W;            // strip width in cells (multiple of 16 bytes of T and of TV)
  int nstrips;      // strips per row
  int R;            // rows per band
  int nbands;
  int units;        // nstrips * nbands, taken by CTAs in order blockIdx.x, + gridDim.x, ...
  int slots;        // ring slots (one staged row of every field of x and v each)
  int slot_bytes;
  int offv;         // byte offset of the v rows inside a slot
  int grid;
  int smem;         // dynamic shared memory: slots and their full/empty barriers
  int per_sm;       // CTAs per SM the ring is sized for
};

// Position in the ring: slot index and the parity of its current fill,
// advanced without divisions.
struct RingPos {
  int slot;
  uint32_t phase;
  __device__ __forceinline__ void next(int slots) {
    if (++slot == slots) { slot = 0; phase ^= 1u; }
  }
};

template <class T, class TV, int NF>
inline bool stage_plan(const ProbDev& P, int nsm, StagePlan* g) {
  constexpr int HX = 16 / (int)sizeof(T), HV = 16 / (int)sizeof(TV), VEC = 16 / (int)sizeof(T);
  if (P.ny < 3 || P.nx % HX != 0 || P.nx % HV != 0) return false;
  const int wmax = kStageWarps * 32 * VEC;
  g->W = P.nx < wmax ? P.nx : wmax;
  g->nstrips = (P.nx + g->W - 1) / g->W;
  const int xrow = (g->W + 2 * HX) * (int)sizeof(T), vrow = (g->W + 2 * HV) * (int)sizeof(TV);
  g->offv = NF * xrow;
  g->slot_bytes = (NF * (xrow + vrow) + 127) / 128 * 128;
  g->per_sm = 3;
  g->slots = kStageRingBytes3 / g->slot_bytes;
  if (g->slots < 6) {
    g->per_sm = 2;
    g->slots = kStageRingBytes2 / g->slot_bytes;
  }
  if (g->slots > kStageMaxSlots) g->slots = kStageMaxSlots;
  if (g->slots < 4) return false;                     // three rows in use and one in flight at least
  const int ctas = g->per_sm * (nsm > 0 ? nsm : 1);
  int nb = (ctas + g->nstrips - 1) / g->nstrips;
  int R = (P.ny + nb - 1) / nb;
  if (R < kStageMinRows) R = kStageMinRows;
  g->R = R;
  g->nbands = (P.ny + R - 1) / R;
  g->units = g->nstrips * g->nbands;
  g->grid = g->units < ctas ? g->units : ctas;
  g->smem = g->slots * g->slot_bytes + g->slots * 16;
  return true;
}

// Rows of one unit as the producer and the consumers both walk them.
struct StageUnit {
  int col0, Wu, j0, j1;
};
__device__ __forceinline__ StageUnit stage_unit(const StagePlan& g, int u, int nx, int ny) {
  StageUnit s;
  const int strip = u % g.nstrips, band = u / g.nstrips;
  s.col0 = strip * g.W;
  s.Wu = nx - s.col0 < g.W ? nx - s.col0 : g.W;
  s.j0 = band * g.R;
  s.j1 = s.j0 + g.R < ny ? s.j0 + g.R : ny;
  return s;
}

// Copy k < 6 NF of ring row rj of unit su into the slot at st: field k / 6;
// x or v; the strip itself, its left or its right halo.
template <class T, class TV, int NF, int POL>
__device__ __forceinline__ void stage_copy(const ProbDev& P, const StagePlan& g, const StageUnit& su, int rj,
                                           const T* x, const TV* v, unsigned char* st, uint64_t* bar, int k) {
  constexpr int HX = 16 / (int)sizeof(T), HV = 16 / (int)sizeof(TV);
  const int nx = P.nx;
  const int f = k / 6, kind = k % 6;
  const bool isv = kind >= 3;
  const int part = kind % 3;
  const int H = isv ? HV : HX;
  const int es = isv ? (int)sizeof(TV) : (int)sizeof(T);
  const int Wrow = g.W + 2 * H;
  const char* base = isv ? (const char*)(v + (size_t)f * P.ncell + (size_t)rj * nx)
                         : (const char*)(x + (size_t)f * P.ncell + (size_t)rj * nx);
  unsigned char* dst = st + (isv ? g.offv : 0) + (size_t)f * Wrow * es;
  int c0, cnt, dpos;
  if (part == 0) {
    c0 = su.col0; cnt = su.Wu; dpos = H;
  } else if (part == 1) {   // the H columns before the strip
    c0 = su.col0 >= H ? su.col0 - H : (POL == BP_WRAP ? nx - H : 0);
    cnt = H; dpos = 0;
  } else {                  // the H columns after it
    c0 = su.col0 + su.Wu < nx ? su.col0 + su.Wu : (POL == BP_WRAP ? 0 : nx - H);
    cnt = H; dpos = H + su.Wu;
  }
  bulk_g2s(dst + (size_t)dpos * es, base + (size_t)c0 * es, (uint32_t)(cnt * es), bar);
}

// Before the grid dependency wait: the x copies of the first rows of the CTA's
// first unit su (as many as the empty ring holds; row q goes to slot q), with
// their bytes added to each slot's transaction count but no arrival, so no
// slot completes before stage_produce_unit adds the v copies and arrives.
// Returns the number of rows started.
template <class T, class TV, int NF, int POL>
__device__ __forceinline__ int stage_prefetch_x(const ProbDev& P, const StagePlan& g, const StageUnit& su,
                                                const T* x, unsigned char* sring, uint64_t* full) {
  constexpr int HX = 16 / (int)sizeof(T);
  const int lane = threadIdx.x & 31;
  const int rows = su.j1 - su.j0 + 2;
  const int pre = rows < g.slots ? rows : g.slots;
  const uint32_t xb = (uint32_t)NF * (su.Wu + 2 * HX) * (uint32_t)sizeof(T);
  for (int q = 0; q < pre; ++q) {
    const int rj = bp_index(su.j0 - 1 + q, P.ny, POL);
    if (lane == 0) mbar_expect_tx(&full[q], xb);
    __syncwarp();
    if (lane < 3 * NF)
      stage_copy<T, TV, NF, POL>(P, g, su, rj, x, (const TV*)nullptr, sring + (size_t)q * g.slot_bytes, &full[q],
                                 (lane / 3) * 6 + lane % 3);
    __syncwarp();
  }
  return pre;
}

// Producer: rows j0 - 1 .. j1 of unit u (wrapped or clamped in y) into the
// ring, row counter q continuing across units. Lane k < 6 NF issues copy k
// (stage_copy). The first xdone rows (the CTA's first unit only) had their x
// copies started by stage_prefetch_x: they take the v copies and the arrival,
// whatever the abort flag says, so that every started slot completes.
template <class T, class TV, int NF, int POL>
__device__ __forceinline__ bool stage_produce_unit(const ProbDev& P, const StagePlan& g, const StageUnit& su,
                                                   const T* x, const TV* v, unsigned char* sring, uint64_t* full,
                                                   uint64_t* empty, RingPos* pos, int* filled, unsigned int* err,
                                                   int* s_abort, int xdone) {
  constexpr int HX = 16 / (int)sizeof(T), HV = 16 / (int)sizeof(TV);
  const int lane = threadIdx.x & 31;
  const uint32_t xb = (uint32_t)NF * (su.Wu + 2 * HX) * (uint32_t)sizeof(T);
  const uint32_t vb = (uint32_t)NF * (su.Wu + 2 * HV) * (uint32_t)sizeof(TV);
  int q = 0;
  for (int r = su.j0 - 1; r <= su.j1; ++r, ++q, pos->next(g.slots), ++*filled) {
    const int slot = pos->slot;
    const bool started = q < xdone;
    if (!started) {
      // a slot's k-th refill waits for the k-th release (empty phase k - 1)
      if (*filled >= g.slots && !mbar_wait_bounded(&empty[slot], pos->phase ^ 1u, kWaitLimitNs)) {
        if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); *s_abort = 1; }
        return false;
      }
      if (*s_abort) return false;
    }
    const int rj = bp_index(r, P.ny, POL);
    unsigned char* st = sring + (size_t)slot * g.slot_bytes;
    if (lane == 0) mbar_arrive_expect_tx(&full[slot], started ? vb : xb + vb);
    __syncwarp();
    if (lane < 6 * NF && (!started || lane % 6 >= 3))
      stage_copy<T, TV, NF, POL>(P, g, su, rj, x, v, st, &full[slot], lane);
    __syncwarp();
  }
  return true;
}

template <class T, int VEC>
__device__ __forceinline__ void lds_vec(T (&r)[VEC], const T* p) {
  typedef typename VecOf<T, VEC>::type VT;
  const VT q = *(const VT*)p;
  const T* e = (const T*)&q;
#pragma unroll
  for (int k = 0; k < VEC; ++k) r[k] = e[k];
}
__device__ __forceinline__ void lds_vec(float (&r)[4], const __nv_bfloat16* p) {
  const uint2 q = *(const uint2*)p;
  const __nv_bfloat162* h = (const __nv_bfloat162*)&q;
  const float2 a = __bfloat1622float2(h[0]), b = __bfloat1622float2(h[1]);
  r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
}

template <class T, class S> __device__ __forceinline__ T stage_cvt(S x) { return (T)x; }
template <> __device__ __forceinline__ float stage_cvt<float, __nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

// One staged row of one field as a thread sees it (a Row of the march form):
// its VEC cells and the cells just west and east of them -- from the halo at
// the ends of the strip, or the cell itself beyond a clamped wall.
template <class T, int VEC, class TS, int POL>
__device__ __forceinline__ void srow_load(Row<T, VEC>& r, const TS* row, int cl, int col, int nx) {
  lds_vec(r.c, row + cl);
  const int wi = (POL == BP_CLAMP && col == 0) ? cl : cl - 1;
  const int ei = (POL == BP_CLAMP && col + VEC >= nx) ? cl + VEC - 1 : cl + VEC;
  r.we = stage_cvt<T>(row[wi]);
  r.ee = stage_cvt<T>(row[ei]);
}

template <class PDE, class T, class TV, int MODE>
__global__ void __launch_bounds__(kStageThreads, 3)
    k_jvp_stage(ProbDev P, StencilArgs a, StagePlan g) {
  typedef Comb<MODE, T> CB;
  typedef typename CB::V V;
  constexpr int NF = PDE::NF;
  constexpr int POL = PDE::POLICY;
  constexpr int VEC = 16 / (int)sizeof(T);
  constexpr int HX = 16 / (int)sizeof(T), HV = 16 / (int)sizeof(TV);
  unsigned int* err = a.err;
  extern __shared__ __align__(128) unsigned char sring[];
  uint64_t* full = (uint64_t*)(sring + (size_t)g.slots * g.slot_bytes);
  uint64_t* empty = full + g.slots;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nx = P.nx, ny = P.ny;
  if (tid == 0) {
    for (int q = 0; q < g.slots; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStageWarps);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  // Launched programmatically, the sweep follows a kernel that does not write
  // the state x (the update pass of a delayed-CGS2 step writes only the basis),
  // so the producer starts the x rows of its first unit while that kernel
  // finishes; v, the scale and the active flag are read after the wait. A
  // plain launch has nothing to overlap and fills its rows in one pass.
  int xpre = 0;
  if (warp == 0 && a.pdl)
    xpre = stage_prefetch_x<T, TV, NF, POL>(P, g, stage_unit(g, blockIdx.x, nx, ny), (const T*)a.x, sring, full);
  grid_dep_wait();      // the kernel that wrote v (and the active flag) has completed (programmatic launch)
  grid_dep_trigger();
  if (a.active && *a.active == 0) {
    // nothing to compute: complete the started slots and let their copies land before the CTA exits
    if (warp == 0 && lane == 0) {
      for (int q = 0; q < xpre; ++q) mbar_arrive(&full[q]);
      const uint64_t deadline = global_timer_ns() + kWaitLimitNs;
      for (int q = 0; q < xpre; ++q) mbar_wait_until(&full[q], 0u, deadline);
    }
    return;
  }
  const T s = a.vscale ? T(*a.vscale) : T(1);
  const T eps = fd_step<T, MODE>(a, s);
  const CB cb = make_comb<MODE, T>(0.0, s, eps);
  if (warp == 0) {
    RingPos pos{0, 0u};
    int filled = 0;
    for (int u = blockIdx.x; u < g.units; u += gridDim.x) {
      const StageUnit su = stage_unit(g, u, nx, ny);
      if (!stage_produce_unit<T, TV, NF, POL>(P, g, su, (const T*)a.x, (const TV*)a.v, sring, full, empty, &pos,
                                               &filled, err, &s_abort, u == (int)blockIdx.x ? xpre : 0))
        break;
    }
    if (s_abort && lane == 0) {   // drain the copies still in flight before the CTA exits
      const uint64_t deadline = global_timer_ns() + kWaitLimitNs;
      for (long long r = (filled - g.slots > 0 ? filled - g.slots : 0); r < filled; ++r)
        mbar_wait_until(&full[r % g.slots], (uint32_t)((r / g.slots) & 1), deadline);
    }
    return;
  }
  const int cl = ((warp - 1) * 32 + lane) * VEC;   // this thread's first column inside the strip
  const T thdt = T(P.thdt);
  RingPos ps{0, 0u};                               // slot of row j - 1 (rows j, j + 1 follow it)
  for (int u = blockIdx.x; u < g.units; u += gridDim.x) {
    const StageUnit su = stage_unit(g, u, nx, ny);
    const bool act = cl < su.Wu;
    const int col = su.col0 + cl;
    const int rows = su.j1 - su.j0;            // rows of the unit; it fills rows + 2 slots
    RingPos pc = ps;
    pc.next(g.slots);
    RingPos pn = pc;
    pn.next(g.slots);
    bool ok = mbar_wait_bounded(&full[ps.slot], ps.phase, kWaitLimitNs) &&
              mbar_wait_bounded(&full[pc.slot], pc.phase, kWaitLimitNs);
    for (int jj = 0; jj < rows && ok; ++jj) {
      ok = mbar_wait_bounded(&full[pn.slot], pn.phase, kWaitLimitNs);
      if (!ok) break;
      const int j = su.j0 + jj;
      if (act) {
        const unsigned char* ss = sring + (size_t)ps.slot * g.slot_bytes;
        const unsigned char* sc = sring + (size_t)pc.slot * g.slot_bytes;
        const unsigned char* sn = sring + (size_t)pn.slot * g.slot_bytes;
        Row<T, VEC> xs[NF], xc[NF], xn[NF], vs[NF], vc[NF], vn[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const size_t ox = (size_t)f * (g.W + 2 * HX) * sizeof(T) + HX * sizeof(T);
          const size_t ov = (size_t)g.offv + (size_t)f * (g.W + 2 * HV) * sizeof(TV) + HV * sizeof(TV);
          srow_load<T, VEC, T, POL>(xc[f], (const T*)(sc + ox), cl, col, nx);
          srow_load<T, VEC, TV, POL>(vc[f], (const TV*)(sc + ov), cl, col, nx);
          if (PDE::DIAG) {
            srow_load<T, VEC, T, POL>(xs[f], (const T*)(ss + ox), cl, col, nx);
            srow_load<T, VEC, T, POL>(xn[f], (const T*)(sn + ox), cl, col, nx);
            srow_load<T, VEC, TV, POL>(vs[f], (const TV*)(ss + ov), cl, col, nx);
            srow_load<T, VEC, TV, POL>(vn[f], (const TV*)(sn + ov), cl, col, nx);
          } else {
            lds_vec(xs[f].c, (const T*)(ss + ox) + cl);
            lds_vec(xn[f].c, (const T*)(sn + ox) + cl);
            lds_vec(vs[f].c, (const TV*)(ss + ov) + cl);
            lds_vec(vn[f].c, (const TV*)(sn + ov) + cl);
          }
        }
        const long long crow = (long long)j * nx;
        T jv[NF][VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          const int i = col + k;
          Nb<V, NF> nb;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            nb.c[f] = cb(xc[f].c[k], vc[f].c[k]);
            nb.w[f] = cb(west_of(xc[f], k), west_of(vc[f], k));
            nb.e[f] = cb(east_of(xc[f], k), east_of(vc[f], k));
            nb.n[f] = cb(xn[f].c[k], vn[f].c[k]);
            nb.s[f] = cb(xs[f].c[k], vs[f].c[k]);
            if (PDE::DIAG) {
              nb.nw[f] = cb(west_of(xn[f], k), west_of(vn[f], k));
              nb.ne[f] = cb(east_of(xn[f], k), east_of(vn[f], k));
              nb.sw[f] = cb(west_of(xs[f], k), west_of(vs[f], k));
              nb.se[f] = cb(east_of(xs[f], k), east_of(vs[f], k));
            }
          }
          const CellAux<T> aux = load_aux<PDE, T>(P, crow + i);
          V M[NF], G[NF];
          PDE::template cell<T, V>(P, i, j, nb, aux, M, G);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            if constexpr (MODE == SM_AD) {
              jv[f][k] = P.bvp ? G[f].d : M[f].d - thdt * G[f].d;
            } else {
              jv[f][k] = P.bvp ? primal(G[f]) : primal(M[f]) - thdt * primal(G[f]);
            }
          }
        }
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
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[ps.slot]);
      ps = pc;
      pc = pn;
      pn.next(g.slots);
    }
    if (!ok) {
      if (lane == 0) { atomicExch(err, (unsigned)STREAM_TIMEOUT); s_abort = 1; }
      return;
    }
    __syncwarp();
    if (lane == 0) {   // the unit's last two rows are no longer needed
      mbar_arrive(&empty[ps.slot]);
      mbar_arrive(&empty[pc.slot]);
    }
    ps = pn;           // the next unit's first row follows them
  }
}

}  // namespace jfnk
