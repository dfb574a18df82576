// common.cuh -- shared device helpers of libjfnk: the forward-mode dual
// number, launch geometry and deterministic block/grid reductions.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace jfnk {

// ---------------------------------------------------------------------------
// Forward-mode AD scalar (Eq. 9): a value and its directional derivative.
// Every operation carries the derivative by the chain rule, so evaluating the
// residual on Dual<T>(x, v) yields F(x) in .v and J(x) v in .d in one sweep.
// ---------------------------------------------------------------------------
template <class T>
struct Dual {
  T v, d;
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(T a, T b) : v(a), d(b) {}
  __device__ __forceinline__ explicit Dual(T a) : v(a), d(T(0)) {}
};

template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T s) { return Dual<T>(a.v + s, a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator+(T s, Dual<T> a) { return Dual<T>(a.v + s, a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T s) { return Dual<T>(a.v - s, a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator-(T s, Dual<T> a) { return Dual<T>(s - a.v, -a.d); }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T s) { return Dual<T>(a.v * s, a.d * s); }
template <class T> __device__ __forceinline__ Dual<T> operator*(T s, Dual<T> a) { return Dual<T>(a.v * s, a.d * s); }
template <class T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, T s) { return Dual<T>(a.v / s, a.d / s); }
// (a/b)' = (a' - (a/b) b') / b
template <class T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T q = a.v / b.v;
  return Dual<T>(q, (a.d - q * b.d) / b.v);
}
template <class T> __device__ __forceinline__ Dual<T> operator/(T s, Dual<T> b) {
  T q = s / b.v;
  return Dual<T>(q, -q * b.d / b.v);
}
// sqrt(a)' = a' / (2 sqrt(a)); only called on arguments bounded away from 0
template <class T> __device__ __forceinline__ Dual<T> dsqrt(Dual<T> a) {
  T r = sqrt(a.v);
  return Dual<T>(r, a.d / (T(2) * r));
}
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }

// Primal value of a plain or dual scalar (branches test the value only).
template <class T> __device__ __forceinline__ T primal(Dual<T> a) { return a.v; }
__device__ __forceinline__ double primal(double a) { return a; }
__device__ __forceinline__ float primal(float a) { return a; }

template <class V> struct scalar_of { typedef V type; };
template <class T> struct scalar_of<Dual<T> > { typedef T type; };

// ---------------------------------------------------------------------------
// Storage conversions (FP64, FP32 and BF16 vectors).
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ float to_f(T x) { return (float)x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <class T> __device__ __forceinline__ double to_d(T x) { return (double)x; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <class T> struct store_as {
  template <class S> __device__ __forceinline__ static T cvt(S x) { return (T)x; }
};
template <> struct store_as<__nv_bfloat16> {
  template <class S> __device__ __forceinline__ static __nv_bfloat16 cvt(S x) { return __float2bfloat16((float)x); }
};
// Arithmetic type for a storage type: BF16 is computed in FP32.
template <class T> struct arith_of { typedef T type; };
template <> struct arith_of<__nv_bfloat16> { typedef float type; };

// ---------------------------------------------------------------------------
// Launch geometry for flat vector kernels. The grid depends only on the
// vector length, so every reduction over a vector of length n always uses
// the same partition and the same summation tree, whatever else runs.
// ---------------------------------------------------------------------------
constexpr int kVecThreads = 256;
constexpr int kMaxVecBlocks = 608;          // 4 blocks per SM on 152 SMs
constexpr int kMaxK = 136;                   // reductions of up to kMaxK values per launch

inline int vec_blocks(long long n) {
  long long b = (n + kVecThreads * 4 - 1) / (kVecThreads * 4);
  if (b < 1) b = 1;
  if (b > kMaxVecBlocks) b = kMaxVecBlocks;
  return (int)b;
}

// Warp sum by a fixed butterfly (deterministic).
template <class A> __device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Float-float numbers: hi + lo with |lo| <= ulp(hi) / 2, about 48 significant
// bits carried in FP32 arithmetic. Sums use Knuth's TwoSum, so adding n FP32
// values keeps the error near n 2^-48 of their magnitude; on GB300 FP32 adds
// run at 64 times the FP64 rate. Rounded intrinsics keep the compiler from
// reassociating the error terms.
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, e);
  return FF{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
// Butterfly over the warp; lane 0's result is the one used (the addition is
// not bitwise symmetric in its operands).
__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const FF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, w);
  }
  return v;
}
// A float-float value stored in (and read from) an 8-byte double slot.
__device__ __forceinline__ void ff_store(double* p, FF v) { *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo); }
__device__ __forceinline__ FF ff_load(const double* p) { const float2 f = *reinterpret_cast<const float2*>(p); return FF{f.x, f.y}; }

// sum over b = lane, lane + 32, ... < n of p[b * stride], added in that
// order; the loads are issued eight at a time (partials written by other
// blocks, read through L2) so the sum costs about one L2 round trip per 256
// entries instead of one per eight.
template <class A>
__device__ __forceinline__ A lane_strided_sum(const A* p, size_t stride, int n, int lane) {
  A s = A(0);
  for (int b0 = 0; b0 < n; b0 += 256) {
    A v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = b0 + lane + 32 * q;
      v[q] = b < n ? __ldcg(p + (size_t)b * stride) : A(0);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (b0 + lane + 32 * q < n) s += v[q];
  }
  return s;
}

// Workspace of one reduction site: per-block partials and an arrival counter
// that the last block resets to zero.
template <class A>
struct RedSite {
  A* partials;            // [cap][kMaxK]
  unsigned int* counter;  // one word, zero between launches
  int cap;                // capacity of partials in blocks
};

// Block-level reduction of k values per thread (k <= KMAX, same k in all
// threads), written to partials[blockLinear * kMaxK + t]. Then the last
// block to arrive sums the partials of all nblocks blocks in block order and
// calls fin(t, sum) once for each t < k (from lane 0 of the warp that owns
// t). Returns true in every thread of the last block, after a block barrier,
// so that what fin wrote to global memory is visible to the whole block.
// smem must hold (blockDim/32) * KMAX values of A.
template <class A, int KMAX, class Fin>
__device__ __forceinline__ bool grid_reduce(A (&vals)[KMAX], int k, RedSite<A> site, int nblocks,
                                            int blockLinear, A* smem, Fin fin) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  if (nblocks > site.cap) return false;   // host sizing error: never write past the partials
#pragma unroll
  for (int t = 0; t < KMAX; ++t) {
    if (t < k) {
      A s = warp_sum(vals[t]);
      if (lane == 0) smem[warp * KMAX + t] = s;
    }
  }
  __syncthreads();
  for (int t = tid; t < k; t += nthr) {
    A s = smem[t];
    for (int w = 1; w < nwarps; ++w) s += smem[w * KMAX + t];
    site.partials[(size_t)blockLinear * kMaxK + t] = s;
  }
  __shared__ unsigned int s_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(site.counter, 1u) == (unsigned)(nblocks - 1));
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  // last block: warp w sums value t = w, w + nwarps, ... over blocks, lane-strided, fixed order
  for (int t = warp; t < k; t += nwarps) {
    A s = lane_strided_sum(site.partials + t, kMaxK, nblocks, lane);
    s = warp_sum(s);
    if (lane == 0) fin(t, s);
  }
  __threadfence_block();
  __syncthreads();
  if (tid == 0) *site.counter = 0u;
  return true;
}

}  // namespace jfnk
