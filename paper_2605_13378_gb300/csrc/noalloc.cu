// noalloc.cu -- jfnk_jvp_fd_noalloc: the finite-difference Jacobian-vector
// product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running where allocation is
// forbidden or already budgeted to the last byte (inside another library's
// memory pool, in a process whose allocator is owned by a host framework, or
// in latency-critical paths that must never hit the driver allocator). The
// context-based jfnk_jvp needs workspace for the two norms of the step rule
// and, when the caller passes no F_out, for F(x); this variant takes that
// workspace from one file-scope device array instead, so it allocates
// nothing. The paper has no counterpart; it is a deployment convenience.
//
// The array is a fixed size (JFNK_NOALLOC_SCRATCH_BYTES). Every GPU that
// loads the library holds it until the process exits. All calls share it and
// it keeps the previous call's contents, so each call clears what must start
// at zero; calls that overlap on the GPU (different streams, or several host
// threads at once) race on it.
#include <cuda_runtime.h>

#include <math.h>
#include <mutex>
#include <string.h>
#include <type_traits>

#include "jfnk.h"
#include "kernels.h"
#include "krylov.h"

namespace jfnk {

// layout: [0, 256) header (arrival counter, then the two squared norms at
// byte 16), [256, 256 + kNaBlocks * 16) per-block partial sums, then F(x).
constexpr int kNaBlocks = 256;
constexpr size_t kNaHeader = 256;
constexpr size_t kNaPartials = (size_t)kNaBlocks * 2 * sizeof(double);
constexpr size_t kNaFxOffset = kNaHeader + 4096;
static_assert(kNaPartials <= 4096, "partials must fit before F(x)");
static_assert(kNaFxOffset + JFNK_NOALLOC_MAX_FX_BYTES == JFNK_NOALLOC_SCRATCH_BYTES, "scratch layout");

static __device__ __align__(256) unsigned char g_noalloc_scratch[JFNK_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the host-side symbol is only a stand-in) and kept
// for the life of the process; a device reset unloads the array, after which
// the kept address is stale (the header tells callers not to reset).
constexpr int kNaMaxDevices = 64;
static void* g_scratch_addr[kNaMaxDevices];
static std::mutex g_scratch_mu;

static cudaError_t scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return cudaSuccess;
}

// ||x||^2 and ||v||^2 over n entries: per-block partials, then the last block
// to arrive sums them in block order (deterministic for a given n).
template <class T>
__global__ void __launch_bounds__(256) k_na_norms(long long n, const T* __restrict__ x, const T* __restrict__ v,
                                                  unsigned char* scratch) {
  typedef typename std::conditional<sizeof(T) == 8, double, float>::type A;
  unsigned int* counter = (unsigned int*)scratch;
  double* norms = (double*)(scratch + 16);
  double* part = (double*)(scratch + kNaHeader);
  A sx = A(0), sv = A(0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const A a = (A)x[i], b = (A)v[i];
    sx += a * a;
    sv += b * b;
  }
  __shared__ double wsum[2][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double dx = (double)sx, dv = (double)sv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dx += __shfl_xor_sync(0xffffffffu, dx, o);
    dv += __shfl_xor_sync(0xffffffffu, dv, o);
  }
  if (lane == 0) { wsum[0][warp] = dx; wsum[1][warp] = dv; }
  __syncthreads();
  __shared__ unsigned int s_last;
  if (threadIdx.x == 0) {
    double bx = 0.0, bv = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { bx += wsum[0][w]; bv += wsum[1][w]; }
    part[2 * blockIdx.x] = bx;
    part[2 * blockIdx.x + 1] = bv;
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    double tx = 0.0, tv = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      tx += __ldcg(&part[2 * b]);
      tv += __ldcg(&part[2 * b + 1]);
    }
    norms[0] = tx;
    norms[1] = tv;
  }
}

// Derived constants of a problem, as jfnk_set_problem computes them; the aux
// arrays are used in place (FP64 device pointers).
static bool na_problem(const jfnk_problem* pr, ProbDev* P) {
  if (!make_probdev(pr, P, nullptr)) return false;
  if (pr->pde == JFNK_MAXWELL_TE2D || pr->pde == JFNK_MAXWELL_VEC2D) {
    P->eps64 = pr->aux[0];
    P->src64 = pr->aux[1];
  }
  return true;
}

}  // namespace jfnk

using namespace jfnk;

extern "C" jfnk_status jfnk_jvp_fd_noalloc(const jfnk_problem* prob, int prec, const void* x, const void* v,
                                           const void* b, void* F_out, void* Jv_out, double fd_eps,
                                           void* cuda_stream) {
  if (!prob || !x || !v || !Jv_out) return JFNK_E_INVALID;
  if (prec != JFNK_FP64 && prec != JFNK_FP32) return JFNK_E_INVALID;
  ProbDev P;
  if (!na_problem(prob, &P)) return JFNK_E_INVALID;
  if (P.cfl > 0.0) return JFNK_E_INVALID;   // an adaptive step exists only inside jfnk_solve
  if ((P.pde == JFNK_MAXWELL_TE2D || P.pde == JFNK_MAXWELL_VEC2D) && prec != JFNK_FP64)
    return JFNK_E_INVALID;   // eps_r, source are FP64
  const int t = prec == JFNK_FP64 ? VT_F64 : VT_F32;
  const size_t es = prec == JFNK_FP64 ? 8 : 4;
  const long long N = P.ncell * P.nf;
  if (!F_out && (size_t)N * es > JFNK_NOALLOC_MAX_FX_BYTES) return JFNK_E_OOM;   // F(x) does not fit the scratch
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return JFNK_E_CUDA;
  unsigned char* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return JFNK_E_CUDA;
  // the counter and the norms must start at zero; the array keeps the last call's values
  if (cudaMemsetAsync(scratch, 0, kNaHeader, st) != cudaSuccess) return JFNK_E_CUDA;
  void* Fx = F_out ? F_out : (void*)(scratch + kNaFxOffset);
  const void* bb = P.bvp ? nullptr : b;
  if (launch_residual(P, t, x, nullptr, 0.0, bb, Fx, nullptr, nullptr, RedWs{nullptr, nullptr, 0}, nullptr, st) !=
      cudaSuccess)
    return JFNK_E_CUDA;
  JvpArgs a;
  memset(&a, 0, sizeof(a));
  a.lin = 1; a.t = t; a.tv = t; a.x = x; a.v = v; a.b = bb; a.Fx = Fx; a.out = Jv_out; a.c_jv = 1.0;
  a.eps_fixed = fd_eps;
  a.eps_rule = JFNK_EPS_SCALED;
  if (fd_eps <= 0.0) {
    long long nb = (N + 2047) / 2048;
    if (nb > kNaBlocks) nb = kNaBlocks;
    if (nb < 1) nb = 1;
    if (t == VT_F64)
      k_na_norms<double><<<(int)nb, 256, 0, st>>>(N, (const double*)x, (const double*)v, scratch);
    else
      k_na_norms<float><<<(int)nb, 256, 0, st>>>(N, (const float*)x, (const float*)v, scratch);
    if (cudaGetLastError() != cudaSuccess) return JFNK_E_CUDA;
    a.xn2 = (const double*)(scratch + 16);
    a.vn2 = (const double*)(scratch + 24);
  }
  if (launch_jvp(P, a, RedWs{nullptr, nullptr, 0}, st) != cudaSuccess) return JFNK_E_CUDA;
  return JFNK_OK;
}
