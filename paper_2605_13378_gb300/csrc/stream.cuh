// stream.cuh -- bulk-copy (TMA) streaming of vector chunks into shared memory.
//
// A persistent CTA walks the chunks it owns and keeps S stages of a shared-
// memory ring in flight. A producer warp arms a stage's "full" mbarrier with
// the byte count and its lanes issue one cp.async.bulk per vector chunk; the
// consumer warps wait on that phase, compute from shared memory and arrive on
// the stage's "empty" mbarrier, after which the producer refills the stage
// with the chunk S positions ahead. Waits are bounded by the global timer: on
// expiry the kernel records an error code and stops, so a fault in the copy
// path cannot hang the device.
#pragma once

#include <stdint.h>

#include <atomic>

#include <cuda_runtime.h>

#include "common.cuh"

namespace jfnk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Adds bytes to the transaction count of the barrier's current phase without
// arriving: the phase still needs its arrivals (a later arrive.expect_tx
// adds the rest of the bytes and arrives).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for phase `parity` of `bar`, at most `limit_ns`; false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
}

// Wait for phase `parity` of `bar` until the global timer passes `deadline_ns`;
// false on expiry. Draining several barriers against one deadline bounds the
// whole drain, not each wait.
__device__ __forceinline__ bool mbar_wait_until(uint64_t* bar, uint32_t parity, uint64_t deadline_ns) {
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() > deadline_ns) return false;
  }
}

// Programmatic dependent launch (PDL). A kernel launched with
// launch_maybe_pdl(true, ...) may be dispatched while the kernel before it in
// the stream is still running: grid_dep_wait() blocks until that kernel has
// completed and its memory is visible (a no-op for an ordinary launch), and
// grid_dep_trigger() lets the next kernel be dispatched before this one ends.
// Every kernel that uses them waits before it reads anything an earlier
// kernel wrote, and its grid fits the GPU in one wave, so a dispatched but
// waiting CTA never holds resources a running CTA of the same grid needs.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Named barrier `id` (1..15) over `nthreads` threads of the block (a multiple of 32).
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Bulk copy global -> shared, completing `bytes` on `bar` (16-byte aligned
// addresses, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;   // one second
constexpr int kStreamThreads = 256;
constexpr int kStreamSmem = 200 * 1024;            // ring budget per CTA

// Opt-in of a kernel to more than 48 KB of dynamic shared memory. The
// attribute belongs to the kernel on one device, so the flag that records it
// is kept per device ordinal (a process may launch on several GPUs).
constexpr int kOptInDevices = 64;
struct SmemOptIn {
  std::atomic<bool> done[kOptInDevices];
};
template <class K>
inline cudaError_t smem_opt_in(K* kernel, SmemOptIn& f, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < kOptInDevices;
  if (cached && f.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  if (cached) f.done[dev].store(true, std::memory_order_release);
  return cudaSuccess;
}

// Dynamic shared memory a block of a kernel may use on the current device:
// the device's opt-in limit per block less the kernel's static shared memory,
// kept per device ordinal.
struct SmemLimit {
  std::atomic<int> bytes[kOptInDevices];
};
template <class K>
inline cudaError_t smem_block_limit(K* kernel, SmemLimit& c, int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < kOptInDevices;
  if (cached) {
    const int v = c.bytes[dev].load(std::memory_order_acquire);
    if (v > 0) { *out = v; return cudaSuccess; }
  }
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int v = optin - (int)fa.sharedSizeBytes;
  if (v <= 0) return cudaErrorInvalidValue;
  if (cached) c.bytes[dev].store(v, std::memory_order_release);
  *out = v;
  return cudaSuccess;
}

// Launch `kernel`, with the programmatic stream serialization attribute when
// pdl is set (see grid_dep_wait).
template <class... KArgs, class... Args>
inline cudaError_t launch_maybe_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Error codes written to the device error word.
enum StreamErr { STREAM_OK = 0, STREAM_TIMEOUT = 1 };

}  // namespace jfnk
