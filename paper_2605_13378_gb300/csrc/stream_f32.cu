// stream_f32.cu -- the basis streaming kernel for the F32 basis
// (see stream_impl.cuh), in a translation unit of its own.
#include "stream_impl.cuh"

namespace jfnk {

cudaError_t basis_stream_f32(int mode, int td, long long n, const void* V, int k, int kmax, void* w, void* d,
                             GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  if (td == VT_F64) return stream_mode<float, float, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  return stream_mode<float, float, float>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
}

}  // namespace jfnk
