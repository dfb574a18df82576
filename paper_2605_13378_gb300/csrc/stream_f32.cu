// stream_f32.cu -- the basis streaming kernel for the F32 basis
// and the delayed-CGS2 passes (see stream_impl.cuh, dcgs_impl.cuh), in a
// translation unit of its own.
#include "dcgs_impl.cuh"
#include "stream_impl.cuh"

namespace jfnk {

cudaError_t basis_stream_f32(int mode, int td, long long n, const void* V, int k, int kmax, void* w, void* d,
                             GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  if (td == VT_F64) return stream_mode<float, float, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
  return stream_mode<float, float, float>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
}

cudaError_t dcgs_f32(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                     unsigned int* err, int nsm, cudaStream_t st, bool pdl, bool defer) {
  return dcgs_dispatch<float, float>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
}

}  // namespace jfnk
