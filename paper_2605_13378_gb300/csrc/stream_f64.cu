// stream_f64.cu -- the basis streaming kernel for the F64 basis
// (see stream_impl.cuh), in a translation unit of its own.
#include "stream_impl.cuh"

namespace jfnk {

cudaError_t basis_stream_f64(int mode, long long n, const void* V, int k, int kmax, void* w, void* d, GmresCtl* ctl,
                             RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  return stream_mode<double, double, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
}

}  // namespace jfnk
