// stream_f64.cu -- the basis streaming kernel for the F64 basis
// and the delayed-CGS2 passes (see stream_impl.cuh, dcgs_impl.cuh), in a
// translation unit of its own.
#include "dcgs_impl.cuh"
#include "stream_impl.cuh"

namespace jfnk {

cudaError_t basis_stream_f64(int mode, long long n, const void* V, int k, int kmax, void* w, void* d, GmresCtl* ctl,
                             RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  return stream_mode<double, double, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
}

cudaError_t dcgs_f64(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                     unsigned int* err, int nsm, cudaStream_t st, bool pdl, bool defer) {
  return dcgs_dispatch<double, double>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
}

}  // namespace jfnk
