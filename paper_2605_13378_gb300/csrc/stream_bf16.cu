// stream_bf16.cu -- the basis streaming kernel for the BF16 basis
// and the delayed-CGS2 passes (see stream_impl.cuh, dcgs_impl.cuh), in a
// translation unit of its own.
#include "dcgs_impl.cuh"
#include "stream_impl.cuh"

namespace jfnk {

cudaError_t basis_stream_bf16(int mode, long long n, const void* V, int k, int kmax, void* w, void* d,
                              GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  return stream_mode<__nv_bfloat16, float, double>(mode, n, V, k, kmax, w, d, ctl, red, err, nsm, st);
}

cudaError_t dcgs_bf16(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                     unsigned int* err, int nsm, cudaStream_t st, bool pdl, bool defer) {
  return dcgs_dispatch<__nv_bfloat16, float>(pass, n, V, j, w, ctl, red, err, nsm, st, pdl, defer);
}

}  // namespace jfnk
