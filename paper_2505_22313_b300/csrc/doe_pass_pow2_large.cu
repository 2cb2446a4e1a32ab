// doe_pass_pow2_large.cu -- power-of-two passes of 8192 and 16384 points.
#include "doe_pass_pow2.cuh"

namespace doe {

cudaError_t pow2_large_pass(int which, int lg, const Batch& bt, cudaStream_t st) {
  switch (lg) {
    case 13: return pow2_run<8192>(which, bt, st);
    case 14: return pow2_run<16384>(which, bt, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t pow2_large_prepare() {
  cudaError_t e;
  if ((e = prep_pow2_t<8192>()) || (e = prep_pow2_t<16384>())) return e;
  return cudaSuccess;
}

}  // namespace doe
