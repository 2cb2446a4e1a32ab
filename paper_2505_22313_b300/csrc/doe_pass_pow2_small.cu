// doe_pass_pow2_small.cu -- power-of-two passes of 32 .. 4096 points.
#include "doe_pass_pow2.cuh"

namespace doe {

cudaError_t pow2_small_pass(int which, int lg, const Batch& bt, cudaStream_t st) {
  switch (lg) {
    case 5: return pow2_run<32>(which, bt, st);
    case 6: return pow2_run<64>(which, bt, st);
    case 7: return pow2_run<128>(which, bt, st);
    case 8: return pow2_run<256>(which, bt, st);
    case 9: return pow2_run<512>(which, bt, st);
    case 10: return pow2_run<1024>(which, bt, st);
    case 11: return pow2_run<2048>(which, bt, st);
    case 12: return pow2_run<4096>(which, bt, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t pow2_small_prepare() {
  cudaError_t e;
  if ((e = prep_pow2_t<32>()) || (e = prep_pow2_t<64>()) || (e = prep_pow2_t<128>()) || (e = prep_pow2_t<256>()) ||
      (e = prep_pow2_t<512>()) || (e = prep_pow2_t<1024>()) || (e = prep_pow2_t<2048>()) || (e = prep_pow2_t<4096>()))
    return e;
  return cudaSuccess;
}

}  // namespace doe
