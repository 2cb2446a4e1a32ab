// doe_launch.cu -- the single device translation unit: twiddle tables, every instantiation of
// the passes for L = 16 .. 16384, and their launchers.
#include "doe_kernels.cuh"
#include "doe_launch.h"

namespace doe {

cudaError_t upload_tables(const float2* stage_tw, size_t n_stage, const float2* big_tw, size_t n_big) {
  cudaError_t e = cudaMemcpyToSymbol(g_tw, stage_tw, n_stage * sizeof(float2));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_tw_big, big_tw, n_big * sizeof(float2));
}

namespace {
template <int L>
constexpr size_t smem_bytes() { return (size_t)smem_words(L) * sizeof(float2); }
template <int L>
constexpr int threads() { return L / elems_for(L); }

#define DOE_DISPATCH(lg, fn, ...)                   \
  switch (lg) {                                     \
    case 4: return fn<16>(__VA_ARGS__);             \
    case 5: return fn<32>(__VA_ARGS__);             \
    case 6: return fn<64>(__VA_ARGS__);             \
    case 7: return fn<128>(__VA_ARGS__);            \
    case 8: return fn<256>(__VA_ARGS__);            \
    case 9: return fn<512>(__VA_ARGS__);            \
    case 10: return fn<1024>(__VA_ARGS__);          \
    case 11: return fn<2048>(__VA_ARGS__);          \
    case 12: return fn<4096>(__VA_ARGS__);          \
    case 13: return fn<8192>(__VA_ARGS__);          \
    case 14: return fn<16384>(__VA_ARGS__);         \
    default: return cudaErrorInvalidValue;          \
  }

template <int L>
cudaError_t prep_t() {
  cudaError_t e;
  const int sb = (int)smem_bytes<L>();
  if ((e = cudaFuncSetAttribute(pass_a_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb))) return e;
  if ((e = cudaFuncSetAttribute(pass_b_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb))) return e;
  if ((e = cudaFuncSetAttribute(pass_c_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb))) return e;
  if ((e = cudaFuncSetAttribute(pass_c_adj_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb))) return e;
  if ((e = cudaFuncSetAttribute(pass_a_adj_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb))) return e;
  return cudaSuccess;
}

template <int L>
cudaError_t pass_a_t(const Batch& bt, cudaStream_t st) {
  pass_a_kernel<L><<<dim3(bt.N, bt.S), threads<L>(), smem_bytes<L>(), st>>>(bt);
  return cudaGetLastError();
}
template <int L>
cudaError_t pass_b_t(const Batch& bt, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(bt.total_tiles * kTile);
  cfg.blockDim = dim3(threads<L>());
  cfg.dynamicSmemBytes = smem_bytes<L>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTile;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, pass_b_kernel<L>, bt);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
template <int L>
cudaError_t pass_c_t(const Batch& bt, cudaStream_t st) {
  pass_c_kernel<L><<<dim3(bt.P, bt.S), threads<L>(), smem_bytes<L>(), st>>>(bt);
  return cudaGetLastError();
}
template <int L>
cudaError_t pass_c_adj_t(const Batch& bt, cudaStream_t st) {
  pass_c_adj_kernel<L><<<dim3(bt.P, bt.S), threads<L>(), smem_bytes<L>(), st>>>(bt);
  return cudaGetLastError();
}
template <int L>
cudaError_t pass_a_adj_t(const Batch& bt, cudaStream_t st) {
  pass_a_adj_kernel<L><<<dim3(bt.N), threads<L>(), smem_bytes<L>(), st>>>(bt);
  return cudaGetLastError();
}
}  // namespace

cudaError_t prepare_kernels() {
  cudaError_t e;
  if ((e = prep_t<16>()) || (e = prep_t<32>()) || (e = prep_t<64>()) || (e = prep_t<128>()) ||
      (e = prep_t<256>()) || (e = prep_t<512>()) || (e = prep_t<1024>()) || (e = prep_t<2048>()) ||
      (e = prep_t<4096>()) || (e = prep_t<8192>()) || (e = prep_t<16384>()))
    return e;
  return cudaSuccess;
}

cudaError_t launch_htab(const Batch& bt, cudaStream_t st) {
  htab_kernel<<<dim3(bt.max_kmax + 1, bt.S), 256, 0, st>>>(bt);
  return cudaGetLastError();
}
cudaError_t launch_pass_a(int lg, const Batch& bt, cudaStream_t st) { DOE_DISPATCH(lg, pass_a_t, bt, st); }
cudaError_t launch_pass_b(int lg, const Batch& bt, cudaStream_t st) { DOE_DISPATCH(lg, pass_b_t, bt, st); }
cudaError_t launch_pass_c(int lg, const Batch& bt, cudaStream_t st) { DOE_DISPATCH(lg, pass_c_t, bt, st); }
cudaError_t launch_pass_c_adj(int lg, const Batch& bt, cudaStream_t st) { DOE_DISPATCH(lg, pass_c_adj_t, bt, st); }
cudaError_t launch_pass_a_adj(int lg, const Batch& bt, cudaStream_t st) { DOE_DISPATCH(lg, pass_a_adj_t, bt, st); }
cudaError_t launch_loss_reduce(const Batch& bt, double* loss, cudaStream_t st) {
  loss_reduce_kernel<<<1, 1024, 0, st>>>(bt, loss);
  return cudaGetLastError();
}
cudaError_t launch_band_mask(const Batch& bt, uint8_t* mask, cudaStream_t st) {
  band_mask_kernel<<<bt.P, 256, 0, st>>>(bt, mask);
  return cudaGetLastError();
}

}  // namespace doe
