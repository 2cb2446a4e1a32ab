// doe_pass_big.cu -- power-of-two grids longer than one CTA's transform (P = 32768, 65536):
// every pass split across a thread-block cluster of Q = P / 8192 CTAs (doe_big.cuh).
#include "doe_big.cuh"
#include "doe_launch_impl.h"

namespace doe {
namespace {

template <int Q>
cudaError_t big_rows_t(int which, const Batch& bt, cudaStream_t st) {
  const void* fn = which == PASS_A ? (bt.illum ? (const void*)pass_a_big_kernel<Q, true> : (const void*)pass_a_big_kernel<Q, false>)
                 : which == PASS_C ? (const void*)pass_c_big_kernel<Q>
                 : which == PASS_C_ADJ ? (const void*)pass_c_adj_big_kernel<Q>
                 : bt.illum   ? (const void*)pass_a_adj_big_kernel<Q, true>
                              : (const void*)pass_a_adj_big_kernel<Q, false>;
  const int rows = (which == PASS_A || which == PASS_A_ADJ) ? bt.N : bt.P;
  const dim3 grid(rows * Q, which == PASS_A_ADJ ? 1 : bt.S);
  void* args[] = {const_cast<Batch*>(&bt)};
  return launch_cluster(fn, grid, Q, smem_bytes<kBigL>(), st, args, kBigL / 32);
}
template <int Q>
cudaError_t big_cols_t(const Batch& bt, cudaStream_t st) {
  void* args[] = {const_cast<Batch*>(&bt)};
  constexpr int CL = big_tile(Q) * Q;
  return launch_cluster((const void*)pass_b_big_kernel<Q>, dim3(bt.total_tiles * CL), CL, smem_bytes<kBigL>(), st,
                        args, kBigL / 32);
}
template <int Q>
cudaError_t big_run(int which, const Batch& bt, cudaStream_t st) {
  return which == PASS_B ? big_cols_t<Q>(bt, st) : big_rows_t<Q>(which, bt, st);
}
template <int Q>
cudaError_t prep_big_t() {
  cudaError_t e;
  const int sb = (int)smem_bytes<kBigL>();
  constexpr int nt = kBigL / 32;
  if ((e = prep_one(pass_a_big_kernel<Q, false>, sb, nt)) || (e = prep_one(pass_a_big_kernel<Q, true>, sb, nt)))
    return e;
  if ((e = prep_one(pass_b_big_kernel<Q>, sb, nt))) return e;
  if constexpr (big_tile(Q) * Q > 8)  // 16-CTA clusters: the non-portable size
    if ((e = cudaFuncSetAttribute(pass_b_big_kernel<Q>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1))) return e;
  if ((e = prep_one(pass_c_big_kernel<Q>, sb, nt))) return e;
  if ((e = prep_one(pass_c_adj_big_kernel<Q>, sb, nt))) return e;
  if ((e = prep_one(pass_a_adj_big_kernel<Q, false>, sb, nt)) ||
      (e = prep_one(pass_a_adj_big_kernel<Q, true>, sb, nt)))
    return e;
  return cudaSuccess;
}

}  // namespace

cudaError_t big_pass(int which, int lg, const Batch& bt, cudaStream_t st) {
  const int tr = which == PASS_A ? TR_PASS_A
               : which == PASS_B ? (bt.mode == MODE_ADJ ? TR_PASS_B_ADJ : TR_PASS_B)
               : which == PASS_C ? TR_PASS_C
               : which == PASS_C_ADJ ? TR_PASS_C_ADJ : TR_PASS_A_ADJ;
  Traced t(tr, st);
  if (lg == 15) return big_run<4>(which, bt, st);
  if (lg == 16) return big_run<8>(which, bt, st);
  return cudaErrorInvalidValue;
}

cudaError_t big_prepare() {
  cudaError_t e;
  if ((e = prep_big_t<4>()) || (e = prep_big_t<8>())) return e;
  return cudaSuccess;
}

}  // namespace doe
