// doe_pass_mr.cu -- grids whose side is not a power of two: the mixed-radix passes of
// doe_mixed.cuh (one CTA of kMrT threads per row / column, the whole transform in shared
// memory) and their cluster splits of doe_mixed_big.cuh.
#include "doe_launch_impl.h"
#include "doe_mixed.cuh"
#include "doe_mixed_big.cuh"

namespace doe {
namespace {

template <int Q, bool CMP>
cudaError_t prep_mrq_t() {
  cudaError_t e;
  constexpr int b = 3 * kMrMax * (int)sizeof(float2);  // twiddle copy and two buffers
  if ((e = prep_one(mrq_rows_fwd_kernel<Q, CMP>, b, kMrT)) || (e = prep_one(mrq_cols_kernel<Q, 1, CMP>, b, kMrT)) ||
      (e = prep_one(mrq_rows_out_kernel<Q, CMP>, b, kMrT)) || (e = prep_one(mrq_rows_adj_c_kernel<Q, CMP>, b, kMrT)) ||
      (e = prep_one(mrq_rows_adj_a_kernel<Q, CMP>, b, kMrT)))
    return e;
  if constexpr (Q <= 8)  // two columns per cluster (2 Q CTAs, at most 16)
    if ((e = prep_one(mrq_cols_kernel<Q, 2, CMP>, b, kMrT))) return e;
  if constexpr (2 * Q > 8 && 2 * Q <= 16)  // two columns per cluster: 10 or 16 CTAs, a non-portable size
    if ((e = cudaFuncSetAttribute(mrq_cols_kernel<Q, 2, CMP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)))
      return e;
  if constexpr (Q > 8) {  // 16-CTA clusters for every pass
    const void* fns[] = {(const void*)mrq_rows_fwd_kernel<Q, CMP>, (const void*)mrq_cols_kernel<Q, 1, CMP>,
                         (const void*)mrq_rows_out_kernel<Q, CMP>, (const void*)mrq_rows_adj_c_kernel<Q, CMP>,
                         (const void*)mrq_rows_adj_a_kernel<Q, CMP>};
    for (const void* f : fns)
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1))) return e;
  }
  return cudaSuccess;
}
template <bool CMP>
cudaError_t prep_mr_t() {
  cudaError_t e;
  constexpr int b = 2 * kMrMax * (int)sizeof(float2);  // two buffers
  // the cluster column pass: two buffers and the transfer-function row (at most Py / 2 + 2)
  constexpr int b4 = (2 * kMrMax + kMrMax / 2 + 2) * (int)sizeof(float2);
  if ((e = prep_one(mr_cols4_kernel<CMP>, b4, kMrT))) return e;
  if ((e = prep_one(mr_rows_fwd_kernel<CMP>, b, kMrT)) || (e = prep_one(mr_cols_kernel<CMP>, b, kMrT)) ||
      (e = prep_one(mr_rows_out_kernel<CMP>, b, kMrT)) || (e = prep_one(mr_rows_adj_c_kernel<CMP>, b, kMrT)) ||
      (e = prep_one(mr_rows_adj_a_kernel<CMP>, b, kMrT)))
    return e;
  if ((e = prep_mrq_t<2, CMP>()) || (e = prep_mrq_t<3, CMP>()) || (e = prep_mrq_t<4, CMP>()) ||
      (e = prep_mrq_t<5, CMP>()) || (e = prep_mrq_t<8, CMP>()) || (e = prep_mrq_t<16, CMP>()))
    return e;
  return cudaSuccess;
}

// shared memory of a one-CTA pass: two transform buffers of its axis (rows: Px; columns: Py)
size_t mr_smem(const Batch& bt, int which) { return (size_t)2 * (which == PASS_B ? bt.Py : bt.P) * sizeof(float2); }

// one CTA per row / column (P <= kMrMax)
template <bool CMP>
cudaError_t mr_one_t(int which, const Batch& bt, cudaStream_t st) {
  const size_t sm = mr_smem(bt, which);
  switch (which) {
    case PASS_A: mr_rows_fwd_kernel<CMP><<<dim3(bt.Ny, bt.S), kMrT, sm, st>>>(bt); break;   // DOE rows
    case PASS_B:  // Px columns: clusters of 4 adjacent columns when Px is a multiple of 4
      if (bt.P % 4 == 0) {
        const int py = bt.Py;
        void* args[] = {const_cast<Batch*>(&bt)};
        return launch_cluster((const void*)mr_cols4_kernel<CMP>, dim3(bt.P, bt.S), 4,
                              (size_t)(2 * py + py / 2 + 2) * sizeof(float2), st, args, kMrT);
      }
      mr_cols_kernel<CMP><<<dim3(bt.P, bt.S), kMrT, sm, st>>>(bt);
      break;
    case PASS_C: mr_rows_out_kernel<CMP><<<dim3(bt.Py, bt.S), kMrT, sm, st>>>(bt); break;   // Py rows
    case PASS_C_ADJ: mr_rows_adj_c_kernel<CMP><<<dim3(bt.Py, bt.S), kMrT, sm, st>>>(bt); break;
    case PASS_A_ADJ: mr_rows_adj_a_kernel<CMP><<<dim3(bt.Ny), kMrT, sm, st>>>(bt); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// split sides (bt.mr_Q > 1): cluster launches
template <int Q, bool CMP>
const void* mrq_fn(int which, bool two) {
  return which == PASS_A   ? (const void*)mrq_rows_fwd_kernel<Q, CMP>
         : which == PASS_B ? (two && Q <= 8 ? (const void*)mrq_cols_kernel<(Q <= 8 ? Q : 8), 2, CMP>
                                          : (const void*)mrq_cols_kernel<Q, 1, CMP>)
         : which == PASS_C ? (const void*)mrq_rows_out_kernel<Q, CMP>
         : which == PASS_C_ADJ ? (const void*)mrq_rows_adj_c_kernel<Q, CMP>
                               : (const void*)mrq_rows_adj_a_kernel<Q, CMP>;
}
template <int Q>
cudaError_t mrq_launch(int which, const Batch& bt, cudaStream_t st) {
  // the column pass takes two adjacent columns per cluster (16-byte row pairs) for transforms
  // with composite stages, whose registers already hold the CTAs to two per SM, while two CTAs
  // of its shared memory still fit on an SM
  const int M = which == PASS_B ? bt.mr_My : bt.mr_M;  // the column pass splits the column axis
  const size_t smem = (size_t)3 * M * sizeof(float2);   // twiddle copy and two buffers
  const bool two = which == PASS_B && bt.mr_cmp && 2 * Q <= 16 && 2 * smem <= (size_t)220 * 1024;
  const void* fn = bt.mr_cmp ? mrq_fn<Q, true>(which, two) : mrq_fn<Q, false>(which, two);
  // DOE rows (A, A*), output rows (C, C'), or columns (B)
  const int lines = (which == PASS_A || which == PASS_A_ADJ) ? bt.Ny : which == PASS_B ? bt.P : bt.Py;
  void* args[] = {const_cast<Batch*>(&bt)};
  return launch_cluster(fn, dim3(lines * Q, which == PASS_A_ADJ ? 1 : bt.S), two ? 2 * Q : Q, smem, st, args, kMrT);
}

}  // namespace

cudaError_t mr_pass(int which, const Batch& bt, cudaStream_t st) {
  const int tr = which == PASS_A ? TR_PASS_A
               : which == PASS_B ? (bt.mode == MODE_ADJ ? TR_PASS_B_ADJ : TR_PASS_B)
               : which == PASS_C ? TR_PASS_C
               : which == PASS_C_ADJ ? TR_PASS_C_ADJ : TR_PASS_A_ADJ;
  Traced t(tr, st);
  // the row passes follow the row transform's split, the column pass the column transform's
  switch (which == PASS_B ? bt.mr_Qy : bt.mr_Q) {
    case 1: return bt.mr_cmp ? mr_one_t<true>(which, bt, st) : mr_one_t<false>(which, bt, st);
    case 2: return mrq_launch<2>(which, bt, st);
    case 3: return mrq_launch<3>(which, bt, st);
    case 4: return mrq_launch<4>(which, bt, st);
    case 5: return mrq_launch<5>(which, bt, st);
    case 8: return mrq_launch<8>(which, bt, st);
    case 16: return mrq_launch<16>(which, bt, st);
    default: return cudaErrorInvalidValue;
  }
}

// The per-stage table of a plan of M (M - 1 entries).
static cudaError_t stage_twiddles(const float2* tws, int M, int nst, const int* radix, cudaStream_t st) {
  MrRadices rad{};
  for (int s = 0; s < nst && s < kMrMaxStages; ++s) rad.r[s] = radix[s];
  if (M > 1)
    mr_stage_twiddle_kernel<<<(unsigned)((M - 1 + 255) / 256), 256, 0, st>>>(const_cast<float2*>(tws), M, nst, rad);
  return cudaGetLastError();
}

cudaError_t mr_twiddles(const Batch& bt, cudaStream_t st) {
  Traced tr(TR_MR_TWIDDLES, st);
  mr_twiddle_kernel<<<(unsigned)((bt.mr_M + 255) / 256), 256, 0, st>>>(const_cast<float2*>(bt.mr_tw), bt.mr_M);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = stage_twiddles(bt.mr_tws, bt.mr_M, bt.mr_nst, bt.mr_radix, st);
  if (e == cudaSuccess && bt.mr_tw_y != bt.mr_tw) {  // rectangular grid: the column transform's tables
    mr_twiddle_kernel<<<(unsigned)((bt.mr_My + 255) / 256), 256, 0, st>>>(const_cast<float2*>(bt.mr_tw_y), bt.mr_My);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = stage_twiddles(bt.mr_tws_y, bt.mr_My, bt.mr_nst_y, bt.mr_radix_y, st);
  }
  if (e == cudaSuccess && bt.mr_Q > 1) {  // the row split's [Px] table
    mr_twiddle_kernel<<<(unsigned)((bt.P + 255) / 256), 256, 0, st>>>(const_cast<float2*>(bt.mr_twP), bt.P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && bt.mr_Qy > 1 && bt.mr_twP_y != bt.mr_twP) {  // a rectangle's column split: [Py]
    mr_twiddle_kernel<<<(unsigned)((bt.Py + 255) / 256), 256, 0, st>>>(const_cast<float2*>(bt.mr_twP_y), bt.Py);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t mr_prepare() {
  cudaError_t e;
  if ((e = prep_mr_t<false>()) || (e = prep_mr_t<true>())) return e;
  return cudaSuccess;
}

}  // namespace doe
