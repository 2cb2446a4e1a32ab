// doe_pass_pow2.cuh -- launchers of the power-of-two passes up to one CTA's transform
// (L = 32 .. 16384), instantiated per length by doe_pass_pow2_small.cu / doe_pass_pow2_large.cu.
#pragma once
#include "doe_kernels.cuh"
#include "doe_launch_impl.h"

namespace doe {
namespace {

// Transforms long enough to matter whose first radix lets the 2x-padding zeros fold away.
template <int L>
constexpr bool kPad2Fold = L >= 1024 && pad2_foldable<L>();

// pass A: exchange buffer plus the staged height row (at most L / 2 floats)
template <int L>
constexpr int pass_a_smem() { return (int)(smem_bytes<L>() + (size_t)(L / 2) * sizeof(float)); }

template <int L>
cudaError_t prep_pow2_t() {
  cudaError_t e;
  const int sb = (int)smem_bytes<L>();
  const int nt = threads<L>();
  if ((e = prep_one(pass_a_kernel<L, false, false>, pass_a_smem<L>(), nt)) ||
      (e = prep_one(pass_a_kernel<L, true, false>, pass_a_smem<L>(), nt)))
    return e;
  if ((e = prep_one(pass_b_kernel<L, false>, sb, nt))) return e;
  if constexpr (kPad2Fold<L>)
    if ((e = prep_one(pass_a_kernel<L, false, true>, pass_a_smem<L>(), nt)) ||
        (e = prep_one(pass_a_kernel<L, true, true>, pass_a_smem<L>(), nt)) ||
        (e = prep_one(pass_b_kernel<L, true>, sb, nt)))
      return e;
  if ((e = prep_one(pass_c_kernel<L>, sb, nt))) return e;
  if ((e = prep_one(pass_c_adj_kernel<L>, sb, nt))) return e;
  if ((e = prep_one(pass_a_adj_kernel<L, false>, sb, nt)) || (e = prep_one(pass_a_adj_kernel<L, true>, sb, nt)))
    return e;
  return cudaSuccess;
}

template <int L, bool ILLUM, bool PAD2>
cudaError_t pass_a_run(const Batch& bt, cudaStream_t st) {
  // persistent: about as many CTAs as are resident at once, each looping over (slice, row) items
  static const int resident = [] {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_a_kernel<L, ILLUM, PAD2>, threads<L>(),
                                                      pass_a_smem<L>()))
      return 0;
    return sms * per_sm;
  }();
  const long items = (long)bt.S * bt.N;
  const int grid = (int)(resident > 0 && resident < items ? resident : items);
  const size_t smem = smem_bytes<L>() + (2 * bt.N <= L ? (size_t)bt.N * sizeof(float) : 0);
  pass_a_kernel<L, ILLUM, PAD2><<<dim3(grid), threads<L>(), smem, st>>>(bt);
  return cudaGetLastError();
}

template <int L>
cudaError_t pow2_run(int which, const Batch& bt, cudaStream_t st) {
  switch (which) {
    case PASS_A: {
      Traced tr(TR_PASS_A, st);
      if constexpr (kPad2Fold<L>)
        if (2 * bt.N == L) return bt.illum ? pass_a_run<L, true, true>(bt, st) : pass_a_run<L, false, true>(bt, st);
      return bt.illum ? pass_a_run<L, true, false>(bt, st) : pass_a_run<L, false, false>(bt, st);
    }
    case PASS_B: {
      Traced tr(bt.mode == MODE_ADJ ? TR_PASS_B_ADJ : TR_PASS_B, st);
      void* args[] = {const_cast<Batch*>(&bt)};
      const void* fn = (const void*)pass_b_kernel<L, false>;
      if constexpr (kPad2Fold<L>)
        if (bt.mode != MODE_ADJ && 2 * bt.N == L) fn = (const void*)pass_b_kernel<L, true>;
      return launch_cluster(fn, dim3(bt.total_tiles * kTile), kTile, smem_bytes<L>(), st, args, threads<L>());
    }
    case PASS_C: {
      Traced tr(TR_PASS_C, st);
      pass_c_kernel<L><<<dim3(bt.P, bt.S), threads<L>(), smem_bytes<L>(), st>>>(bt);
      return cudaGetLastError();
    }
    case PASS_C_ADJ: {
      Traced tr(TR_PASS_C_ADJ, st);
      pass_c_adj_kernel<L><<<dim3(bt.P, bt.S), threads<L>(), smem_bytes<L>(), st>>>(bt);
      return cudaGetLastError();
    }
    case PASS_A_ADJ: {
      Traced tr(TR_PASS_A_ADJ, st);
      if (bt.illum)
        pass_a_adj_kernel<L, true><<<dim3(bt.N), threads<L>(), smem_bytes<L>(), st>>>(bt);
      else
        pass_a_adj_kernel<L, false><<<dim3(bt.N), threads<L>(), smem_bytes<L>(), st>>>(bt);
      return cudaGetLastError();
    }
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace doe
