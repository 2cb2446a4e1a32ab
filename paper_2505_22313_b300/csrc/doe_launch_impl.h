// doe_launch_impl.h -- what the kernel translation units share: launch tracing, kernel
// attribute set-up, cluster launches, and the per-family launchers that doe_launch.cu routes to.
// The kernel families compile in separate translation units (doe_pass_*.cu) so the build runs
// them in parallel.
#pragma once
#include <cuda_runtime.h>

#include "doe_launch.h"
#include "doe_plan.h"

namespace doe {

// Tracing (doe_launch.cu): every pass launch counts; while tracing is enabled its launch is
// bracketed by two CUDA events on the launching stream.
int trace_begin(int pass, cudaStream_t st);  // the record slot, or -1
void trace_end(int slot, cudaStream_t st);
struct Traced {
  int slot;
  cudaStream_t st;
  Traced(int pass, cudaStream_t s) : slot(trace_begin(pass, s)), st(s) {}
  ~Traced() {
    if (slot >= 0) trace_end(slot, st);
  }
};

// Dynamic shared memory above 48 KB must be opted into, and the carveout preference set to
// the maximum so that several CTAs of a pass fit on one SM; then the carveout is lowered to
// what the register-limited resident CTAs use, so the rest of the SM's 256 KB serves as L1
// for the twiddle tables.
cudaError_t prep_kernel(const void* kern, int smem, int threads);
template <typename K>
cudaError_t prep_one(K* kern, int smem, int threads) {
  return prep_kernel(reinterpret_cast<const void*>(kern), smem, threads);
}

// Launch with a thread-block cluster of `cluster` CTAs along x.
cudaError_t launch_cluster(const void* fn, dim3 grid, int cluster, size_t smem, cudaStream_t st, void** args,
                           int threads);

template <int L>
constexpr size_t smem_bytes() { return (size_t)smem_words(L) * sizeof(float2); }
template <int L>
constexpr int threads() { return L / 32; }

// Pass families.  `which` selects the pass: PASS_A (DOE rows, forward), PASS_B (columns, both
// directions), PASS_C (output rows), PASS_C_ADJ (adjoint rows), PASS_A_ADJ (DOE-row adjoint).
enum : int { PASS_A = 0, PASS_B = 1, PASS_C = 2, PASS_C_ADJ = 3, PASS_A_ADJ = 4 };
// power-of-two sides up to one CTA's transform (doe_pass_pow2_*.cu); lg = log2 P
cudaError_t pow2_small_pass(int which, int lg, const Batch& bt, cudaStream_t st);  // lg 5 .. 12
cudaError_t pow2_large_pass(int which, int lg, const Batch& bt, cudaStream_t st);  // lg 13, 14
cudaError_t pow2_small_prepare();
cudaError_t pow2_large_prepare();
// power-of-two sides split over a cluster (doe_pass_big.cu); lg 15, 16
cudaError_t big_pass(int which, int lg, const Batch& bt, cudaStream_t st);
cudaError_t big_prepare();
// non-power-of-two sides (doe_pass_mr.cu)
cudaError_t mr_pass(int which, const Batch& bt, cudaStream_t st);
cudaError_t mr_twiddles(const Batch& bt, cudaStream_t st);
cudaError_t mr_prepare();
// render and Wiener passes (doe_pass_render.cu)
cudaError_t render_prepare();

}  // namespace doe
