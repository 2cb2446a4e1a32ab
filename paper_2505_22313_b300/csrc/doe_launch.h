// doe_launch.h -- host-callable launchers of the device passes (defined in doe_launch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "doe_plan.h"

namespace doe {
cudaError_t upload_tables(const float2* stage_tw, size_t n_stage, const float2* big_tw, size_t n_big);
cudaError_t read_faults(unsigned int* word);  // ORs and clears the fault words of every kernel unit
cudaError_t prepare_kernels();
cudaError_t launch_htab(const Batch& bt, cudaStream_t st);
cudaError_t launch_mr_twiddles(const Batch& bt, cudaStream_t st);
cudaError_t launch_pass_a(int lg, const Batch& bt, cudaStream_t st);
cudaError_t launch_pass_b(int lg, const Batch& bt, cudaStream_t st);
cudaError_t launch_pass_c(int lg, const Batch& bt, cudaStream_t st);
cudaError_t launch_pass_c_adj(int lg, const Batch& bt, cudaStream_t st);
cudaError_t launch_pass_a_adj(int lg, const Batch& bt, cudaStream_t st);
cudaError_t launch_loss_reduce(const Batch& bt, double* loss, cudaStream_t st);
cudaError_t launch_band_mask(const Batch& bt, uint8_t* mask, cudaStream_t st);
cudaError_t launch_wait_check(unsigned polls, cudaStream_t st);  // a bounded wait that runs out
cudaError_t launch_upsample_adjoint(const float* g, float* gc, int N, int uf, cudaStream_t st);
cudaError_t launch_lanczos_up(const float* hl, float* tmp, float* hs, int N, const LanczosTab& tb, cudaStream_t st);
cudaError_t launch_lanczos_adjoint(const float* g, float* tmp, float* gl, int N, const LanczosTab& tb,
                                   cudaStream_t st);
cudaError_t launch_adam(float* h, const float* g, float* m, float* v, long long n, float lr_hat, float beta1,
                        float beta2, float eps_hat, float h_min, float h_max, cudaStream_t st);
cudaError_t launch_radial_heights(const float* c, int n_c, int N, float* h, cudaStream_t st);
cudaError_t launch_radial_grad(const float* g, int n_c, int N, double* part, float* c_grad, cudaStream_t st);

struct RenderArgs;

// pass identifiers reported by the tracer (doe_trace_read / doe_pass_name)
enum : int {
  TR_HTAB = 0, TR_PASS_A, TR_PASS_B, TR_PASS_C, TR_PASS_C_ADJ, TR_PASS_B_ADJ, TR_PASS_A_ADJ, TR_LOSS,
  TR_RENDER_ROWS, TR_RENDER_COLS, TR_RENDER_OUT, TR_MASK, TR_UPSAMPLE_ADJ, TR_ADAM, TR_LANCZOS, TR_LANCZOS_ADJ,
  TR_RADIAL, TR_RADIAL_GRAD, TR_MR_TWIDDLES, TR_COUNT
};
int trace_enable(int max_records);
int trace_read(int max, int* pass_ids, float* ms);
long long launch_count();
cudaError_t launch_render(const RenderArgs& ra, cudaStream_t st);
}  // namespace doe

int render_entry(int C, int H, int W, const float* psf, int Py, int Px, const float* img, float* out, void* ws,
                 size_t ws_bytes, void* stream);
size_t render_workspace(int C, int H, int W);
int wiener_entry(int C, int H, int W, const float* psf, int Py, int Px, const float* y, double gamma, float* out,
                 void* ws, size_t ws_bytes, void* stream);
size_t wiener_workspace(int C, int H, int W);
