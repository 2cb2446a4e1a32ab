// doe_launch.cu -- launch infrastructure (tracing, kernel set-up, cluster launches, the
// per-device twiddle-table registry), the small non-transform kernels, and the routing of
// each pass to its kernel family: power-of-two sides up to one CTA's transform
// (doe_pass_pow2_*.cu), longer power-of-two sides split over a cluster (doe_pass_big.cu),
// non-power-of-two sides (doe_pass_mr.cu).
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "doe_launch_impl.h"
#include "doe_misc.cuh"

namespace doe {

// ------------------------------------------------------------------ tracing
// When enabled, every pass launch is bracketed by two CUDA events recorded on the launching
// stream; doe_trace_read() later reports each pass's device time.  A launch counter is kept
// always.  Host-side bookkeeping only: no device memory is allocated.
namespace {
std::mutex g_tr_mu;
std::vector<cudaEvent_t> g_ev;
std::vector<int> g_tr_pass;
int g_tr_cap = 0;
std::atomic<long long> g_launches{0};
}  // namespace

int trace_begin(int pass, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_tr_mu);
  if (g_tr_cap <= 0 || (int)g_tr_pass.size() >= g_tr_cap) return -1;
  const int slot = (int)g_tr_pass.size();
  g_tr_pass.push_back(pass);
  cudaEventRecord(g_ev[2 * slot], st);
  return slot;
}
void trace_end(int slot, cudaStream_t st) { cudaEventRecord(g_ev[2 * slot + 1], st); }

int trace_enable(int max_records) {
  std::lock_guard<std::mutex> lk(g_tr_mu);
  for (auto e : g_ev) cudaEventDestroy(e);
  g_ev.clear();
  g_tr_pass.clear();
  g_tr_cap = 0;
  if (max_records <= 0) return 0;
  g_ev.resize(2 * (size_t)max_records);
  for (auto& e : g_ev)
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
  g_tr_cap = max_records;
  return 0;
}

int trace_read(int max, int* pass_ids, float* ms) {
  std::lock_guard<std::mutex> lk(g_tr_mu);
  const int n = (int)g_tr_pass.size() < max ? (int)g_tr_pass.size() : max;
  for (int i = 0; i < n; ++i) {
    if (cudaEventSynchronize(g_ev[2 * i + 1]) != cudaSuccess) return -1;
    pass_ids[i] = g_tr_pass[i];
    if (cudaEventElapsedTime(&ms[i], g_ev[2 * i], g_ev[2 * i + 1]) != cudaSuccess) return -1;
  }
  g_tr_pass.clear();
  return n;
}

long long launch_count() { return g_launches.load(); }

// ------------------------------------------------------------------ twiddle tables
// Each kernel translation unit registers the uploader of its own copy of the tables (during
// static initialisation, hence the function-local registry).
namespace {
std::vector<TableUpload>& table_registry() {
  static std::vector<TableUpload> r;
  return r;
}
}  // namespace
int register_table_upload(TableUpload fn) {
  table_registry().push_back(fn);
  return (int)table_registry().size();
}
cudaError_t upload_tables(const float2* stage_tw, size_t n_stage, const float2* big_tw, size_t n_big) {
  for (TableUpload fn : table_registry()) {
    const cudaError_t e = fn(stage_tw, n_stage, big_tw, n_big);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
std::vector<FaultRead>& fault_registry() {
  static std::vector<FaultRead> r;
  return r;
}
}  // namespace
int register_fault_reader(FaultRead fn) {
  fault_registry().push_back(fn);
  return (int)fault_registry().size();
}
cudaError_t read_faults(unsigned int* word) {
  *word = 0;
  for (FaultRead fn : fault_registry()) {
    unsigned int w = 0;
    const cudaError_t e = fn(&w);
    if (e != cudaSuccess) return e;
    *word |= w;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ kernel set-up, launches
cudaError_t prep_kernel(const void* kern, int smem, int threads) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared)))
    return e;
  int dev = 0, blocks = 0, per_sm = 0, reserved = 0;
  cudaFuncAttributes fa;
  if ((e = cudaGetDevice(&dev)) || (e = cudaFuncGetAttributes(&fa, kern)) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, threads, smem)) ||
      (e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) ||
      (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)))
    return e;
  if (blocks < 1 || per_sm <= 0) return cudaSuccess;
  const long need = (long)blocks * ((long)smem + (long)fa.sharedSizeBytes + reserved);
  // the CUDA driver rounds the percentage up to the next shared-memory configuration, so start
  // from the rounded-down percentage and step up only if the resident CTAs would drop
  for (int pct = (int)(need * 100 / per_sm); pct <= 100; ++pct) {
    int b = 0;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem)))
      return e;
    if (b >= blocks) break;
  }
  return cudaSuccess;
}

cudaError_t launch_cluster(const void* fn, dim3 grid, int cluster, size_t smem, cudaStream_t st, void** args,
                           int threads) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t prepare_kernels() {
  cudaError_t e;
  if ((e = pow2_small_prepare()) || (e = pow2_large_prepare()) || (e = big_prepare()) || (e = mr_prepare()) ||
      (e = render_prepare()))
    return e;
  return cudaSuccess;
}

// ------------------------------------------------------------------ pass routing
namespace {
cudaError_t run_pass(int which, int lg, const Batch& bt, cudaStream_t st) {
  if (bt.mr) return mr_pass(which, bt, st);
  if (lg >= 15) return big_pass(which, lg, bt, st);
  if (lg >= 13) return pow2_large_pass(which, lg, bt, st);
  return pow2_small_pass(which, lg, bt, st);
}
}  // namespace
cudaError_t launch_pass_a(int lg, const Batch& bt, cudaStream_t st) { return run_pass(PASS_A, lg, bt, st); }
cudaError_t launch_pass_b(int lg, const Batch& bt, cudaStream_t st) { return run_pass(PASS_B, lg, bt, st); }
cudaError_t launch_pass_c(int lg, const Batch& bt, cudaStream_t st) { return run_pass(PASS_C, lg, bt, st); }
cudaError_t launch_pass_c_adj(int lg, const Batch& bt, cudaStream_t st) { return run_pass(PASS_C_ADJ, lg, bt, st); }
cudaError_t launch_pass_a_adj(int lg, const Batch& bt, cudaStream_t st) { return run_pass(PASS_A_ADJ, lg, bt, st); }
cudaError_t launch_mr_twiddles(const Batch& bt, cudaStream_t st) { return mr_twiddles(bt, st); }

// ------------------------------------------------------------------ small kernels
cudaError_t launch_htab(const Batch& bt, cudaStream_t st) {
  Traced tr(TR_HTAB, st);
  htab_kernel<<<dim3(bt.max_kmax + 1, bt.S), 256, 0, st>>>(bt);
  return cudaGetLastError();
}
cudaError_t launch_loss_reduce(const Batch& bt, double* loss, cudaStream_t st) {
  Traced tr(TR_LOSS, st);
  loss_reduce_kernel<<<1, 1024, 0, st>>>(bt, loss);
  return cudaGetLastError();
}
cudaError_t launch_lanczos_up(const float* hl, float* tmp, float* hs, int N, const LanczosTab& tb, cudaStream_t st) {
  {
    Traced tr(TR_LANCZOS, st);
    const long long n = (long long)tb.nl * N;
    lanczos_up_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(hl, tmp, N, tb);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  Traced tr(TR_LANCZOS, st);
  const long long n = (long long)N * N;
  lanczos_up_cols_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tmp, hs, N, tb);
  return cudaGetLastError();
}
cudaError_t launch_lanczos_adjoint(const float* g, float* tmp, float* gl, int N, const LanczosTab& tb,
                                   cudaStream_t st) {
  {
    Traced tr(TR_LANCZOS_ADJ, st);
    const long long n = (long long)N * tb.nl;
    lanczos_adjoint_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, tmp, N, tb);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  Traced tr(TR_LANCZOS_ADJ, st);
  const long long n = (long long)tb.nl * tb.nl;
  lanczos_adjoint_cols_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tmp, gl, N, tb);
  return cudaGetLastError();
}
cudaError_t launch_adam(float* h, const float* g, float* m, float* v, long long n, float lr_hat, float beta1,
                        float beta2, float eps_hat, float h_min, float h_max, cudaStream_t st) {
  Traced tr(TR_ADAM, st);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(h, g, m, v, n, lr_hat, beta1, beta2, eps_hat, h_min, h_max);
  return cudaGetLastError();
}
// inverse squared half-side (N/2)^-2 in FP64, split into a float pair
static void radial_inv_r2(int N, float& hi, float& lo) {
  const double v = 1.0 / ((0.5 * N) * (0.5 * N));
  hi = (float)v;
  lo = (float)(v - (double)hi);
}
cudaError_t launch_radial_heights(const float* c, int n_c, int N, float* h, cudaStream_t st) {
  Traced tr(TR_RADIAL, st);
  const long long n = (long long)N * N;
  float hi, lo;
  radial_inv_r2(N, hi, lo);
  radial_heights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, n_c, N, hi, lo, h);
  return cudaGetLastError();
}
cudaError_t launch_radial_grad(const float* g, int n_c, int N, double* part, float* c_grad, cudaStream_t st) {
  {
    Traced tr(TR_RADIAL_GRAD, st);
    float hi, lo;
    radial_inv_r2(N, hi, lo);
    radial_grad_kernel<<<kRadialBlocks, 256, 0, st>>>(g, n_c, N, hi, lo, part);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  Traced tr(TR_RADIAL_GRAD, st);
  radial_grad_final_kernel<<<1, 32, 0, st>>>(part, kRadialBlocks, n_c, c_grad);
  return cudaGetLastError();
}
cudaError_t launch_upsample_adjoint(const float* g, float* gc, int N, int uf, cudaStream_t st) {
  Traced tr(TR_UPSAMPLE_ADJ, st);
  const long long cells = (long long)(N >> uf) * (N >> uf);
  upsample_adjoint_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(g, gc, N, uf);
  return cudaGetLastError();
}
cudaError_t launch_band_mask(const Batch& bt, uint8_t* mask, cudaStream_t st) {
  Traced tr(TR_MASK, st);
  band_mask_kernel<<<bt.Py, 256, 0, st>>>(bt, mask);
  return cudaGetLastError();
}

cudaError_t launch_wait_check(unsigned polls, cudaStream_t st) {
  wait_check_kernel<<<1, 32, 0, st>>>(polls);
  return cudaGetLastError();
}

}  // namespace doe
