// doe_launch.cu -- the single device translation unit: twiddle tables, every instantiation of
// the passes for L = 16 .. 16384, and their launchers.
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "doe_big.cuh"
#include "doe_kernels.cuh"
#include "doe_launch.h"
#include "doe_mixed.cuh"
#include "doe_mixed_big.cuh"
#include "doe_render.cuh"

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

struct Traced {
  int pass;
  cudaStream_t st;
  int slot = -1;
  Traced(int p, cudaStream_t s) : pass(p), st(s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_tr_mu);
    if (g_tr_cap > 0 && (int)g_tr_pass.size() < g_tr_cap) {
      slot = (int)g_tr_pass.size();
      g_tr_pass.push_back(p);
      cudaEventRecord(g_ev[2 * slot], st);
    }
  }
  ~Traced() {
    if (slot >= 0) cudaEventRecord(g_ev[2 * slot + 1], st);
  }
};
}  // namespace

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

cudaError_t upload_tables(const float2* stage_tw, size_t n_stage, const float2* big_tw, size_t n_big) {
  cudaError_t e = cudaMemcpyToSymbol(g_tw, stage_tw, n_stage * sizeof(float2));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_tw_big, big_tw, n_big * sizeof(float2));
}

namespace {
template <int L>
constexpr size_t smem_bytes() { return (size_t)smem_words(L) * sizeof(float2); }
template <int L>
constexpr int threads() { return L / 32; }
// pass A: exchange buffer plus the staged height row (at most L / 2 floats)
template <int L>
constexpr int pass_a_smem() { return (int)(smem_bytes<L>() + (size_t)(L / 2) * sizeof(float)); }

#define DOE_DISPATCH(lg, fn, ...)                   \
  switch (lg) {                                     \
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

// Dynamic shared memory above 48 KB must be opted into, and the carveout preference set to
// the maximum so that several CTAs of a pass fit on one SM.
template <typename K>
cudaError_t prep_one(K* kern, int smem, int threads) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared)))
    return e;
  // Registers, not shared memory, bound the resident CTAs of these kernels; give shared memory
  // only what those CTAs use, so the rest of the SM's 256 KB serves as L1 for the twiddle tables.
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
template <int L>
cudaError_t prep_t() {
  cudaError_t e;
  const int sb = (int)smem_bytes<L>();
  const int nt = threads<L>();
  if ((e = prep_one(pass_a_kernel<L, false>, pass_a_smem<L>(), nt)) ||
      (e = prep_one(pass_a_kernel<L, true>, pass_a_smem<L>(), nt)))
    return e;
  if ((e = prep_one(pass_b_kernel<L>, sb, nt))) return e;
  if ((e = prep_one(pass_c_kernel<L>, sb, nt))) return e;
  if ((e = prep_one(pass_c_adj_kernel<L>, sb, nt))) return e;
  if ((e = prep_one(pass_a_adj_kernel<L, false>, sb, nt)) || (e = prep_one(pass_a_adj_kernel<L, true>, sb, nt)))
    return e;
  if ((e = prep_one(render_rows_kernel<L, false>, sb, nt)) || (e = prep_one(render_rows_kernel<L, true>, sb, nt)))
    return e;
  if constexpr (L <= kRenderColsMax)  // two L-sample buffers must fit one CTA's shared memory
    if ((e = prep_one(render_cols_kernel<L, false>, 2 * sb, nt)) ||
        (e = prep_one(render_cols_kernel<L, true>, 2 * sb, nt)))
      return e;
  if ((e = prep_one(render_out_kernel<L, false>, sb, nt)) || (e = prep_one(render_out_kernel<L, true>, sb, nt)))
    return e;
  return cudaSuccess;
}

template <int L, bool ILLUM>
cudaError_t pass_a_run(const Batch& bt, cudaStream_t st) {
  // persistent: about as many CTAs as are resident at once, each looping over (slice, row) items
  static const int resident = [] {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_a_kernel<L, ILLUM>, threads<L>(),
                                                      pass_a_smem<L>()))
      return 0;
    return sms * per_sm;
  }();
  const long items = (long)bt.S * bt.N;
  const int grid = (int)(resident > 0 && resident < items ? resident : items);
  const size_t smem = smem_bytes<L>() + (2 * bt.N <= L ? (size_t)bt.N * sizeof(float) : 0);
  pass_a_kernel<L, ILLUM><<<dim3(grid), threads<L>(), smem, st>>>(bt);
  return cudaGetLastError();
}
template <int L>
cudaError_t pass_a_t(const Batch& bt, cudaStream_t st) {
  Traced tr(TR_PASS_A, st);
  return bt.illum ? pass_a_run<L, true>(bt, st) : pass_a_run<L, false>(bt, st);
}
template <int L>
cudaError_t pass_b_t(const Batch& bt, cudaStream_t st) {
  Traced tr(bt.mode == MODE_ADJ ? TR_PASS_B_ADJ : TR_PASS_B, st);
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
  Traced tr(TR_PASS_C, st);
  pass_c_kernel<L><<<dim3(bt.P, bt.S), threads<L>(), smem_bytes<L>(), st>>>(bt);
  return cudaGetLastError();
}
template <int L>
cudaError_t pass_c_adj_t(const Batch& bt, cudaStream_t st) {
  Traced tr(TR_PASS_C_ADJ, st);
  pass_c_adj_kernel<L><<<dim3(bt.P, bt.S), threads<L>(), smem_bytes<L>(), st>>>(bt);
  return cudaGetLastError();
}
template <int L>
cudaError_t pass_a_adj_t(const Batch& bt, cudaStream_t st) {
  Traced tr(TR_PASS_A_ADJ, st);
  if (bt.illum)
    pass_a_adj_kernel<L, true><<<dim3(bt.N), threads<L>(), smem_bytes<L>(), st>>>(bt);
  else
    pass_a_adj_kernel<L, false><<<dim3(bt.N), threads<L>(), smem_bytes<L>(), st>>>(bt);
  return cudaGetLastError();
}
// ---- grids longer than one CTA (P = Q * 8192 sub-transforms): cluster launches
cudaError_t launch_cluster(const void* fn, dim3 grid, int cluster, size_t smem, cudaStream_t st, void** args,
                           int threads = kBigL / 32) {
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
template <int Q>
cudaError_t big_rows_t(int which, const Batch& bt, cudaStream_t st) {
  const void* fn = which == 0 ? (bt.illum ? (const void*)pass_a_big_kernel<Q, true> : (const void*)pass_a_big_kernel<Q, false>)
                 : which == 1 ? (const void*)pass_c_big_kernel<Q>
                 : which == 2 ? (const void*)pass_c_adj_big_kernel<Q>
                 : bt.illum   ? (const void*)pass_a_adj_big_kernel<Q, true>
                              : (const void*)pass_a_adj_big_kernel<Q, false>;
  const int rows = (which == 0 || which == 3) ? bt.N : bt.P;
  const dim3 grid(rows * Q, which == 3 ? 1 : bt.S);
  void* args[] = {const_cast<Batch*>(&bt)};
  return launch_cluster(fn, grid, Q, smem_bytes<kBigL>(), st, args);
}
template <int Q>
cudaError_t big_cols_t(const Batch& bt, cudaStream_t st) {
  void* args[] = {const_cast<Batch*>(&bt)};
  constexpr int CL = big_tile(Q) * Q;
  return launch_cluster((const void*)pass_b_big_kernel<Q>, dim3(bt.total_tiles * CL), CL, smem_bytes<kBigL>(), st,
                        args, kBigL / 32);
}
template <int Q>
cudaError_t prep_big_t() {
  cudaError_t e;
  const int sb = (int)smem_bytes<kBigL>();
  constexpr int nt = kBigL / 32;
  if ((e = prep_one(pass_a_big_kernel<Q, false>, sb, nt)) || (e = prep_one(pass_a_big_kernel<Q, true>, sb, nt)))
    return e;
  if ((e = prep_one(pass_b_big_kernel<Q>, sb, nt))) return e;
  if ((e = prep_one(pass_c_big_kernel<Q>, sb, nt))) return e;
  if ((e = prep_one(pass_c_adj_big_kernel<Q>, sb, nt))) return e;
  if ((e = prep_one(pass_a_adj_big_kernel<Q, false>, sb, nt)) ||
      (e = prep_one(pass_a_adj_big_kernel<Q, true>, sb, nt)))
    return e;
  return cudaSuccess;
}

template <int L>
cudaError_t render_rows_t(const RenderArgs& ra, cudaStream_t st) {
  Traced tr(TR_RENDER_ROWS, st);
  if (ra.mode == RENDER_WIENER)
    render_rows_kernel<L, true><<<dim3(ra.H, ra.C), threads<L>(), smem_bytes<L>(), st>>>(ra);
  else
    render_rows_kernel<L, false><<<dim3(ra.H, ra.C), threads<L>(), smem_bytes<L>(), st>>>(ra);
  return cudaGetLastError();
}
template <int L>
cudaError_t render_cols_t(const RenderArgs& ra, cudaStream_t st) {
  if constexpr (L > kRenderColsMax) return cudaErrorInvalidValue;
  Traced tr(TR_RENDER_COLS, st);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ra.C * (ra.wpr / kTile) * kTile);
  cfg.blockDim = dim3(threads<L>());
  cfg.dynamicSmemBytes = 2 * smem_bytes<L>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTile;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = ra.mode == RENDER_WIENER ? cudaLaunchKernelEx(&cfg, render_cols_kernel<L, true>, ra)
                                            : cudaLaunchKernelEx(&cfg, render_cols_kernel<L, false>, ra);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
template <int L>
cudaError_t render_out_t(const RenderArgs& ra, cudaStream_t st) {
  Traced tr(TR_RENDER_OUT, st);
  if (ra.mode == RENDER_WIENER)
    render_out_kernel<L, true><<<dim3(ra.H / 2, ra.C), threads<L>(), smem_bytes<L>(), st>>>(ra);
  else
    render_out_kernel<L, false><<<dim3(ra.H / 2, ra.C), threads<L>(), smem_bytes<L>(), st>>>(ra);
  return cudaGetLastError();
}
int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
}  // namespace

cudaError_t launch_render(const RenderArgs& ra, cudaStream_t st) {
  cudaError_t e;
  // linear render: 2W x 2H transforms; Wiener (circular): W x H
  const int f = ra.mode == RENDER_WIENER ? 1 : 2;
  const int lw = ilog2i(f * ra.W), lh = ilog2i(f * ra.H);
  if ((e = [&]() -> cudaError_t { DOE_DISPATCH(lw, render_rows_t, ra, st); }())) return e;
  if ((e = [&]() -> cudaError_t { DOE_DISPATCH(lh, render_cols_t, ra, st); }())) return e;
  return [&]() -> cudaError_t { DOE_DISPATCH(lw, render_out_t, ra, st); }();
}

template <int Q, bool CMP>
cudaError_t prep_mrq_t() {
  cudaError_t e;
  constexpr int b = 3 * kMrMax * (int)sizeof(float2);
  if ((e = prep_one(mrq_rows_fwd_kernel<Q, CMP>, b, kMrT)) || (e = prep_one(mrq_cols_kernel<Q, CMP>, b, kMrT)) ||
      (e = prep_one(mrq_rows_out_kernel<Q, CMP>, b, kMrT)) || (e = prep_one(mrq_rows_adj_c_kernel<Q, CMP>, b, kMrT)) ||
      (e = prep_one(mrq_rows_adj_a_kernel<Q, CMP>, b, kMrT)))
    return e;
  return cudaSuccess;
}
template <bool CMP>
cudaError_t prep_mr_t() {
  cudaError_t e;
  constexpr int b = 3 * kMrMax * (int)sizeof(float2);  // twiddles and two buffers
  if ((e = prep_one(mr_rows_fwd_kernel<CMP>, b, kMrT)) || (e = prep_one(mr_cols_kernel<CMP>, b, kMrT)) ||
      (e = prep_one(mr_rows_out_kernel<CMP>, b, kMrT)) || (e = prep_one(mr_rows_adj_c_kernel<CMP>, b, kMrT)) ||
      (e = prep_one(mr_rows_adj_a_kernel<CMP>, b, kMrT)))
    return e;
  if ((e = prep_mrq_t<2, CMP>()) || (e = prep_mrq_t<3, CMP>()) || (e = prep_mrq_t<4, CMP>()) ||
      (e = prep_mrq_t<5, CMP>()) || (e = prep_mrq_t<8, CMP>()))
    return e;
  return cudaSuccess;
}
cudaError_t prep_mr() {
  cudaError_t e;
  if ((e = prep_mr_t<false>()) || (e = prep_mr_t<true>())) return e;
  return cudaSuccess;
}

cudaError_t prepare_kernels() {
  cudaError_t e;
  if ((e = prep_t<32>()) || (e = prep_t<64>()) || (e = prep_t<128>()) ||
      (e = prep_t<256>()) || (e = prep_t<512>()) || (e = prep_t<1024>()) || (e = prep_t<2048>()) ||
      (e = prep_t<4096>()) || (e = prep_t<8192>()) || (e = prep_t<16384>()) || (e = prep_big_t<4>()) ||
      (e = prep_big_t<8>()))
    return e;
  if ((e = prep_mr())) return e;
  return cudaSuccess;
}

cudaError_t launch_htab(const Batch& bt, cudaStream_t st) {
  Traced tr(TR_HTAB, st);
  htab_kernel<<<dim3(bt.max_kmax + 1, bt.S), 256, 0, st>>>(bt);
  return cudaGetLastError();
}
// Grids longer than one CTA (lg = 15, 16) go to the cluster-split passes of doe_big.cuh.
#define DOE_BIG_ROWS(which, trace)                                          \
  if (lg == 15) { Traced tr(trace, st); return big_rows_t<4>(which, bt, st); } \
  if (lg == 16) { Traced tr(trace, st); return big_rows_t<8>(which, bt, st); }
// Non-power-of-two sides (bt.mr): the mixed-radix passes of doe_mixed.cuh, one CTA of kMrT
// threads per row / column pair, the whole transform in shared memory.
// shared memory: the twiddle table plus two transform buffers
size_t mr_smem(const Batch& bt) { return (size_t)3 * bt.P * sizeof(float2); }
#define DOE_MR(kern, grid)                                      \
  do {                                                          \
    if (bt.mr_cmp)                                              \
      kern<true><<<grid, kMrT, mr_smem(bt), st>>>(bt);          \
    else                                                        \
      kern<false><<<grid, kMrT, mr_smem(bt), st>>>(bt);         \
    return cudaGetLastError();                                  \
  } while (0)
cudaError_t launch_mr_twiddles(const Batch& bt, cudaStream_t st) {
  {
    Traced tr(TR_MR_TWIDDLES, st);
    mr_twiddle_kernel<<<(unsigned)((bt.mr_M + 255) / 256), 256, 0, st>>>(const_cast<float2*>(bt.mr_tw), bt.mr_M);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || bt.mr_Q == 1) return e;
  }
  Traced tr(TR_MR_TWIDDLES, st);
  mr_twiddle_kernel<<<(unsigned)((bt.P + 255) / 256), 256, 0, st>>>(const_cast<float2*>(bt.mr_twP), bt.P);
  return cudaGetLastError();
}
// Split sides (bt.mr_Q > 1): cluster launches of doe_mixed_big.cuh.  which: 0 rows forward (A),
// 1 columns (B / B*), 2 rows out (C), 3 rows adjoint (C'), 4 DOE-row adjoint (A*).
template <int Q, bool CMP>
const void* mrq_fn(int which) {
  return which == 0   ? (const void*)mrq_rows_fwd_kernel<Q, CMP>
         : which == 1 ? (const void*)mrq_cols_kernel<Q, CMP>
         : which == 2 ? (const void*)mrq_rows_out_kernel<Q, CMP>
         : which == 3 ? (const void*)mrq_rows_adj_c_kernel<Q, CMP>
                      : (const void*)mrq_rows_adj_a_kernel<Q, CMP>;
}
template <int Q>
cudaError_t mrq_launch(int which, const Batch& bt, cudaStream_t st) {
  const void* fn = bt.mr_cmp ? mrq_fn<Q, true>(which) : mrq_fn<Q, false>(which);
  const int lines = (which == 0 || which == 4) ? bt.N : bt.P;
  void* args[] = {const_cast<Batch*>(&bt)};
  return launch_cluster(fn, dim3(lines * Q, which == 4 ? 1 : bt.S), Q, (size_t)3 * bt.mr_M * sizeof(float2), st,
                        args, kMrT);
}
cudaError_t mrq_dispatch(int which, const Batch& bt, cudaStream_t st) {
  switch (bt.mr_Q) {
    case 2: return mrq_launch<2>(which, bt, st);
    case 3: return mrq_launch<3>(which, bt, st);
    case 4: return mrq_launch<4>(which, bt, st);
    case 5: return mrq_launch<5>(which, bt, st);
    case 8: return mrq_launch<8>(which, bt, st);
    default: return cudaErrorInvalidValue;
  }
}
#define DOE_MRQ(which)                                      \
  if (bt.mr_Q > 1) return mrq_dispatch(which, bt, st)
cudaError_t launch_pass_a(int lg, const Batch& bt, cudaStream_t st) {
  if (bt.mr) {
    Traced tr(TR_PASS_A, st);
    DOE_MRQ(0);
    DOE_MR(mr_rows_fwd_kernel, dim3(bt.N, bt.S));
  }
  DOE_BIG_ROWS(0, TR_PASS_A)
  DOE_DISPATCH(lg, pass_a_t, bt, st);
}
cudaError_t launch_pass_b(int lg, const Batch& bt, cudaStream_t st) {
  if (bt.mr) {
    Traced tr(bt.mode == MODE_ADJ ? TR_PASS_B_ADJ : TR_PASS_B, st);
    DOE_MRQ(1);
    DOE_MR(mr_cols_kernel, dim3(bt.P, bt.S));
  }
  if (lg >= 15) {  // columns longer than one CTA's transform: Q = P / 8192 sub-transforms of 8192 points
    Traced tr(bt.mode == MODE_ADJ ? TR_PASS_B_ADJ : TR_PASS_B, st);
    return lg == 15 ? big_cols_t<4>(bt, st) : big_cols_t<8>(bt, st);
  }
  DOE_DISPATCH(lg, pass_b_t, bt, st);
}
cudaError_t launch_pass_c(int lg, const Batch& bt, cudaStream_t st) {
  if (bt.mr) {
    Traced tr(TR_PASS_C, st);
    DOE_MRQ(2);
    DOE_MR(mr_rows_out_kernel, dim3(bt.P, bt.S));
  }
  DOE_BIG_ROWS(1, TR_PASS_C)
  DOE_DISPATCH(lg, pass_c_t, bt, st);
}
cudaError_t launch_pass_c_adj(int lg, const Batch& bt, cudaStream_t st) {
  if (bt.mr) {
    Traced tr(TR_PASS_C_ADJ, st);
    DOE_MRQ(3);
    DOE_MR(mr_rows_adj_c_kernel, dim3(bt.P, bt.S));
  }
  DOE_BIG_ROWS(2, TR_PASS_C_ADJ)
  DOE_DISPATCH(lg, pass_c_adj_t, bt, st);
}
cudaError_t launch_pass_a_adj(int lg, const Batch& bt, cudaStream_t st) {
  if (bt.mr) {
    Traced tr(TR_PASS_A_ADJ, st);
    DOE_MRQ(4);
    DOE_MR(mr_rows_adj_a_kernel, dim3(bt.N));
  }
  DOE_BIG_ROWS(3, TR_PASS_A_ADJ)
  DOE_DISPATCH(lg, pass_a_adj_t, bt, st);
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
  band_mask_kernel<<<bt.P, 256, 0, st>>>(bt, mask);
  return cudaGetLastError();
}

}  // namespace doe
