// doe_pass_render.cu -- the render (linear convolution) and Wiener passes of doe_render.cuh.
#include "doe_launch_impl.h"
#include "doe_render.cuh"

namespace doe {
namespace {

template <int L>
cudaError_t prep_render_t() {
  cudaError_t e;
  const int sb = (int)smem_bytes<L>();
  const int nt = threads<L>();
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
  if constexpr (L > kRenderColsMax) {
    return cudaErrorInvalidValue;
  } else {
    Traced tr(TR_RENDER_COLS, st);
    void* args[] = {const_cast<RenderArgs*>(&ra)};
    const void* fn = ra.mode == RENDER_WIENER ? (const void*)render_cols_kernel<L, true>
                                              : (const void*)render_cols_kernel<L, false>;
    return launch_cluster(fn, dim3(ra.C * (ra.wpr / kTile) * kTile), kTile, 2 * smem_bytes<L>(), st, args,
                          threads<L>());
  }
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

#define DOE_RENDER_DISPATCH(lg, fn, ...)            \
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

int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

}  // namespace

cudaError_t launch_render(const RenderArgs& ra, cudaStream_t st) {
  cudaError_t e;
  // linear render: 2W x 2H transforms; Wiener (circular): W x H
  const int f = ra.mode == RENDER_WIENER ? 1 : 2;
  const int lw = ilog2i(f * ra.W), lh = ilog2i(f * ra.H);
  if ((e = [&]() -> cudaError_t { DOE_RENDER_DISPATCH(lw, render_rows_t, ra, st); }())) return e;
  if ((e = [&]() -> cudaError_t { DOE_RENDER_DISPATCH(lh, render_cols_t, ra, st); }())) return e;
  return [&]() -> cudaError_t { DOE_RENDER_DISPATCH(lw, render_out_t, ra, st); }();
}

cudaError_t render_prepare() {
  cudaError_t e;
  if ((e = prep_render_t<32>()) || (e = prep_render_t<64>()) || (e = prep_render_t<128>()) ||
      (e = prep_render_t<256>()) || (e = prep_render_t<512>()) || (e = prep_render_t<1024>()) ||
      (e = prep_render_t<2048>()) || (e = prep_render_t<4096>()) || (e = prep_render_t<8192>()) ||
      (e = prep_render_t<16384>()))
    return e;
  return cudaSuccess;
}

}  // namespace doe
