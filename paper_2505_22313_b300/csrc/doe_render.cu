// doe_render.cu -- host side of doe_render: validation, workspace layout, launch sequence
// (kernels in doe_render.cuh).
#include <cuda_runtime.h>

#include <cstdint>

#include "doe.h"
#include "doe_launch.h"
#include "doe_plan.h"
#include "doe_render_args.h"


namespace {
bool pow2(long n) { return n > 0 && (n & (n - 1)) == 0; }
size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct RLayout {
  size_t sa = 0, sb = 0, sc = 0, ks = 0, total = 0;
  int wpr = 0;
};

int render_check(int C, int H, int W) {
  if (C < 1 || !pow2(H) || !pow2(W) || H < 16 || W < 16) return DOE_EINVAL;
  if (2L * H > doe::kRenderColsMax || 2L * W > (1L << doe::kMaxLog)) return DOE_EUNSUPPORTED;
  return DOE_OK;
}

RLayout render_layout(int C, int H, int W) {
  RLayout L;
  L.wpr = (W + 1 + doe::kTile - 1) / doe::kTile * doe::kTile;
  const size_t plane = (size_t)C * H * L.wpr * sizeof(float2);
  L.sa = 0;
  L.sb = a256(plane);
  L.sc = L.sb + a256(plane);
  L.ks = L.sc + a256(plane);
  L.total = L.ks + a256((size_t)C * H * sizeof(double));
  return L;
}
}  // namespace

int render_ensure_device();

size_t render_workspace(int C, int H, int W) {
  if (render_check(C, H, W) != DOE_OK) return 0;
  return render_layout(C, H, W).total;
}

int render_entry(int C, int H, int W, const float* psf, int Py, int Px, const float* img, float* out, void* ws,
                 size_t ws_bytes, void* stream) {
  int rc = render_check(C, H, W);
  if (rc != DOE_OK) return rc;
  if (!psf || !img || !out) return DOE_EINVAL;
  if (Py < H || Px < W || (Py & 1) || (Px & 1)) return DOE_EINVAL;
  const RLayout lay = render_layout(C, H, W);
  if (!ws || ws_bytes < lay.total || (reinterpret_cast<uintptr_t>(ws) & 255u)) return DOE_ENOWS;
  if ((rc = render_ensure_device()) != DOE_OK) return rc;
  doe::RenderArgs ra;
  ra.C = C;
  ra.H = H;
  ra.W = W;
  ra.Py = Py;
  ra.Px = Px;
  ra.wpr = lay.wpr;
  ra.psf = psf;
  ra.img = img;
  ra.out = out;
  char* base = static_cast<char*>(ws);
  ra.sa = reinterpret_cast<float2*>(base + lay.sa);
  ra.sb = reinterpret_cast<float2*>(base + lay.sb);
  ra.sc = reinterpret_cast<float2*>(base + lay.sc);
  ra.ksum = reinterpret_cast<double*>(base + lay.ks);
  if (doe::launch_render(ra, static_cast<cudaStream_t>(stream)) != cudaSuccess) return DOE_ECUDA;
  return DOE_OK;
}
