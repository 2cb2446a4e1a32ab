// doe_render.cu -- host side of doe_render and doe_wiener: validation, workspace layout,
// launch sequence (kernels in doe_render.cuh).
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

// f = 2: linear render on 2H x 2W transforms; f = 1: circular Wiener on H x W transforms.
int render_check(int C, int H, int W, int f) {
  if (C < 1 || !pow2(H) || !pow2(W) || f * H < 32 || f * W < 32) return DOE_EINVAL;
  if ((long)f * H > doe::kRenderColsMax || (long)f * W > (1L << doe::kMaxLog)) return DOE_EUNSUPPORTED;
  return DOE_OK;
}

// nk = stored columns of a row spectrum (f W / 2 + 1)
RLayout render_layout(int C, int H, int nk) {
  RLayout L;
  L.wpr = (nk + doe::kTile - 1) / doe::kTile * doe::kTile;
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
  if (render_check(C, H, W, 2) != DOE_OK) return 0;
  return render_layout(C, H, W + 1).total;
}

size_t wiener_workspace(int C, int H, int W) {
  if (render_check(C, H, W, 1) != DOE_OK) return 0;
  return render_layout(C, H, W / 2 + 1).total;
}

namespace {
int run(int mode, int C, int H, int W, const float* psf, int Py, int Px, const float* img, double gamma, float* out,
        void* ws, size_t ws_bytes, void* stream) {
  const int f = mode == doe::RENDER_WIENER ? 1 : 2;
  int rc = render_check(C, H, W, f);
  if (rc != DOE_OK) return rc;
  if (!psf || !img || !out) return DOE_EINVAL;
  // the crop's rows start at column Px/2 - W/2 and are read as 8-byte pairs: Px % 4 == 0
  if (Py < H || Px < W || (Py & 1) || (Px & 3)) return DOE_EINVAL;
  if (mode == doe::RENDER_WIENER && !(gamma >= 0.0)) return DOE_EINVAL;
  const int nk = f * W / 2 + 1;
  const RLayout lay = render_layout(C, H, nk);
  if (!ws || ws_bytes < lay.total || (reinterpret_cast<uintptr_t>(ws) & 255u)) return DOE_ENOWS;
  if ((rc = render_ensure_device()) != DOE_OK) return rc;
  doe::RenderArgs ra = {};
  ra.mode = mode;
  ra.gamma = (float)gamma;
  ra.C = C;
  ra.H = H;
  ra.W = W;
  ra.Py = Py;
  ra.Px = Px;
  ra.nk = nk;
  ra.wpr = lay.wpr;
  ra.psf = psf;
  ra.img = img;
  ra.out = out;
  char* base = static_cast<char*>(ws);
  ra.sa = reinterpret_cast<float2*>(base + lay.sa);
  ra.sb = reinterpret_cast<float2*>(base + lay.sb);
  ra.sc = reinterpret_cast<float2*>(base + lay.sc);
  ra.ksum = reinterpret_cast<double*>(base + lay.ks);
  ra.n_psf = (long long)C * Py * Px;
  ra.n_img = ra.n_out = (long long)C * H * W;
  ra.n_s = (long long)C * H * lay.wpr;
  ra.n_ksum = (long long)C * H;
  if (doe::launch_render(ra, static_cast<cudaStream_t>(stream)) != cudaSuccess) return DOE_ECUDA;
  return DOE_OK;
}
}  // namespace

int render_entry(int C, int H, int W, const float* psf, int Py, int Px, const float* img, float* out, void* ws,
                 size_t ws_bytes, void* stream) {
  return run(doe::RENDER_LINEAR, C, H, W, psf, Py, Px, img, 0.0, out, ws, ws_bytes, stream);
}

int wiener_entry(int C, int H, int W, const float* psf, int Py, int Px, const float* y, double gamma, float* out,
                 void* ws, size_t ws_bytes, void* stream) {
  return run(doe::RENDER_WIENER, C, H, W, psf, Py, Px, y, gamma, out, ws, ws_bytes, stream);
}
