// doe_render_args.h -- parameter block of the render kernels (host and device).
#pragma once
#include <cuda_runtime.h>

namespace doe {
constexpr int RENDER_LINEAR = 0;  // doe_render: linear convolution, 2H x 2W transforms
constexpr int RENDER_WIENER = 1;  // doe_wiener: circular Wiener deconvolution, H x W transforms
struct RenderArgs {
  int C, H, W;          // channels, image rows, image columns
  int Py, Px;           // PSF grid
  int wpr;              // row pitch of SA / SB (complex), >= nk, multiple of kTile
  const float* psf;     // [C][Py][Px]
  const float* img;     // [C][H][W]: scene (render) or blurred image (Wiener)
  float* out;           // [C][H][W]
  float2* sa;           // [C] column-tiled H x wpr: image row spectra
  float2* sb;           // [C] column-tiled H x wpr: kernel row spectra
  float2* sc;           // [C][H][wpr] natural layout: product / filtered spectrum after the column IFFT
  double* ksum;         // [C][H]
  int mode;             // RENDER_LINEAR or RENDER_WIENER
  float gamma;          // Wiener regulariser (RENDER_WIENER)
  int nk;               // stored row-spectrum columns: row transform length / 2 + 1
  // extents in elements, for the bounds checks of the DOE_DEBUG build: psf, img and out, one
  // spectrum buffer (sa, sb or sc: C H wpr) and ksum
  long long n_psf, n_img, n_out, n_s, n_ksum;
};
}  // namespace doe
