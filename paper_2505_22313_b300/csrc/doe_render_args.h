// doe_render_args.h -- parameter block of the render kernels (host and device).
#pragma once
#include <cuda_runtime.h>

namespace doe {
struct RenderArgs {
  int C, H, W;          // channels, image rows, image columns
  int Py, Px;           // PSF grid
  int wpr;              // row pitch of SA / SB (complex), >= W + 1, multiple of kTile
  const float* psf;     // [C][Py][Px]
  const float* img;     // [C][H][W]
  float* out;           // [C][H][W]
  float2* sa;           // [C] column-tiled H x wpr: image row spectra
  float2* sb;           // [C] column-tiled H x wpr: kernel row spectra
  float2* sc;           // [C][H][wpr] natural layout: product after the column IFFT
  double* ksum;         // [C][H]
};
}  // namespace doe
