// doe_render.cu -- host side of doe_render (PSF convolution).  Not yet implemented.
#include "doe.h"
#include "doe_launch.h"

int render_entry(int, int, int, const float*, int, int, const float*, float*, void*, size_t, void*) {
  return DOE_EUNSUPPORTED;
}
size_t render_workspace(int, int, int) { return 0; }
