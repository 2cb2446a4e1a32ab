// doe_design.cu -- design-loop tools around doe_grad.
//  * doe_adam_step: one step of Adam (Kingma & Ba 2015, the optimiser the paper uses for its
//    designs, Sec. 3.2's toy example and the applications of Sec. 5) on the height map,
//    followed by a projection onto the fabricable height range [h_min, h_max].  Elementwise,
//    one thread per height sample, FP32 state.
//  * doe_radial_heights / doe_radial_grad: the radially symmetric parameterisation of Sec. 5.4's
//    broadband design (an even polynomial of degree 16 in the normalised radius) and its
//    transpose, which maps doe_grad's height gradient to the coefficients.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "doe.h"
#include "doe_launch.h"

extern "C" int doe_adam_step(float* h, const float* grad, float* m, float* v, long long n, double lr, double beta1,
                             double beta2, double eps, int t, double h_min, double h_max, void* stream) {
  if (!h || !grad || !m || !v || n < 1 || t < 1) return DOE_EINVAL;
  if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) ||
      !(h_min <= h_max))
    return DOE_EINVAL;
  const double c1 = 1.0 - std::pow(beta1, (double)t), c2 = std::sqrt(1.0 - std::pow(beta2, (double)t));
  // bias corrections folded into the step: lr_hat = lr sqrt(1 - beta2^t) / (1 - beta1^t),
  // eps_hat = eps sqrt(1 - beta2^t)
  const cudaError_t e = doe::launch_adam(h, grad, m, v, n, (float)(lr * c2 / c1), (float)beta1, (float)beta2,
                                         (float)(eps * c2), (float)h_min, (float)h_max,
                                         static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DOE_OK : DOE_ECUDA;
}

static bool radial_size_ok(int n, int n_c) {
  return n >= 16 && n <= 65536 && (n & 1) == 0 && n_c >= 1 && n_c <= doe::kMaxRadial;
}

extern "C" int doe_radial_heights(int n, const float* c, int n_c, float* h, void* stream) {
  if (!c || !h || !radial_size_ok(n, n_c)) return DOE_EINVAL;
  return doe::launch_radial_heights(c, n_c, n, h, static_cast<cudaStream_t>(stream)) == cudaSuccess ? DOE_OK
                                                                                                     : DOE_ECUDA;
}

extern "C" size_t doe_radial_workspace_bytes(int n_c) {
  if (n_c < 1 || n_c > doe::kMaxRadial) return 0;
  return (size_t)doe::kRadialBlocks * n_c * sizeof(double);
}

extern "C" int doe_radial_grad(int n, int n_c, const float* grad_h, float* c_grad, void* ws, size_t ws_bytes,
                               void* stream) {
  if (!grad_h || !c_grad || !radial_size_ok(n, n_c)) return DOE_EINVAL;
  if (!ws || ws_bytes < doe_radial_workspace_bytes(n_c) || (reinterpret_cast<uintptr_t>(ws) & 7u)) return DOE_ENOWS;
  return doe::launch_radial_grad(grad_h, n_c, n, static_cast<double*>(ws), c_grad,
                                 static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? DOE_OK
             : DOE_ECUDA;
}
