// doe_design.cu -- one step of the design optimiser: Adam (Kingma & Ba 2015, the optimiser the
// paper uses for its designs, Sec. 4's toy example and the applications of Sec. 5) on the
// height map with the gradient from doe_grad, followed by a projection onto the fabricable
// height range [h_min, h_max].  Elementwise, one thread per height sample, FP32 state.
#include <cuda_runtime.h>

#include <cmath>

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
