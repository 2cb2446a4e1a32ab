// compare_cufft.cu -- the PSF chain built from cuFFT, for comparison in the benchmark only.
// Not part of libdoe (it is linked into a separate libdoe_cufft.so that the product never
// loads).  Same physics and precision handling as libdoe, unfused: per wavelength a full
// P x P complex64 field is padded, transformed by cufftExecC2C, multiplied by the transfer
// function, transformed back and squared, each step a separate launch over the whole grid.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <map>
#include <mutex>

#include "doe.h"
#include "doe_internal.cuh"

namespace {
using namespace doe;

__global__ void pad_transmittance(float2* f, const float* h, int N, int P, int off, float kp_hi, float kp_lo) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)P * P) return;
  const int y = (int)(i / P), x = (int)(i % P);
  const int r = y - off, c = x - off;
  f[i] = ((unsigned)r < (unsigned)N && (unsigned)c < (unsigned)N) ? transmittance(h[(size_t)r * N + c], kp_hi, kp_lo)
                                                                    : make_float2(0.f, 0.f);
}

__global__ void apply_transfer(float2* f, int P, Slice s) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)P * P) return;
  const int l = (int)(i / P), k = (int)(i % P);
  const int a = l < P / 2 ? l : P - l, b = k < P / 2 ? k : P - k;
  float2 v = make_float2(0.f, 0.f);
  const long long m = (long long)a * a + (long long)b * b;
  if (a <= s.kmax && b <= s.kmax && m < s.mev) v = cmul(f[i], transfer_value((unsigned)m, s));
  f[i] = v;
}

__global__ void intensity(const float2* f, float* out, size_t n, float s) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 e = cscale(f[i], s);
  out[i] = fmaf(e.x, e.x, e.y * e.y);
}

std::mutex g_mu;
std::map<int, cufftHandle> g_plans;

void split(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}
}  // namespace

// PSFs [n_lambda][P][P] of geometry g with cuFFT; ws must hold P * P complex64.
extern "C" int doe_cufft_psf(const doe_geom* g, const float* h, float* psf, void* ws, size_t ws_bytes, void* stream) {
  const int N = g->nx, P = g->pad * g->nx, off = (P - N) / 2;
  if (ws_bytes < (size_t)P * P * sizeof(float2)) return DOE_ENOWS;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cufftHandle plan;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(P);
    if (it == g_plans.end()) {
      if (cufftPlan2d(&plan, P, P, CUFFT_C2C) != CUFFT_SUCCESS) return DOE_ECUDA;
      g_plans[P] = plan;
    } else {
      plan = it->second;
    }
  }
  if (cufftSetStream(plan, st) != CUFFT_SUCCESS) return DOE_ECUDA;
  float2* f = static_cast<float2*>(ws);
  const size_t n = (size_t)P * P;
  const int TB = 256;
  const unsigned nb = (unsigned)((n + TB - 1) / TB);
  int32_t kmax[64];
  int64_t mev[64];
  if (doe_band_limits(g, kmax, mev) != DOE_OK) return DOE_EINVAL;
  for (int j = 0; j < g->n_lambda; ++j) {
    const double lam = g->lambda[j], du = 1.0 / ((double)P * g->dx), kPi = 3.14159265358979323846;
    Slice s = {};
    s.kmax = kmax[j];
    s.mev = mev[j];
    split((lam * du) * (lam * du), s.c_hi, s.c_lo);
    const double phi0 = 2.0 * kPi * g->z / lam;
    split(phi0, s.phi0_hi, s.phi0_lo);
    split(std::fmod(phi0, 2.0 * kPi), s.th0_hi, s.th0_lo);
    split(2.0 * kPi * (g->n_index[j] - 1.0) / lam, s.kp_hi, s.kp_lo);
    pad_transmittance<<<nb, TB, 0, st>>>(f, h, N, P, off, s.kp_hi, s.kp_lo);
    if (cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(f), reinterpret_cast<cufftComplex*>(f), CUFFT_FORWARD) != CUFFT_SUCCESS)
      return DOE_ECUDA;
    apply_transfer<<<nb, TB, 0, st>>>(f, P, s);
    if (cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(f), reinterpret_cast<cufftComplex*>(f), CUFFT_INVERSE) != CUFFT_SUCCESS)
      return DOE_ECUDA;
    intensity<<<nb, TB, 0, st>>>(f, psf + (size_t)j * n, n, (float)(1.0 / ((double)P * P)));
  }
  return cudaGetLastError() == cudaSuccess ? DOE_OK : DOE_ECUDA;
}
