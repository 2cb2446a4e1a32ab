// doe_misc.cuh -- the small non-transform kernels: the transfer-function table, the loss
// reduction, the design-loop kernels (Adam, Lanczos-3 and nearest upsampling adjoints, the
// radial parameterisation) and the band-mask debug view.  Included by doe_launch.cu only.
#pragma once
#include "doe_kernels.cuh"

namespace doe {

// ------------------------------------------------------------------ transfer-function table
// Grid (max_kmax + 1, S); row b = |kt|, entries a = |lt| (at htab_col).  Integer band logic: the table
// covers |kt|, |lt| <= kmax; a sample is zero iff kt^2 + lt^2 >= mev (evanescent).
__global__ void __launch_bounds__(256) htab_kernel(const __grid_constant__ Batch bt) {
  const Slice& sl = bt.s[blockIdx.y];
  const int b = blockIdx.x;  // |kt| (row frequency)
  if (b > sl.kmax) return;
  float2* row = sl.htab + (size_t)b * sl.hp;
  const bool square = sl.sqa == 1 && sl.sqb == 1;
  for (int a = threadIdx.x; a <= sl.kmax_y; a += blockDim.x) {  // a = |lt| (column frequency)
    const long long m = (long long)b * b * sl.sqb + (long long)a * a * sl.sqa;
    if (DOE_IN((size_t)b * sl.hp + htab_col(sl, a), sl.n_htab))
      row[htab_col(sl, a)] = m >= sl.mev ? make_float2(0.f, 0.f)
                             : square    ? transfer_value((unsigned int)m, sl)
                                         : transfer_value64((unsigned long long)m, sl);
  }
}

// Adjoint of nearest upsampling by f = 2^uf: the layout gradient is the sum of the simulation-
// grid gradient over each f x f block, in a fixed order.  One thread per layout cell.
__global__ void __launch_bounds__(256) upsample_adjoint_kernel(const float* __restrict__ g, float* __restrict__ gc,
                                                              int N, int uf) {
  const int nc = N >> uf, f = 1 << uf;
  const long long cell = blockIdx.x * 256LL + threadIdx.x;
  if (cell >= (long long)nc * nc) return;
  const int ic = (int)(cell / nc), xc = (int)(cell % nc);
  float acc = 0.f;
  for (int di = 0; di < f; ++di) {
    const float* row = g + (size_t)(ic * f + di) * N + (size_t)xc * f;
    for (int dx = 0; dx < f; ++dx) acc += row[dx];
  }
  gc[cell] = acc;
}

// One Adam step on the height map (Kingma & Ba 2015), then projection onto [h_min, h_max]:
//   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
//   h = clamp(h - lr_hat m / (sqrt(v) + eps_hat))
// with the bias corrections folded into lr_hat and eps_hat by the caller.
__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ h, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, long long n,
                                                   float lr_hat, float beta1, float beta2, float eps_hat,
                                                   float h_min, float h_max) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(beta1, m[i] - gi, gi);            // beta1 m + (1 - beta1) g
  const float vi = fmaf(beta2, v[i] - gi * gi, gi * gi);  // beta2 v + (1 - beta2) g^2
  m[i] = mi;
  v[i] = vi;
  const float hi = h[i] - lr_hat * mi / (sqrtf(vi) + eps_hat);
  h[i] = fminf(fmaxf(hi, h_min), h_max);
}

// Lanczos-3 interpolation of the (nl x nl) height layout onto the N x N simulation grid,
// separable with the tap table tb, in two passes through an [nl][N] buffer (the row sums of
// each layout row, then the column sums; the same order of operations as the 2-D sum taken
// row by row).  One thread per output element.
__global__ void __launch_bounds__(256) lanczos_up_rows_kernel(const float* __restrict__ hl, float* __restrict__ tmp,
                                                             int N, const __grid_constant__ LanczosTab tb) {
  const long long e = blockIdx.x * 256LL + threadIdx.x;
  if (e >= (long long)tb.nl * N) return;
  const int m = (int)(e / N), x = (int)(e % N);
  const int f = tb.f, nl = tb.nl, rx = x & (f - 1), mx = x / f + tb.off[rx];
  const float* row = hl + (size_t)m * nl;
  float s = 0.f;
#pragma unroll
  for (int dx = 0; dx < 6; ++dx) s = fmaf(tb.w[rx][dx], __ldg(row + min(max(mx + dx, 0), nl - 1)), s);
  tmp[e] = s;
}
__global__ void __launch_bounds__(256) lanczos_up_cols_kernel(const float* __restrict__ tmp, float* __restrict__ hs,
                                                             int N, const __grid_constant__ LanczosTab tb) {
  const long long idx = blockIdx.x * 256LL + threadIdx.x;
  if (idx >= (long long)N * N) return;
  const int i = (int)(idx / N), x = (int)(idx % N);
  const int f = tb.f, nl = tb.nl, ri = i & (f - 1), my = i / f + tb.off[ri];
  float acc = 0.f;
#pragma unroll
  for (int dy = 0; dy < 6; ++dy) acc = fmaf(tb.w[ri][dy], __ldg(tmp + (size_t)min(max(my + dy, 0), nl - 1) * N + x), acc);
  hs[idx] = acc;
}

// Weight of layout cell m in simulation sample i's interpolation (taps clamped to the layout).
__device__ __forceinline__ float lanczos_coef(const LanczosTab& tb, int i, int m) {
  const int r = i & (tb.f - 1), n0 = i / tb.f + tb.off[r];
  float c = 0.f;
#pragma unroll
  for (int d = 0; d < 6; ++d)
    if (min(max(n0 + d, 0), tb.nl - 1) == m) c += tb.w[r][d];
  return c;
}

// Adjoint of lanczos_up_kernel, separable like the interpolation (gl = W^T g W), in two
// fixed-order passes through a [N][nl] buffer: rows first, tmp[i][n] = sum_x w(x, n) g[i][x],
// then columns, gl[m][n] = sum_i w(i, m) tmp[i][n]; the samples whose taps reach cell n are
// x in [f (n - 3), f (n + 4)) (edge clamping included).  One thread per output element.
__global__ void __launch_bounds__(256) lanczos_adjoint_rows_kernel(const float* __restrict__ g, float* __restrict__ tmp,
                                                                  int N, const __grid_constant__ LanczosTab tb) {
  const long long e = blockIdx.x * 256LL + threadIdx.x;
  if (e >= (long long)N * tb.nl) return;
  const int i = (int)(e / tb.nl), n = (int)(e % tb.nl), f = tb.f;
  const int x0 = max(0, f * (n - 3)), x1 = min(N, f * (n + 4));
  const float* gr = g + (size_t)i * N;
  float s = 0.f;
  for (int x = x0; x < x1; ++x) s = fmaf(lanczos_coef(tb, x, n), __ldg(gr + x), s);
  tmp[e] = s;
}
__global__ void __launch_bounds__(256) lanczos_adjoint_cols_kernel(const float* __restrict__ tmp, float* __restrict__ gl,
                                                                  int N, const __grid_constant__ LanczosTab tb) {
  const long long cell = blockIdx.x * 256LL + threadIdx.x;
  if (cell >= (long long)tb.nl * tb.nl) return;
  const int m = (int)(cell / tb.nl), n = (int)(cell % tb.nl), f = tb.f;
  const int i0 = max(0, f * (m - 3)), i1 = min(N, f * (m + 4));
  float s = 0.f;
  for (int i = i0; i < i1; ++i) s = fmaf(lanczos_coef(tb, i, m), __ldg(tmp + (size_t)i * tb.nl + n), s);
  gl[cell] = s;
}

// ------------------------------------------------------------------ radial parameterisation
// Squared normalised radius s = ((i - N/2)^2 + (x - N/2)^2) / (N/2)^2 of sample idx = i N + x,
// as a float pair: the integer numerator is split into two exactly representable parts and
// multiplied by (N/2)^-2 = inv_hi + inv_lo (FP64 on the host; a power of two when N is).
__device__ __forceinline__ dfl radial_s(long long idx, int N, float inv_hi, float inv_lo) {
  const int i = (int)(idx / N) - N / 2, x = (int)(idx % N) - N / 2;
  const unsigned int m = (unsigned int)(i * i) + (unsigned int)(x * x);  // <= 2^31
  const dfl inv = {inv_hi, inv_lo};
  return df_add(df_mul_f(inv, (float)(m & 0xFFFFF000u)), df_mul_f(inv, (float)(m & 0x00000FFFu)));
}

// Radially symmetric heights h = sum_k c[k] s^k (Horner in double-float, rounded once).
__global__ void __launch_bounds__(256) radial_heights_kernel(const float* __restrict__ c, int n_c, int N,
                                                            float inv_hi, float inv_lo, float* __restrict__ h) {
  const long long idx = blockIdx.x * 256LL + threadIdx.x;
  if (idx >= (long long)N * N) return;
  const dfl s = radial_s(idx, N, inv_hi, inv_lo);
  dfl acc = {__ldg(c + n_c - 1), 0.f};
  for (int k = n_c - 2; k >= 0; --k) acc = df_add(df_mul(acc, s), {__ldg(c + k), 0.f});
  h[idx] = __fadd_rn(acc.hi, acc.lo);
}

// Transpose of radial_heights_kernel, first stage: CTA b writes part[b][k] = the sum of
// g s^k over its grid-stride share of the samples (double-float terms and per-thread sums,
// then a fixed-order FP64 block sum).
__global__ void __launch_bounds__(256) radial_grad_kernel(const float* __restrict__ g, int n_c, int N, float inv_hi,
                                                         float inv_lo, double* __restrict__ part) {
  __shared__ double red[32];
  dfl acc[kMaxRadial];
#pragma unroll
  for (int k = 0; k < kMaxRadial; ++k) acc[k] = {0.f, 0.f};
  const long long n = (long long)N * N, step = (long long)gridDim.x * 256;
  for (long long idx = blockIdx.x * 256LL + threadIdx.x; idx < n; idx += step) {
    const dfl s = radial_s(idx, N, inv_hi, inv_lo);
    dfl p = {__ldcs(g + idx), 0.f};  // g s^k
#pragma unroll
    for (int k = 0; k < kMaxRadial; ++k)
      if (k < n_c) {
        acc[k] = df_add(acc[k], p);
        p = df_mul(p, s);
      }
  }
#pragma unroll
  for (int k = 0; k < kMaxRadial; ++k)
    if (k < n_c) {
      const double tot = block_sum<256>((double)acc[k].hi + (double)acc[k].lo, red);
      if (threadIdx.x == 0) part[(size_t)blockIdx.x * n_c + k] = tot;
    }
}

// Second stage: c_grad[k] = sum over the CTAs of part[b][k], in CTA order.
__global__ void radial_grad_final_kernel(const double* __restrict__ part, int blocks, int n_c, float* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= n_c) return;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += part[(size_t)b * n_c + k];
  out[k] = (float)s;
}

// Sum of the per-row loss partials of all slices, in a fixed order (one CTA).
__global__ void __launch_bounds__(1024) loss_reduce_kernel(const __grid_constant__ Batch bt, double* loss) {
  __shared__ double red[32];
  double acc = 0.0;
  const int n = bt.Py * bt.qf;  // per-row of the Py output rows (and, for split rows, per-CTA) partials
  for (int j = 0; j < bt.S; ++j)
    for (int y = threadIdx.x; y < n; y += 1024)
      if (DOE_IN(y, bt.s[j].n_loss)) acc += bt.s[j].loss_part[y];
  const double tot = block_sum<1024>(acc, red);
  if (threadIdx.x == 0) *loss = bt.mode == GRAD_L2 ? tot : 0.0;
}

// Debug: band mask of slice 0 read back from its transfer table, [P][P] uint8 in FFT order.
__global__ void band_mask_kernel(const __grid_constant__ Batch bt, uint8_t* mask) {
  const Slice& sl = bt.s[0];
  const int l = blockIdx.x;  // row of the [Py][Px] mask: column frequency lt
  const int P = bt.P;
  const int a = abs_signed(l, bt.Py);
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const int b = abs_signed(k, P);
    uint8_t mv = 0;
    if (a <= sl.kmax_y && b <= sl.kmax) {
      const float2 hv = DOE_IN((size_t)b * sl.hp + htab_col(sl, a), sl.n_htab) ? sl.htab[(size_t)b * sl.hp + htab_col(sl, a)]
                                                                           : make_float2(0.f, 0.f);
      mv = (hv.x != 0.f || hv.y != 0.f) ? 1 : 0;
    }
    mask[(size_t)l * P + k] = mv;
  }
}

// Check of the bounded waits' failure path: one CTA announces 16 bytes of copies on an mbarrier
// and issues none, so the phase never completes; every thread's wait gives up after `polls`
// polls and the fault word records DOE_FAULT_WAIT_TIMEOUT.  No copy is in flight when it exits.
__global__ void __launch_bounds__(32) wait_check_kernel(unsigned polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_arrive_expect_tx(&bar, 16);
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0, polls) && threadIdx.x == 0) raise_fault(FAULT_WAIT_TIMEOUT);
}

}  // namespace doe
