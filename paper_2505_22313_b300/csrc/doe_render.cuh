// doe_render.cuh -- image formation by PSF convolution (the imaging application's model
// behind Eq. 9): out_c = img_c (*) k_c, linear convolution with zero boundary and a "same"
// output window, computed with 2H x 2W transforms and real-data packing:
//   R1  per image row u (channel c): z = img_c[u] + i k_c[u] (both real, zero-padded to 2W),
//       one complex FFT of length 2W, then the two real spectra are separated in the CTA,
//       X_img[k] = (Z[k] + conj Z[2W-k]) / 2, X_k[k] = (Z[k] - conj Z[2W-k]) / (2i), k <= W,
//       and written to SA, SB (column-tiled, H rows).  The crop k_c is read straight from the PSF
//       around the optical axis; its row sums go to ksum[c][u] (FP64).
//   R2  per column k <= W (4-column cluster, as the propagation's column pass): each CTA reads
//       its columns of SA and SB directly, column FFTs (zero-padded to 2H), product, column
//       IFFT, rows [H/2, 3H/2) gathered across the cluster -> SC.
//   R3  per pair of output rows: the two Hermitian half spectra are packed as X0 + i X1,
//       extended to 2W by conjugate symmetry, one complex IFFT, real part = row y, imaginary
//       part = row y + 1, window [W/2, 3W/2), scaled by 1 / (4 H W sum(k_c)).
// The same three kernels run Wiener deconvolution (Eq. 9, circular model, RENDER_WIENER) on
// H x W transforms without padding: R1 packs the blurred row with the (unshifted) crop row;
// R2 replaces the product by the filter conj(K) Y / (|K|^2 + gamma) with K = FFT2(crop) /
// sum(crop) times (-1)^(l + k) (the crop's centre moved to the origin), and keeps all H rows;
// R3 keeps all W columns and scales by 1 / (H W).
#pragma once
#include <cooperative_groups.h>

#include "doe_internal.cuh"
#include "doe_render_args.h"

namespace doe {



// R1: one CTA per (row u, channel c); transform length L = 2W.
template <int L, bool WIENER>
__global__ void __launch_bounds__(L / 32) render_rows_kernel(const __grid_constant__ RenderArgs ra) {
  using F = First<L, false>;
  using G = Last<L, false>;
  constexpr int T = L / 32;
  extern __shared__ float2 sm[];
  __shared__ double red[32];
  const int u = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
  const int W = ra.W, H = ra.H;
  const float* irow = ra.img + ((size_t)c * H + u) * W;
  const float* krow = ra.psf + ((size_t)c * ra.Py + (ra.Py / 2 - H / 2 + u)) * ra.Px + (ra.Px / 2 - W / 2);
  float2 v[32];
  double ks = 0.0;
#pragma unroll
  for (int b = 0; b < F::B; b += 2)
#pragma unroll
    for (int r = 0; r < F::R; ++r) {
      const int n = F::idx(t, b, r);  // even
      float2 a = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
      if (n < W && DOE_IN(((size_t)c * H + u) * W + n + 1, ra.n_img) &&
          DOE_IN(((size_t)c * ra.Py + (ra.Py / 2 - H / 2 + u)) * ra.Px + (ra.Px / 2 - W / 2) + n + 1, ra.n_psf)) {
        const float2 iv = __ldcs(reinterpret_cast<const float2*>(irow + n));
        const float2 kv = __ldcs(reinterpret_cast<const float2*>(krow + n));
        a = make_float2(iv.x, kv.x);
        d = make_float2(iv.y, kv.y);
        ks += (double)kv.x + (double)kv.y;
      }
      v[b * F::R + r] = a;
      v[(b + 1) * F::R + r] = d;
    }
  fft_run<L, 32, false>(v, t, sm);
  __syncthreads();
  float4* s4 = reinterpret_cast<float4*>(sm);
#pragma unroll
  for (int b = 0; b < G::B; b += 2)
#pragma unroll
    for (int r = 0; r < G::R; ++r) {
      const float2 a = v[b * G::R + r], d = v[(b + 1) * G::R + r];
      if (DOE_IN(swz(G::idx(t, b, r) >> 1), L / 2)) s4[swz(G::idx(t, b, r) >> 1)] = make_float4(a.x, a.y, d.x, d.y);
    }
  __syncthreads();
  float2* sa = ra.sa + (size_t)c * H * ra.wpr;
  float2* sb = ra.sb + (size_t)c * H * ra.wpr;
  for (int k = t; k <= (WIENER ? W / 2 : W); k += T) {  // the L / 2 + 1 stored columns
    const float2 zk = sm[phys(k)];
    const float2 zm = sm[phys((L - k) & (L - 1))];
    // X_img = (Z[k] + conj Z[-k]) / 2, X_k = (Z[k] - conj Z[-k]) / (2i)
    const size_t o = tiled_at(u, k, H, kTile);
    if (!DOE_IN((size_t)c * H * ra.wpr + o, ra.n_s)) continue;
    sa[o] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    sb[o] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
  const double tot = block_sum<T>(ks, red);
  if (t == 0 && DOE_IN((size_t)c * H + u, ra.n_ksum)) ra.ksum[(size_t)c * H + u] = tot;
}

// Loads column `col` of a column-tiled buffer (n rows, 4-wide tiles) into the first-stage
// registers of a length-L forward transform; rows n..L-1 are zero padding.  A register pair
// (rows e, e + 1; e even, n even) is two 8-byte loads 32 bytes apart.
template <int L>
__device__ __forceinline__ void load_tiled_col(float2 (&v)[32], int t, const float2* col, int n, bool live,
                                               size_t col_off, long long extent) {
  using F = First<L, false>;
  static_assert(F::PAIRED, "first stage holds adjacent pairs");
#pragma unroll
  for (int b = 0; b < F::B; b += 2)
#pragma unroll
    for (int r = 0; r < F::R; ++r) {
      const int y = F::idx(t, b, r);
      float2 a = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
      if (live && y < n && DOE_IN(col_off + (size_t)(y + 1) * kTile, extent)) {
        a = __ldcs(col + (size_t)y * kTile);
        d = __ldcs(col + (size_t)(y + 1) * kTile);
      }
      v[b * F::R + r] = a;
      v[(b + 1) * F::R + r] = d;
    }
}

// R2: cluster of kTile CTAs per 4 adjacent columns of one channel; transform length L = 2H.
// CTA q reads its own column of SA and of SB straight into registers, keeps the image column's
// spectrum in sma while the kernel column is transformed in smb, multiplies, inverse-transforms,
// and the cluster gathers rows [H/2, 3H/2) of its four columns as 32-byte row segments of SC.
// From 1024 to 4096 points the two buffers let 384 threads (3 CTAs at 4096 points) share an SM, and
// the registers are capped to match, 168 per thread (without the cap the two spectra and their
// product take 230: 2 CTAs).
template <int L, bool WIENER>
__global__ void __launch_bounds__(L / 32, L >= 1024 && L <= 4096 ? 12288 / L : 1) render_cols_kernel(const __grid_constant__ RenderArgs ra) {
  using G = Last<L, false>;
  using Hh = Last<L, true>;
  constexpr int T = L / 32;
  constexpr int F4 = kTile / 2;
  static_assert(F4 == 2, "two column pairs per tile");
  extern __shared__ float2 sm[];
  float2* sma = sm;
  float2* smb = sm + L;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int t = threadIdx.x;
  const int H = ra.H;
  const int tiles = ra.wpr / kTile;
  const int tile = (blockIdx.x / kTile) % tiles;
  const int c = (blockIdx.x / kTile) / tiles;
  const int pos0 = tile * kTile, mypos = pos0 + q;
  const bool live = mypos < ra.nk;  // columns past the half spectrum are unused
  constexpr bool wiener = WIENER;
  float ks = 0.f;  // Wiener: sum of the crop, in a fixed order (FP64)
  if constexpr (wiener) {
    __shared__ double red[32];
    double a = 0.0;
    for (int u = t; u < H; u += T) a += ra.ksum[(size_t)c * H + u];
    a = block_sum<T>(a, red);  // the total is in thread 0
    if (t == 0) red[0] = a;
    __syncthreads();
    ks = (float)red[0];
  }
  const float2* colA = ra.sa + (size_t)c * H * ra.wpr + tiled_at(0, mypos, H, kTile);
  const float2* colB = ra.sb + (size_t)c * H * ra.wpr + tiled_at(0, mypos, H, kTile);
  float2* baseC = ra.sc + (size_t)c * H * ra.wpr;
  float2 v[32];
  // spectrum of the image column, kept in sma at its own register positions
  load_tiled_col<L>(v, t, colA, H, live, (size_t)c * H * ra.wpr + tiled_at(0, mypos, H, kTile), ra.n_s);
  fft_run<L, 32, false>(v, t, sma);
  __syncthreads();
  {
    float4* s4 = reinterpret_cast<float4*>(sma);
#pragma unroll
    for (int b = 0; b < G::B; b += 2)
#pragma unroll
      for (int r = 0; r < G::R; ++r) {
        const float2 a = v[b * G::R + r], d = v[(b + 1) * G::R + r];
        if (DOE_IN(swz(G::idx(t, b, r) >> 1), L / 2)) s4[swz(G::idx(t, b, r) >> 1)] = make_float4(a.x, a.y, d.x, d.y);
      }
  }
  // spectrum of the kernel column, times the image spectrum (same thread, same positions), or
  // the Wiener filter sign conj(K) ks Y / (|K|^2 + gamma ks^2) with K unnormalised
  load_tiled_col<L>(v, t, colB, H, live, (size_t)c * H * ra.wpr + tiled_at(0, mypos, H, kTile), ra.n_s);
  fft_run<L, 32, false>(v, t, smb);
  {
    const float4* s4 = reinterpret_cast<const float4*>(sma);
    if constexpr (!wiener) {
#pragma unroll
      for (int b = 0; b < G::B; b += 2)
#pragma unroll
        for (int r = 0; r < G::R; ++r) {
          const float4 a = DOE_IN(swz(G::idx(t, b, r) >> 1), L / 2) ? s4[swz(G::idx(t, b, r) >> 1)] : make_float4(0.f, 0.f, 0.f, 0.f);
          v[b * G::R + r] = cmul(v[b * G::R + r], make_float2(a.x, a.y));
          v[(b + 1) * G::R + r] = cmul(v[(b + 1) * G::R + r], make_float2(a.z, a.w));
        }
    } else {
      const float g2 = ra.gamma * ks * ks;
      const float s0 = (mypos & 1) ? -ks : ks;  // rows l even, column mypos: sign (-1)^(l + k)
#pragma unroll
      for (int b = 0; b < G::B; b += 2)
#pragma unroll
        for (int r = 0; r < G::R; ++r) {
          const float4 a = DOE_IN(swz(G::idx(t, b, r) >> 1), L / 2) ? s4[swz(G::idx(t, b, r) >> 1)] : make_float4(0.f, 0.f, 0.f, 0.f);
          float2& k0 = v[b * G::R + r];        // row l = idx (even)
          float2& k1 = v[(b + 1) * G::R + r];  // row l + 1: opposite sign
          const float f0 = s0 / fmaf(k0.x, k0.x, fmaf(k0.y, k0.y, g2));
          const float f1 = -s0 / fmaf(k1.x, k1.x, fmaf(k1.y, k1.y, g2));
          k0 = cscale(cmulc(make_float2(a.x, a.y), k0), f0);
          k1 = cscale(cmulc(make_float2(a.z, a.w), k1), f1);
        }
    }
  }
  fft_run<L, 32, true>(v, t, smb);
  __syncthreads();
  {
    float4* s4 = reinterpret_cast<float4*>(smb);
#pragma unroll
    for (int b = 0; b < Hh::B; b += 2)
#pragma unroll
      for (int r = 0; r < Hh::R; ++r) {
        const float2 a = v[b * Hh::R + r], d = v[(b + 1) * Hh::R + r];
        if (DOE_IN(swz(Hh::idx(t, b, r) >> 1), L / 2)) s4[swz(Hh::idx(t, b, r) >> 1)] = make_float4(a.x, a.y, d.x, d.y);
      }
  }
  const float4* rsb[kTile];
#pragma unroll
  for (int cc = 0; cc < kTile; ++cc) rsb[cc] = reinterpret_cast<const float4*>(cl.map_shared_rank(smb, cc));
  cl.sync();  // all four columns are in shared memory (and every CTA of the cluster has started)
  {
    // rows [H/2, 3H/2) (render) or [0, H) (Wiener) of the column IFFT -> SC rows [0, H); item
    // = (pair of output rows, column pair f), all remote loads issued before the first store
    constexpr int IT = ((WIENER ? L : L / 2) / kTile / 2) * F4 / T;  // H = L (Wiener) or L / 2 rows
    constexpr int CH = IT < 4 ? IT : 4;           // items whose loads are in flight together
    const int rows = H / kTile, rbeg = q * rows, lim = (rows / 2) * F4;
    const int r0 = wiener ? 0 : H / 2;
#pragma unroll
    for (int c0 = 0; c0 < IT; c0 += CH) {
      float4 a[CH], b[CH];
#pragma unroll
      for (int it = 0; it < CH; ++it) {
        const int idx = t + (c0 + it) * T, f = idx & 1;
        if (idx < lim) {
          const int ch = swz((r0 + rbeg + 2 * (idx / F4)) >> 1);
          a[it] = b[it] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (DOE_IN(ch, L / 2)) {
            a[it] = (f ? rsb[2] : rsb[0])[ch];  // rows rr, rr + 1 of column 2f
            b[it] = (f ? rsb[3] : rsb[1])[ch];  // of column 2f + 1
          }
        }
      }
#pragma unroll
      for (int it = 0; it < CH; ++it) {
        const int idx = t + (c0 + it) * T, f = idx & 1;
        if (idx < lim &&
            DOE_IN((size_t)c * H * ra.wpr + (size_t)(rbeg + 2 * (idx / F4) + 1) * ra.wpr + pos0 + 2 * f + 1, ra.n_s)) {
          float2* dst = baseC + (size_t)(rbeg + 2 * (idx / F4)) * ra.wpr + pos0 + 2 * f;
          __stcs(reinterpret_cast<float4*>(dst), make_float4(a[it].x, a[it].y, b[it].x, b[it].y));
          __stcs(reinterpret_cast<float4*>(dst + ra.wpr), make_float4(a[it].z, a[it].w, b[it].z, b[it].w));
        }
      }
    }
  }
  cluster_sync_relaxed();  // peers have finished reading this CTA's shared memory
}

// R3: one CTA per (pair of output rows, channel); transform length L = 2W.
template <int L, bool WIENER>
__global__ void __launch_bounds__(L / 32) render_out_kernel(const __grid_constant__ RenderArgs ra) {
  using F = First<L, true>;
  using Hh = Last<L, true>;
  constexpr int T = L / 32;
  extern __shared__ float2 sm[];
  __shared__ double red[32];
  const int y = 2 * blockIdx.x, c = blockIdx.y, t = threadIdx.x;
  const int W = ra.W, H = ra.H;
  const float2* x0 = ra.sc + ((size_t)c * H + y) * ra.wpr;
  const float2* x1 = x0 + ra.wpr;
  constexpr bool wiener = WIENER;
  // render: sum of the kernel crop (fixed order, FP64); Wiener: normalised in R2 already
  double ks = 1.0;
  if constexpr (!wiener) {
    ks = 0.0;
    for (int u = t; u < H; u += T) ks += ra.ksum[(size_t)c * H + u];
    ks = block_sum<T>(ks, red);
    if (t == 0) red[0] = ks;
    __syncthreads();
    ks = red[0];
  }
  const float scale = (float)(1.0 / ((double)L * (wiener ? (double)H : 2.0 * H) * ks));
  float2 v[32];
#pragma unroll
  for (int b = 0; b < F::B; ++b)
#pragma unroll
    for (int r = 0; r < F::R; ++r) {
      const int k = F::idx(t, b, r);
      float2 a, d;  // X0[k], X1[k] with Hermitian extension above L / 2
      if (!DOE_IN(((size_t)c * H + y + 1) * ra.wpr + (k <= L / 2 ? k : L - k), ra.n_s)) {
        a = d = make_float2(0.f, 0.f);
      } else if (k <= L / 2) {
        a = x0[k];
        d = x1[k];
      } else {
        a = x0[L - k];
        d = x1[L - k];
        a.y = -a.y;
        d.y = -d.y;
      }
      v[b * F::R + r] = make_float2(a.x - d.y, a.y + d.x);  // X0 + i X1
    }
  fft_run<L, 32, true>(v, t, sm);
  float* o0 = ra.out + ((size_t)c * H + y) * W;
  float* o1 = o0 + W;
#pragma unroll
  for (int b = 0; b < Hh::B; b += 2)
#pragma unroll
    for (int r = 0; r < Hh::R; ++r) {
      const int n = Hh::idx(t, b, r) - (L - W) / 2;  // even; window offset W/2 (render) or 0
      if ((unsigned)n < (unsigned)W && DOE_IN(((size_t)c * H + y + 1) * W + n + 1, ra.n_out)) {
        const float2 a = v[b * Hh::R + r], d = v[(b + 1) * Hh::R + r];
        __stcs(reinterpret_cast<float2*>(o0 + n), make_float2(a.x * scale, d.x * scale));
        __stcs(reinterpret_cast<float2*>(o1 + n), make_float2(a.y * scale, d.y * scale));
      }
    }
}

}  // namespace doe
