// doe_kernels.cuh -- the passes of the propagation, its adjoint and the band-table builder.
//
// Forward PSF, per (request, wavelength) slice, padded side P, DOE side N, offset off:
//   table  H(|kt|, |lt|) for |kt|, |lt| <= kmax                        (Eq. 3's H_lambda)
//   A      per DOE row i: E_doe = exp(+i k' h) E_in on the fly (Eq. 1-2), zero-padded row FFT,
//          keep the band columns -> buf rows [0, N)                    (I1)
//   B      per band column (4-column cluster): column FFT of the N non-zero rows (zeros
//          elsewhere), times H, column IFFT -> buf rows [0, P)         (I2, in place)
//   C      per output row y: row IFFT of the band columns, 1/P^2, |.|^2 -> PSF row
// Adjoint (gradient), same buffer in place:
//   C'     per row y: row IFFT, E, g = 2 (I - T) E or (dL/dI) E, row FFT -> buf rows [0, P)  (J1)
//   B*     per column: column FFT of all P rows, times conj(H), column IFFT, keep the DOE
//          rows [off, off + N) -> buf rows [0, N)                                           (J2)
//   A*     per DOE row i: row IFFT, crop to the DOE window, -2 k' Im(conj(g) E_doe), summed
//          over the wavelengths of the request -> grad_h row i
#pragma once
#include <cooperative_groups.h>

#include "doe_internal.cuh"

namespace doe {
namespace cg = cooperative_groups;

// ------------------------------------------------------------------ transfer-function table
// Grid (max_kmax + 1, S); row b = |kt|, entries a = |lt|.  Integer band logic: the table
// covers |kt|, |lt| <= kmax; a sample is zero iff kt^2 + lt^2 >= mev (evanescent).
__global__ void __launch_bounds__(256) htab_kernel(const __grid_constant__ Batch bt) {
  const Slice& sl = bt.s[blockIdx.y];
  const int b = blockIdx.x;
  if (b > sl.kmax) return;
  float2* row = sl.htab + (size_t)b * sl.hp;
  for (int a = threadIdx.x; a <= sl.kmax; a += blockDim.x) {
    const long long m = (long long)b * b + (long long)a * a;
    row[a] = (m < sl.mev) ? transfer_value((unsigned int)m, sl) : make_float2(0.f, 0.f);
  }
}

// ------------------------------------------------------------------ pass A: DOE rows
template <int L>
__global__ void __launch_bounds__(L / elems_for(L)) pass_a_kernel(const __grid_constant__ Batch bt) {
  constexpr int E = elems_for(L), T = L / E;
  constexpr int R0 = first_radix<L, false>(), B0 = E / R0;
  constexpr int RL = last_radix<L, false>(), BL = E / RL;
  extern __shared__ float2 sm[];
  const Slice& sl = bt.s[blockIdx.y];
  const int i = blockIdx.x;
  const int t = threadIdx.x;
  const int N = bt.N, off = bt.off;
  const float* hrow = sl.h + (size_t)i * N;
  const float2* erow = sl.e_in ? sl.e_in + (size_t)i * N : nullptr;
  float2 v[E];
#pragma unroll
  for (int b = 0; b < B0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int x = t + b * T + r * (L / R0) - off;
      float2 val = make_float2(0.f, 0.f);
      if ((unsigned)x < (unsigned)N) {
        val = transmittance(__ldg(hrow + x), sl.kp_hi, sl.kp_lo);
        if (erow) val = cmul(val, erow[x]);
      }
      v[b * R0 + r] = val;
    }
  fft_run<L, E, false>(v, t, sm);
  float2* dst = sl.buf + (size_t)i * sl.wp;
#pragma unroll
  for (int b = 0; b < BL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int pos = band_pos(t + b * T + r * (L / RL), L, sl.kmax, sl.w);
      if (pos >= 0) dst[pos] = v[b * RL + r];
    }
}

// ------------------------------------------------------------------ pass B / B*: columns
// A cluster of kTile CTAs owns kTile adjacent stored columns; CTA q transforms column q in
// its own shared memory.  Global rows are moved as whole 32-byte sectors (one float4 per 2
// columns): each CTA loads a quarter of the rows and scatters them into the owners' shared
// memory (distributed shared memory), and after the transforms gathers a quarter of the
// output rows from all four CTAs.
template <int L>
__global__ void __launch_bounds__(L / elems_for(L)) pass_b_kernel(const __grid_constant__ Batch bt) {
  constexpr int E = elems_for(L), T = L / E;
  constexpr int RF = last_radix<L, false>(), BF = E / RF;  // forward's last = inverse's first (16)
  constexpr int RL = last_radix<L, true>(), BL = E / RL;
  constexpr int F4 = kTile / 2;
  static_assert(last_radix<L, false>() == first_radix<L, true>(), "register hand-off needs equal radices");
  extern __shared__ float2 sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int t = threadIdx.x;
  const int tile_g = blockIdx.x / kTile;
  int si = 0;
  while (si + 1 < bt.S && bt.s[si + 1].tile_begin <= tile_g) ++si;
  const Slice& sl = bt.s[si];
  const int pos0 = (tile_g - sl.tile_begin) * kTile;
  const int mypos = pos0 + q;
  const bool adj = bt.mode == MODE_ADJ;
  const int N = bt.N, off = bt.off;
  const int nin = adj ? L : N, yin0 = adj ? 0 : off;     // input rows (padded coordinates)
  const int nout = adj ? N : L, yout0 = adj ? off : 0;   // output rows (padded coordinates)

  for (int y = t; y < L; y += T)
    if (y < yin0 || y >= yin0 + nin) sm[phys(y)] = make_float2(0.f, 0.f);
  float2* rsm[kTile];
#pragma unroll
  for (int c = 0; c < kTile; ++c) rsm[c] = cl.map_shared_rank(sm, c);
  {
    const int rows = nin / kTile, rbeg = q * rows;
    for (int idx = t; idx < rows * F4; idx += T) {
      const int rr = rbeg + idx / F4, f = idx % F4;
      const float4 val = *reinterpret_cast<const float4*>(sl.buf + (size_t)rr * sl.wp + pos0 + 2 * f);
      float2 a = make_float2(val.x, val.y), b = make_float2(val.z, val.w);
      if (pos0 + 2 * f >= sl.w) a = make_float2(0.f, 0.f);
      if (pos0 + 2 * f + 1 >= sl.w) b = make_float2(0.f, 0.f);
      rsm[2 * f][phys(yin0 + rr)] = a;
      rsm[2 * f + 1][phys(yin0 + rr)] = b;
    }
  }
  cl.sync();

  float2 v[E];
  stage_load<L, E, false, 0>(v, t, sm);
  fft_run<L, E, false>(v, t, sm);
  {
    const int bq = abs_signed(pos_to_k(mypos, L, sl.kmax, sl.w), L);
    const bool live = mypos < sl.w;
    const float2* hrow = sl.htab + (size_t)bq * sl.hp;
#pragma unroll
    for (int b = 0; b < BF; ++b)
#pragma unroll
      for (int r = 0; r < RF; ++r) {
        const int a = abs_signed(t + b * T + r * (L / RF), L);
        float2& x = v[b * RF + r];
        if (live && a <= sl.kmax) {
          const float2 hv = hrow[a];
          x = adj ? cmulc(x, hv) : cmul(x, hv);
        } else {
          x = make_float2(0.f, 0.f);
        }
      }
  }
  fft_run<L, E, true>(v, t, sm);
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) sm[phys(t + b * T + r * (L / RL))] = v[b * RL + r];
  cl.sync();
  {
    const int rows = nout / kTile, rbeg = q * rows;
    for (int idx = t; idx < rows * F4; idx += T) {
      const int rr = rbeg + idx / F4, f = idx % F4;
      const float2 a = rsm[2 * f][phys(yout0 + rr)];
      const float2 b = rsm[2 * f + 1][phys(yout0 + rr)];
      *reinterpret_cast<float4*>(sl.buf + (size_t)rr * sl.wp + pos0 + 2 * f) = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  cl.sync();
}

// Loads a stored band row into the first-stage registers of a row IFFT.
template <int L>
__device__ __forceinline__ void load_band_row(float2 (&v)[elems_for(L)], int t, const float2* src, const Slice& sl) {
  constexpr int E = elems_for(L), T = L / E;
  constexpr int R0 = first_radix<L, true>(), B0 = E / R0;
#pragma unroll
  for (int b = 0; b < B0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int pos = band_pos(t + b * T + r * (L / R0), L, sl.kmax, sl.w);
      v[b * R0 + r] = pos >= 0 ? src[pos] : make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------------ pass C: output rows
template <int L>
__global__ void __launch_bounds__(L / elems_for(L)) pass_c_kernel(const __grid_constant__ Batch bt) {
  constexpr int E = elems_for(L), T = L / E;
  constexpr int RL = last_radix<L, true>(), BL = E / RL;
  extern __shared__ float2 sm[];
  const Slice& sl = bt.s[blockIdx.y];
  const int y = blockIdx.x;
  const int t = threadIdx.x;
  float2 v[E];
  load_band_row<L>(v, t, sl.buf + (size_t)y * sl.wp, sl);
  fft_run<L, E, true>(v, t, sm);
  const float s = bt.inv_p2;
  if (bt.mode == OUT_PSF) {
    float* dst = static_cast<float*>(sl.out) + (size_t)y * L;
#pragma unroll
    for (int b = 0; b < BL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const float2 e = cscale(v[b * RL + r], s);
        dst[t + b * T + r * (L / RL)] = fmaf(e.x, e.x, e.y * e.y);
      }
  } else {
    float2* dst = static_cast<float2*>(sl.out) + (size_t)y * L;
#pragma unroll
    for (int b = 0; b < BL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) dst[t + b * T + r * (L / RL)] = cscale(v[b * RL + r], s);
  }
}

// Deterministic block sum of one double per thread (result valid in thread 0).
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* red) {
  if constexpr (NT < 32) {  // partial warp: no full-mask shuffles
    red[threadIdx.x] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < NT; ++i) s += red[i];
      x = s;
    }
    return x;
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if constexpr (NT > 32) {
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      __syncthreads();
      if (lane == 0) red[w] = x;
      __syncthreads();
      x = 0.0;
      if (w == 0) {
        x = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      }
    }
    return x;
  }
}

// ------------------------------------------------------------------ pass C': adjoint rows
template <int L>
__global__ void __launch_bounds__(L / elems_for(L)) pass_c_adj_kernel(const __grid_constant__ Batch bt) {
  constexpr int E = elems_for(L), T = L / E;
  constexpr int RL = last_radix<L, true>(), BL = E / RL;
  constexpr int RF = last_radix<L, false>(), BF = E / RF;
  static_assert(last_radix<L, true>() == first_radix<L, false>(), "register hand-off needs equal radices");
  extern __shared__ float2 sm[];
  __shared__ double red[32];
  const Slice& sl = bt.s[blockIdx.y];
  const int y = blockIdx.x;
  const int t = threadIdx.x;
  float2* row = sl.buf + (size_t)y * sl.wp;
  float2 v[E];
  load_band_row<L>(v, t, row, sl);
  fft_run<L, E, true>(v, t, sm);
  const float s = bt.inv_p2;
  const float* trow = sl.tgt + (size_t)y * L;
  float acc = 0.f;
#pragma unroll
  for (int b = 0; b < BL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const float2 e = cscale(v[b * RL + r], s);
      const float tv = __ldg(trow + t + b * T + r * (L / RL));
      float w;
      if (bt.mode == GRAD_L2) {
        const float d = fmaf(e.x, e.x, e.y * e.y) - tv;
        acc = fmaf(d, d, acc);
        w = 2.f * d;
      } else {
        w = tv;
      }
      v[b * RL + r] = cscale(e, w);
    }
  fft_run<L, E, false>(v, t, sm);
  // the row is re-written in place: every thread has finished reading it before fft_run's
  // first barrier, and the band positions written are the ones read
#pragma unroll
  for (int b = 0; b < BF; ++b)
#pragma unroll
    for (int r = 0; r < RF; ++r) {
      const int pos = band_pos(t + b * T + r * (L / RF), L, sl.kmax, sl.w);
      if (pos >= 0) row[pos] = v[b * RF + r];
    }
  const double tot = block_sum<T>((double)acc, red);
  if (t == 0 && sl.loss_part) sl.loss_part[y] = tot;
}

// ------------------------------------------------------------------ pass A*: DOE-row adjoint
// One CTA per DOE row; loops over the slices (wavelengths of one request) and sums.
template <int L>
__global__ void __launch_bounds__(L / elems_for(L)) pass_a_adj_kernel(const __grid_constant__ Batch bt) {
  constexpr int E = elems_for(L), T = L / E;
  constexpr int RL = last_radix<L, true>(), BL = E / RL;
  extern __shared__ float2 sm[];
  const int i = blockIdx.x;
  const int t = threadIdx.x;
  const int N = bt.N, off = bt.off;
  float acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = 0.f;
  for (int j = 0; j < bt.S; ++j) {
    const Slice& sl = bt.s[j];
    float2 v[E];
    load_band_row<L>(v, t, sl.buf + (size_t)i * sl.wp, sl);
    fft_run<L, E, true>(v, t, sm);
    const float* hrow = sl.h + (size_t)i * N;
    const float2* erow = sl.e_in ? sl.e_in + (size_t)i * N : nullptr;
    const float k2 = -2.f * sl.kp_hi;
#pragma unroll
    for (int b = 0; b < BL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int x = t + b * T + r * (L / RL) - off;
        if ((unsigned)x < (unsigned)N) {
          const float2 g = cscale(v[b * RL + r], bt.inv_p2);
          float2 ed = transmittance(__ldg(hrow + x), sl.kp_hi, sl.kp_lo);
          if (erow) ed = cmul(ed, erow[x]);
          acc[b * RL + r] = fmaf(k2, fmaf(g.x, ed.y, -g.y * ed.x), acc[b * RL + r]);
        }
      }
  }
  float* grow = bt.grad + (size_t)i * N;
#pragma unroll
  for (int b = 0; b < BL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int x = t + b * T + r * (L / RL) - off;
      if ((unsigned)x < (unsigned)N) grow[x] = acc[b * RL + r];
    }
}

// Sum of the per-row loss partials of all slices, in a fixed order (one CTA).
__global__ void __launch_bounds__(1024) loss_reduce_kernel(const __grid_constant__ Batch bt, double* loss) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int j = 0; j < bt.S; ++j)
    for (int y = threadIdx.x; y < bt.P; y += 1024) acc += bt.s[j].loss_part[y];
  const double tot = block_sum<1024>(acc, red);
  if (threadIdx.x == 0) *loss = bt.mode == GRAD_L2 ? tot : 0.0;
}

// Debug: band mask of slice 0 read back from its transfer table, [P][P] uint8 in FFT order.
__global__ void band_mask_kernel(const __grid_constant__ Batch bt, uint8_t* mask) {
  const Slice& sl = bt.s[0];
  const int l = blockIdx.x;
  const int P = bt.P;
  const int a = abs_signed(l, P);
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    const int b = abs_signed(k, P);
    uint8_t mv = 0;
    if (a <= sl.kmax && b <= sl.kmax) {
      const float2 hv = sl.htab[(size_t)b * sl.hp + a];
      mv = (hv.x != 0.f || hv.y != 0.f) ? 1 : 0;
    }
    mask[(size_t)l * P + k] = mv;
  }
}

}  // namespace doe
