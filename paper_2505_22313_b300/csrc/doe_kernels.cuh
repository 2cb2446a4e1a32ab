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
// Every transform uses the in-CTA engine of doe_fft.cuh (32 samples per thread, adjacent
// pairs); global rows are read and written as 16-byte pairs of adjacent samples.
#pragma once
#include <cooperative_groups.h>

#include "doe_internal.cuh"

namespace doe {
namespace cg = cooperative_groups;

// Writes the stored band positions of a spectrum held in the last-stage layout of a forward
// row FFT into row `row` of the slice's column-tiled buffer (R rows); entries outside the
// band (at most one per segment) are written as zeros.
template <int L>
__device__ __forceinline__ void store_band_row(const float2 (&v)[32], int t, int row, int R, const Slice& sl) {
  using G = Last<L, false>;
#pragma unroll
  for (int b = 0; b < G::B; b += 2)
#pragma unroll
    for (int r = 0; r < G::R; ++r) {
      const int k = G::idx(t, b, r);
      const int pos = band_pos(k, L, sl.seg_a, sl.w);
      if (pos >= 0) {
        float2 a = v[b * G::R + r], c = v[(b + 1) * G::R + r];
        if (abs_signed(k, L) > sl.kmax) a = make_float2(0.f, 0.f);
        if (abs_signed(k + 1, L) > sl.kmax) c = make_float2(0.f, 0.f);
        const size_t o = tiled_at(row, pos, R, kTile);
        if (DOE_IN(o + 1, sl.n_tbuf)) __stcs(reinterpret_cast<float4*>(sl.tbuf + o), make_float4(a.x, a.y, c.x, c.y));
      }
    }
}

// Loads stored band row `row` of the slice's field buffer into the first-stage registers of a
// row IFFT (16-byte pairs).
template <int L>
__device__ __forceinline__ void load_band_row(float2 (&v)[32], int t, int row, const Slice& sl) {
  using F = First<L, true>;
  const size_t r0 = (size_t)row * sl.wp;
  const float4* s4 = reinterpret_cast<const float4*>(sl.buf + r0);
#pragma unroll
  for (int b = 0; b < F::B; b += 2)
#pragma unroll
    for (int r = 0; r < F::R; ++r) {
      const int pos = band_pos(F::idx(t, b, r), L, sl.seg_a, sl.w);
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (pos >= 0 && DOE_IN(r0 + pos + 1, sl.n_buf)) q = __ldcs(s4 + (pos >> 1));
      v[b * F::R + r] = make_float2(q.x, q.y);
      v[(b + 1) * F::R + r] = make_float2(q.z, q.w);
    }
}

// With 2x zero padding the DOE fills the middle half [L/4, 3L/4) of a forward transform's
// input.  First-stage register r of every thread holds input j + r L/R0 with j < L/R0, so for a
// first radix R0 >= 4 it lies inside the DOE exactly when R0/4 <= r < 3 R0/4: a compile-time
// pattern, so the first butterflies of the transform fold the zero inputs away.
template <int L>
__host__ __device__ constexpr bool pad2_foldable() { return First<L, false>::R >= 4; }
template <int L>
__device__ __forceinline__ constexpr bool pad2_live(int r) {
  return r >= First<L, false>::R / 4 && r < 3 * First<L, false>::R / 4;
}

// ------------------------------------------------------------------ pass A: DOE rows
// 16-byte asynchronous copies of the n heights at element o of the slice's layout into shared
// memory (cp.async, L2 only).
__device__ __forceinline__ void stage_heights(float* dst, const Slice& sl, size_t o, int n, int t, int nt) {
  const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
  const float* src = sl.h + o;
  for (int k = t; k < n / 4; k += nt)
    if (DOE_IN(o + 4 * k + 3, sl.n_h))
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + 16u * k), "l"(src + 4 * k) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void wait_staged() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Persistent: CTA b transforms the (slice, DOE row) items k = b, b + gridDim.x, ... of all
// S x N items (slice k / N, row k mod N).  The first stage's register pairs are adjacent padded
// columns x, x + 1 (x even; the DOE offset is even).  When a height row fits behind the
// exchange buffer (N <= L / 2, i.e. pad 2) the next item's heights are copied into shared
// memory while the current row is transformed; otherwise they are read from global memory.
// ILLUM: some slice has a parametric incident field (evaluated per sample with the phase).
// PAD2: 2x padding (N = L / 2) with the compile-time input pattern of pad2_live.
template <int L, bool ILLUM, bool PAD2>
__global__ void __launch_bounds__(L / 32, min_blocks(L)) pass_a_kernel(const __grid_constant__ Batch bt) {
  using F = First<L, false>;
  constexpr int T = L / 32;
  extern __shared__ float2 sm[];
  float* hs = reinterpret_cast<float*>(sm + L);  // staged height row (N floats)
  const int t = threadIdx.x;
  const int N = bt.N, off = bt.off;
  const bool staged = 2 * N <= L;
  const int items = bt.S * N, k0 = blockIdx.x, dk = gridDim.x;
  // height layout row of DOE row i: row i >> uf of the (N >> uf)-wide layout
  auto layout_off = [&](int kk) { const Slice& q = bt.s[kk / N]; return (size_t)((kk % N) >> q.uf) * (N >> q.uf); };
  auto layout_n = [&](int kk) { return N >> bt.s[kk / N].uf; };
  if (staged && k0 < items) stage_heights(hs, bt.s[k0 / N], layout_off(k0), layout_n(k0), t, T);
  for (int k = k0; k < items; k += dk) {
    const Slice& sl = bt.s[k / N];
    const int i = k % N, uf = sl.uf;
    const bool erow = sl.e_in != nullptr;
    float2 hv[F::B / 2][F::R];
    if (staged) {
      wait_staged();
      __syncthreads();  // row i is in hs for every thread
    }
#pragma unroll
    for (int b = 0; b < F::B; b += 2)
#pragma unroll
      for (int r = 0; r < F::R; ++r) {
        const int x = F::idx(t, b, r) - off;  // even
        hv[b / 2][r] = make_float2(0.f, 0.f);
        if (PAD2 ? pad2_live<L>(r) : (unsigned)x < (unsigned)N) {
          if (!staged) hv[b / 2][r] = heights_pair(sl, N, i, x);
          else if (uf == 0) hv[b / 2][r] = DOE_IN(x + 1, N) ? *reinterpret_cast<const float2*>(hs + x) : make_float2(0.f, 0.f);
          else hv[b / 2][r] = DOE_IN(x >> uf, N >> uf) ? make_float2(hs[x >> uf], hs[x >> uf]) : make_float2(0.f, 0.f);
        }
      }
    if (staged) {
      __syncthreads();  // every thread has read hs
      const int kn = k + dk;
      if (kn < items) stage_heights(hs, bt.s[kn / N], layout_off(kn), layout_n(kn), t, T);
    }
    float2 v[32];
    IncRow ir = {0.f, 0u};
    if constexpr (ILLUM) ir = incident_row(sl, i - N / 2);
#pragma unroll
    for (int b = 0; b < F::B; b += 2)
#pragma unroll
      for (int r = 0; r < F::R; ++r) {
        const int x = F::idx(t, b, r) - off;
        float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
        if (PAD2 ? pad2_live<L>(r) : (unsigned)x < (unsigned)N) {
          if (ILLUM && sl.illum) {
            a = transmittance_inc(hv[b / 2][r].x, sl, ir, x - N / 2);
            c = transmittance_inc(hv[b / 2][r].y, sl, ir, x + 1 - N / 2);
          } else {
            a = transmittance(hv[b / 2][r].x, sl.kp_hi, sl.kp_lo);
            c = uf ? a : transmittance(hv[b / 2][r].y, sl.kp_hi, sl.kp_lo);  // one layout cell
          }
          if (erow) {
            const float4 ev = ein_pair(sl, N, i, x);
            a = cmul(a, make_float2(ev.x, ev.y));
            c = cmul(c, make_float2(ev.z, ev.w));
          }
        }
        v[b * F::R + r] = a;
        v[(b + 1) * F::R + r] = c;
      }
    fft_run<L, 32, false>(v, t, sm);  // its first exchange waits for every thread's previous row
    store_band_row<L>(v, t, i, N, sl);
  }
}

// ------------------------------------------------------------------ pass B / B*: columns
// A cluster of kTile CTAs owns kTile adjacent stored columns; CTA q transforms column q.
// Input: each CTA reads its own column of the column-tiled buffer directly into registers
// (the cluster's CTAs together consume whole 32-byte sectors).  Output: after the transforms
// each CTA gathers a quarter of the output rows of all four columns from the cluster's shared
// memory (distributed shared memory) and writes them as 32-byte row segments.
// PAD2F: the forward pass at 2x padding (N = L / 2), with the compile-time input pattern of
// pad2_live.
template <int L, bool PAD2F>
__global__ void __launch_bounds__(L / 32, min_blocks(L)) pass_b_kernel(const __grid_constant__ Batch bt) {
  using G = Last<L, false>;  // forward's last stage = inverse's first stage (radix 16)
  using H = Last<L, true>;
  constexpr int T = L / 32;
  constexpr int F4 = kTile / 2;
  static_assert(G::R == First<L, true>::R, "register hand-off needs equal radices");
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
  const bool adj = !PAD2F && bt.mode == MODE_ADJ;
  const int N = bt.N, off = bt.off;
  const int nin = adj ? L : N, yin0 = adj ? 0 : off;     // input rows (padded coordinates)
  const int nout = adj ? N : L, yout0 = adj ? off : 0;   // output rows (padded coordinates)
  const int kcol = pos_to_k(mypos, L, sl.seg_a, sl.w);
  const bool live = mypos < sl.w && abs_signed(kcol, L) <= sl.kmax;

  float4* rsm[kTile];
#pragma unroll
  for (int c = 0; c < kTile; ++c) rsm[c] = reinterpret_cast<float4*>(cl.map_shared_rank(sm, c));
  const float2* hrow = sl.htab + (size_t)abs_signed(kcol, L) * sl.hp;
  if (live) {  // this column's transfer-function row, into L1 ahead of the multiply
    const char* hb = reinterpret_cast<const char*>(hrow);
    for (int o = 128 * t; o < (sl.kmax + 1) * (int)sizeof(float2); o += 128 * T)
      asm volatile("prefetch.global.L1 [%0];" ::"l"(hb + o));
  }
  // This CTA's column straight into the first stage's registers: rows e, e + 1 of the pair
  // are two 8-byte loads 32 bytes apart in the tile (e - yin0 and nin are even, so both are
  // inside or both outside the input rows).  The cluster's CTAs read the four columns of each
  // 32-byte sector together, so DRAM still delivers every sector once.
  float2 v[32];
  {
    using F = First<L, false>;
    static_assert(F::PAIRED, "first stage holds adjacent pairs");
    const size_t c0 = tiled_at(0, mypos, nin, kTile);
    const float2* col = sl.tbuf + c0;
#pragma unroll
    for (int b = 0; b < F::B; b += 2)
#pragma unroll
      for (int r = 0; r < F::R; ++r) {
        const int y = F::idx(t, b, r) - yin0;
        float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
        if (PAD2F ? pad2_live<L>(r) : (unsigned)y < (unsigned)nin) {
          if (live && DOE_IN(c0 + (size_t)(y + 1) * kTile, sl.n_tbuf)) {
            a = __ldcs(col + (size_t)y * kTile);
            c = __ldcs(col + (size_t)(y + 1) * kTile);
          }
        }
        v[b * F::R + r] = a;
        v[(b + 1) * F::R + r] = c;
      }
  }
  fft_run<L, 32, false>(v, t, sm);
  {
#pragma unroll
    for (int b = 0; b < G::B; ++b)
#pragma unroll
      for (int r = 0; r < G::R; ++r) {
        const int a = abs_signed(G::idx(t, b, r), L);
        float2& x = v[b * G::R + r];
        if (live && a <= sl.kmax && DOE_IN((size_t)abs_signed(kcol, L) * sl.hp + a, sl.n_htab)) {
          const float2 hv = hrow[a];
          x = adj ? cmulc(x, hv) : cmul(x, hv);
        } else {
          x = make_float2(0.f, 0.f);
        }
      }
  }
  fft_run<L, 32, true>(v, t, sm);
  __syncthreads();
  {
    float4* s4 = reinterpret_cast<float4*>(sm);
#pragma unroll
    for (int b = 0; b < H::B; b += 2)
#pragma unroll
      for (int r = 0; r < H::R; ++r) {
        const float2 a = v[b * H::R + r], c = v[(b + 1) * H::R + r];
        if (DOE_IN(swz(H::idx(t, b, r) >> 1), L / 2)) s4[swz(H::idx(t, b, r) >> 1)] = make_float4(a.x, a.y, c.x, c.y);
      }
  }
  cl.sync();  // all four columns are in shared memory (and every CTA of the cluster has started)
  {
    // item idx = (row pair, column pair f): IT items per thread, all remote loads issued
    // before the first store so their latencies overlap
    static_assert(F4 == 2, "two column pairs per tile");
    constexpr int IT = (L / kTile / 2) * F4 / T;
    const int rows = nout / kTile, rbeg = q * rows, lim = (rows / 2) * F4;
    float4 a[IT], b[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int idx = t + it * T, f = idx & 1;  // f = t & 1 whenever T is even
      if (idx < lim) {
        const int ch = swz((yout0 + rbeg + 2 * (idx / F4)) >> 1);
        a[it] = b[it] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (DOE_IN(ch, L / 2)) {
          a[it] = (f ? rsm[2] : rsm[0])[ch];  // rows rr, rr + 1 of column 2f
          b[it] = (f ? rsm[3] : rsm[1])[ch];  // of column 2f + 1
        }
      }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int idx = t + it * T, f = idx & 1;
      if (idx < lim) {
        const int rr = rbeg + 2 * (idx / F4);
        const size_t o = (size_t)rr * sl.wp + pos0 + 2 * f;
        float2* dst = sl.buf + o;
        if (DOE_IN(o + sl.wp + 1, sl.n_buf)) {
          __stcs(reinterpret_cast<float4*>(dst), make_float4(a[it].x, a[it].y, b[it].x, b[it].y));
          __stcs(reinterpret_cast<float4*>(dst + sl.wp), make_float4(a[it].z, a[it].w, b[it].z, b[it].w));
        }
      }
    }
  }
  cluster_sync_relaxed();  // the peers have read this CTA's shared memory before it exits
}

// ------------------------------------------------------------------ pass C: output rows
template <int L>
__global__ void __launch_bounds__(L / 32, min_blocks(L)) pass_c_kernel(const __grid_constant__ Batch bt) {
  using H = Last<L, true>;
  extern __shared__ float2 sm[];
  const Slice& sl = bt.s[blockIdx.y];
  const int y = blockIdx.x;
  const int t = threadIdx.x;
  float2 v[32];
  load_band_row<L>(v, t, y, sl);
  fft_run<L, 32, true>(v, t, sm);
  const float s = bt.inv_p2;
  if (bt.mode == OUT_PSF) {
    float2* dst = reinterpret_cast<float2*>(static_cast<float*>(sl.out) + (size_t)y * L);
#pragma unroll
    for (int b = 0; b < H::B; b += 2)
#pragma unroll
      for (int r = 0; r < H::R; ++r) {
        const float2 a = cscale(v[b * H::R + r], s), c = cscale(v[(b + 1) * H::R + r], s);
        if (DOE_IN((size_t)y * L + H::idx(t, b, r) + 1, sl.n_out))
          __stcs(dst + (H::idx(t, b, r) >> 1), make_float2(fmaf(a.x, a.x, a.y * a.y), fmaf(c.x, c.x, c.y * c.y)));
      }
  } else {
    float4* dst = reinterpret_cast<float4*>(static_cast<float2*>(sl.out) + (size_t)y * L);
#pragma unroll
    for (int b = 0; b < H::B; b += 2)
#pragma unroll
      for (int r = 0; r < H::R; ++r) {
        const float2 a = cscale(v[b * H::R + r], s), c = cscale(v[(b + 1) * H::R + r], s);
        if (DOE_IN((size_t)y * L + H::idx(t, b, r) + 1, sl.n_out))
          __stcs(dst + (H::idx(t, b, r) >> 1), make_float4(a.x, a.y, c.x, c.y));
      }
  }
}

// ------------------------------------------------------------------ pass C': adjoint rows
template <int L>
__global__ void __launch_bounds__(L / 32, min_blocks(L)) pass_c_adj_kernel(const __grid_constant__ Batch bt) {
  using H = Last<L, true>;
  static_assert(H::R == First<L, false>::R, "register hand-off needs equal radices");
  extern __shared__ float2 sm[];
  __shared__ double red[32];
  const Slice& sl = bt.s[blockIdx.y];
  const int y = blockIdx.x;
  const int t = threadIdx.x;
  float2 v[32];
  load_band_row<L>(v, t, y, sl);
  fft_run<L, 32, true>(v, t, sm);
  const float s = bt.inv_p2;
  const float2* trow = reinterpret_cast<const float2*>(sl.tgt + (size_t)y * L);
  float acc = 0.f;
#pragma unroll
  for (int b = 0; b < H::B; b += 2)
#pragma unroll
    for (int r = 0; r < H::R; ++r) {
      const float2 tv = DOE_IN((size_t)y * L + H::idx(t, b, r) + 1, sl.n_tgt) ? __ldcs(trow + (H::idx(t, b, r) >> 1))
                                                                              : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 e = cscale(v[(b + u) * H::R + r], s);
        const float tt = u ? tv.y : tv.x;
        float w;
        if (bt.mode == GRAD_L2) {
          const float d = fmaf(e.x, e.x, e.y * e.y) - tt;
          acc = fmaf(d, d, acc);
          w = 2.f * d;
        } else {
          w = tt;
        }
        v[(b + u) * H::R + r] = cscale(e, w);
      }
    }
  fft_run<L, 32, false>(v, t, sm);
  store_band_row<L>(v, t, y, L, sl);  // J1 row y of the column-tiled buffer (P rows)
  const double tot = block_sum<L / 32>((double)acc, red);
  if (t == 0 && sl.loss_part && DOE_IN(y, sl.n_loss)) sl.loss_part[y] = tot;
}

// ------------------------------------------------------------------ pass A*: DOE-row adjoint
// One CTA per DOE row; loops over the slices (wavelengths of one request) and sums.
template <int L, bool ILLUM>
__global__ void __launch_bounds__(L / 32, min_blocks(L)) pass_a_adj_kernel(const __grid_constant__ Batch bt) {
  using H = Last<L, true>;
  extern __shared__ float2 sm[];
  const int i = blockIdx.x;
  const int t = threadIdx.x;
  const int N = bt.N, off = bt.off;
  float acc[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) acc[e] = 0.f;
  for (int j = 0; j < bt.S; ++j) {
    const Slice& sl = bt.s[j];
    float2 v[32];
    load_band_row<L>(v, t, i, sl);
    fft_run<L, 32, true>(v, t, sm);
    const bool erow = sl.e_in != nullptr;
    const float k2 = -2.f * sl.kp_hi;
    IncRow ir = {0.f, 0u};
    if constexpr (ILLUM) ir = incident_row(sl, i - N / 2);
#pragma unroll
    for (int b = 0; b < H::B; b += 2)
#pragma unroll
      for (int r = 0; r < H::R; ++r) {
        const int x = H::idx(t, b, r) - off;  // even
        if ((unsigned)x < (unsigned)N) {
          const float2 hv = heights_pair(sl, N, i, x);
          float2 e0, e1;
          if (ILLUM && sl.illum) {
            e0 = transmittance_inc(hv.x, sl, ir, x - N / 2);
            e1 = transmittance_inc(hv.y, sl, ir, x + 1 - N / 2);
          } else {
            e0 = transmittance(hv.x, sl.kp_hi, sl.kp_lo);
            e1 = sl.uf ? e0 : transmittance(hv.y, sl.kp_hi, sl.kp_lo);
          }
          if (erow) {
            const float4 ev = ein_pair(sl, N, i, x);
            e0 = cmul(e0, make_float2(ev.x, ev.y));
            e1 = cmul(e1, make_float2(ev.z, ev.w));
          }
          const float2 g0 = cscale(v[b * H::R + r], bt.inv_p2);
          const float2 g1 = cscale(v[(b + 1) * H::R + r], bt.inv_p2);
          acc[b * H::R + r] = fmaf(k2, fmaf(g0.x, e0.y, -g0.y * e0.x), acc[b * H::R + r]);
          acc[(b + 1) * H::R + r] = fmaf(k2, fmaf(g1.x, e1.y, -g1.y * e1.x), acc[(b + 1) * H::R + r]);
        }
      }
  }
  float2* grow = reinterpret_cast<float2*>(bt.grad + (size_t)i * N);
#pragma unroll
  for (int b = 0; b < H::B; b += 2)
#pragma unroll
    for (int r = 0; r < H::R; ++r) {
      const int x = H::idx(t, b, r) - off;
      if ((unsigned)x < (unsigned)N && DOE_IN((size_t)i * N + x + 1, bt.n_grad))
        grow[x >> 1] = make_float2(acc[b * H::R + r], acc[(b + 1) * H::R + r]);
    }
}

}  // namespace doe
