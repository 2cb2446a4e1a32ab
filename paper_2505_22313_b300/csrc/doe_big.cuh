// doe_big.cuh -- transforms split across a cluster: P = Q * L with sub-transforms of L = 8192
// points, for grids longer than one CTA's transform (P = 32768: Q = 4, P = 65536: Q = 8).
// 64 KB of shared memory and 256 threads per CTA, so two CTAs share an SM and one CTA's
// global / distributed-shared-memory phases overlap another's transforms.
//
// A length-P transform is split across a cluster of Q CTAs, each running the in-CTA engine
// on L points (sub-transform s):
//   forward (decimation in frequency)  x = n1 L + n2:
//     y_s[n2] = W_P^{n2 s} sum_{n1} x[n1 L + n2] W_Q^{n1 s},  X[s + Q k2] = FFT_L(y_s)[k2]
//   inverse (decimation in time)  output x = x2 + L q, input V_s[k2] = V[s + Q k2]:
//     out[x2 + L q] = sum_s W_Q^{-s q} W_P^{-s x2} IFFT_L(V_s)[x2]
// The radix-Q step is done once per element: each CTA takes a 1/Q share of n2 (or x2),
// reads the Q values it needs from the other CTAs' shared memory (distributed shared memory)
// or from global memory, and writes the Q results to their owners.  Spectra of rows are
// stored in sub-transform order: position s L + k2 holds frequency k = s + Q k2 (no band
// compaction; out-of-band columns are zeroed by the column pass).
#pragma once
#include <cooperative_groups.h>

#include "doe_kernels.cuh"

namespace doe {

constexpr int kBigL = 8192;  // sub-transform length of split rows / columns

// W_P^m (forward sign) for 0 <= m < P <= 65536.  With n = m 65536 / P = 256 hi + lo,
// W_65536^n = W_65536^{256 hi} W_65536^{lo}: two lookups in 256-entry tables (4 KB in all,
// L1-resident) and one complex product, instead of a scattered read of a 512 KB table.
template <int P>
__device__ __forceinline__ float2 wbig(int m) {
  const int n = (m * ((1 << kBigLog) / P)) & ((1 << kBigLog) - 1);
  return cmul(__ldg(g_tw_big + 256 + (n >> 8)), __ldg(g_tw_big + (n & 255)));
}
template <bool INV>
__device__ __forceinline__ float2 tw_apply(float2 a, float2 w) { return INV ? cmulc(a, w) : cmul(a, w); }

// frequency index of stored column position pos when rows are stored in sub-transform order
__device__ __forceinline__ int big_pos_to_k(int pos, int Q) { return (pos % kBigL) * Q + pos / kBigL; }
// column tile of split grids: two adjacent stored columns per cluster (one cluster = 2 Q CTAs:
// 8 at P = 32768, 16 at P = 65536, the non-portable cluster size), so that the output rows
// are written as 16-byte pairs and the input read 16 bytes per row
__host__ __device__ constexpr int big_tile(int) { return 2; }

// ------------------------------------------------------------------ rows, forward (pass A)
template <int Q, bool ILLUM>
__global__ void __launch_bounds__(kBigL / 32, min_blocks(kBigL)) pass_a_big_kernel(const __grid_constant__ Batch bt) {
  constexpr int L = kBigL, T = L / 32, P = L * Q, SH = L / Q;
  using G = Last<L, false>;
  extern __shared__ float2 sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int s = (int)cl.block_rank();
  const int i = blockIdx.x / Q;
  const Slice& sl = bt.s[blockIdx.y];
  const int t = threadIdx.x, N = bt.N, off = bt.off;
  const bool erow = sl.e_in != nullptr;
  IncRow ir = {0.f, 0u};
  if constexpr (ILLUM) ir = incident_row(sl, i - N / 2);
  float4* rsm[Q];
#pragma unroll
  for (int c = 0; c < Q; ++c) rsm[c] = reinterpret_cast<float4*>(cl.map_shared_rank(sm, c));
  cluster_sync_relaxed();  // every CTA of the cluster has started before its shared memory is written
#pragma unroll
  for (int it = 0; it < SH / (2 * T); ++it) {  // compile-time count: loads of all items in flight together
    const int n2 = s * SH + 2 * t + it * 2 * T;
    float2 xa[Q], xb[Q];
#pragma unroll
    for (int n1 = 0; n1 < Q; ++n1) {
      const int x = n1 * L + n2 - off;  // even
      xa[n1] = xb[n1] = make_float2(0.f, 0.f);
      if ((unsigned)x < (unsigned)N) {
        const float2 hv = heights_pair(sl, N, i, x);
        if (ILLUM && sl.illum) {
          xa[n1] = transmittance_inc(hv.x, sl, ir, x - N / 2);
          xb[n1] = transmittance_inc(hv.y, sl, ir, x + 1 - N / 2);
        } else {
          xa[n1] = transmittance(hv.x, sl.kp_hi, sl.kp_lo);
          xb[n1] = sl.uf ? xa[n1] : transmittance(hv.y, sl.kp_hi, sl.kp_lo);
        }
        if (erow) {
          const float4 ev = ein_pair(sl, N, i, x);
          xa[n1] = cmul(xa[n1], make_float2(ev.x, ev.y));
          xb[n1] = cmul(xb[n1], make_float2(ev.z, ev.w));
        }
      }
    }
    dft<Q, false>(xa);
    dft<Q, false>(xb);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float2 a = cmul(xa[q], wbig<P>(n2 * q)), b = cmul(xb[q], wbig<P>((n2 + 1) * q));
      if (DOE_IN(swz(n2 >> 1), L / 2)) rsm[q][swz(n2 >> 1)] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  cl.sync();
  float2 v[32];
  stage_load<L, 32, false, 0>(v, t, sm);
  fft_run<L, 32, false>(v, t, sm);
  // column-tiled buffer, 4-wide tiles at every grid size: the pair (pos, pos + 1) is 16 bytes
#pragma unroll
  for (int b = 0; b < G::B; b += 2)
#pragma unroll
    for (int r = 0; r < G::R; ++r) {
      const float2 a = v[b * G::R + r], c = v[(b + 1) * G::R + r];
      const int pos = s * L + G::idx(t, b, r);
      if (DOE_IN(tiled_at(i, pos, N, kTile) + 1, sl.n_tbuf))
        __stcs(reinterpret_cast<float4*>(sl.tbuf + tiled_at(i, pos, N, kTile)), make_float4(a.x, a.y, c.x, c.y));
    }
}

// Inverse sub-transform s of a stored row (positions s L .. s L + L - 1), result written to
// this CTA's shared memory in natural order.
template <int Q>
__device__ __forceinline__ void big_row_inverse_to_smem(const Slice& sl, int y, int s, int t, float2* sm) {
  constexpr int L = kBigL;
  using F = First<L, true>;
  using H = Last<L, true>;
  const size_t r0 = (size_t)y * sl.wp + (size_t)s * L;
  const float4* src = reinterpret_cast<const float4*>(sl.buf + r0);
  float2 v[32];
#pragma unroll
  for (int b = 0; b < F::B; b += 2)
#pragma unroll
    for (int r = 0; r < F::R; ++r) {
      const float4 q = DOE_IN(r0 + F::idx(t, b, r) + 1, sl.n_buf) ? __ldcs(src + (F::idx(t, b, r) >> 1))
                                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
      v[b * F::R + r] = make_float2(q.x, q.y);
      v[(b + 1) * F::R + r] = make_float2(q.z, q.w);
    }
  fft_run<L, 32, true>(v, t, sm);
  __syncthreads();
  float4* s4 = reinterpret_cast<float4*>(sm);
#pragma unroll
  for (int b = 0; b < H::B; b += 2)
#pragma unroll
    for (int r = 0; r < H::R; ++r) {
      const float2 a = v[b * H::R + r], c = v[(b + 1) * H::R + r];
      if (DOE_IN(swz(H::idx(t, b, r) >> 1), L / 2)) s4[swz(H::idx(t, b, r) >> 1)] = make_float4(a.x, a.y, c.x, c.y);
    }
}

// Decimation-in-time combine for the pair (x2, x2 + 1): reads IFFT_L(V_s)[x2..] from every
// CTA of the cluster and returns out[x2 + L q] in oa[q], out[x2 + 1 + L q] in ob[q].
template <int Q>
__device__ __forceinline__ void big_combine(float4* const (&rsm)[Q], int x2, float2 (&oa)[Q], float2 (&ob)[Q]) {
  constexpr int P = kBigL * Q;
#pragma unroll
  for (int sp = 0; sp < Q; ++sp) {
    const float4 q4 = DOE_IN(swz(x2 >> 1), kBigL / 2) ? rsm[sp][swz(x2 >> 1)] : make_float4(0.f, 0.f, 0.f, 0.f);
    oa[sp] = cmulc(make_float2(q4.x, q4.y), wbig<P>(sp * x2));
    ob[sp] = cmulc(make_float2(q4.z, q4.w), wbig<P>(sp * (x2 + 1)));
  }
  dft<Q, true>(oa);
  dft<Q, true>(ob);
}

// ------------------------------------------------------------------ rows, inverse (pass C)
template <int Q>
__global__ void __launch_bounds__(kBigL / 32, min_blocks(kBigL)) pass_c_big_kernel(const __grid_constant__ Batch bt) {
  constexpr int L = kBigL, T = L / 32, SH = L / Q;
  extern __shared__ float2 sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int s = (int)cl.block_rank();
  const int y = blockIdx.x / Q;
  const Slice& sl = bt.s[blockIdx.y];
  const int t = threadIdx.x;
  const int P = L * Q;
  float4* rsm[Q];
#pragma unroll
  for (int c = 0; c < Q; ++c) rsm[c] = reinterpret_cast<float4*>(cl.map_shared_rank(sm, c));
  big_row_inverse_to_smem<Q>(sl, y, s, t, sm);
  cl.sync();
  const float sc = bt.inv_p2;
#pragma unroll
  for (int it = 0; it < SH / (2 * T); ++it) {
    const int x2 = s * SH + 2 * t + it * 2 * T;
    float2 oa[Q], ob[Q];
    big_combine<Q>(rsm, x2, oa, ob);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float2 a = cscale(oa[q], sc), b = cscale(ob[q], sc);
      const size_t o = (size_t)y * P + (size_t)q * L + x2;
      if (!DOE_IN(o + 1, sl.n_out)) continue;
      if (bt.mode == OUT_PSF)
        __stcs(reinterpret_cast<float2*>(static_cast<float*>(sl.out) + o),
               make_float2(fmaf(a.x, a.x, a.y * a.y), fmaf(b.x, b.x, b.y * b.y)));
      else
        __stcs(reinterpret_cast<float4*>(static_cast<float2*>(sl.out) + o), make_float4(a.x, a.y, b.x, b.y));
    }
  }
  cluster_sync_relaxed();  // peers have finished reading this CTA's shared memory
}

// ------------------------------------------------------------------ columns (pass B / B*)
// Cluster of TC x Q CTAs (TC = big_tile(Q) adjacent stored columns x Q sub-transforms, at
// most 16); rank = c Q + s.
// Rows are stored in sub-transform order (the row passes above).  Both exchanges between the
// CTAs are pushes (remote stores, which no thread waits on): the decimation-in-frequency step
// writes each sub-transform's inputs into its owner's buffer, and after the inverse
// sub-transforms each CTA writes its results into the buffer of the CTA that combines those
// rows.  The transfer-function entries arrive by bulk copy during the forward transform.
template <int Q>
__global__ void __launch_bounds__(kBigL / 32, min_blocks(kBigL)) pass_b_big_kernel(const __grid_constant__ Batch bt) {
  constexpr int L = kBigL, T = L / 32, P = L * Q, TC = big_tile(Q), CL = TC * Q, SH = L / CL;
  static_assert(kTile % TC == 0, "a cluster's columns lie inside one tile of the buffer");
  using G = Last<L, false>;
  using Hh = Last<L, true>;
  static_assert(G::R == First<L, true>::R, "register hand-off needs equal radices");
  extern __shared__ float2 sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int c = rank / Q, s = rank % Q;
  const int t = threadIdx.x;
  const int tile_g = blockIdx.x / CL;
  int si = 0;
  while (si + 1 < bt.S && bt.s[si + 1].tile_begin <= tile_g) ++si;
  const Slice& sl = bt.s[si];
  const int pos0 = (tile_g - sl.tile_begin) * TC;
  const int kcol = big_pos_to_k(pos0 + c, Q);
  const int ak = abs_signed(kcol, P);
  const bool live = pos0 + c < sl.w && ak <= sl.kmax;
  // The transfer-function entries sub-transform s multiplies after its forward transform are
  // those of the frequencies f = s + Q k2: for f <= P/2 entry a = f (residue class s of the
  // table row, position k2); above P/2 the mirror a = P - f (class (Q - s) mod Q, position
  // L - k2 for s = 0, L - 1 - k2 otherwise).  Both runs are copied into the exchange buffer
  // while the forward transform's last stage computes: class s at entry 0 (L/2 + 2 entries
  // for s = 0, where it also holds the mirrors; L/2 otherwise), class Q - s at entry L/2 (L/2
  // entries; none for s = Q/2, whose mirrors share class s).  Table rows hold hq (even)
  // entries per class, so each run starts on a 16-byte boundary.
  __shared__ __align__(8) uint64_t hbar;  // completion of the copies
  const int hb = (Q - s) % Q;
  const int nA = min(s == 0 ? L / 2 + 2 : L / 2, sl.hq), nB = hb == s ? 0 : min(L / 2, sl.hq);
  const float2* hrow = sl.htab + (size_t)ak * sl.hp;
  const bool hcopy = live && DOE_IN((size_t)ak * sl.hp + (size_t)s * sl.hq + nA - 1, sl.n_htab) &&
                     (nB == 0 || DOE_IN((size_t)ak * sl.hp + (size_t)hb * sl.hq + nB - 1, sl.n_htab));
  if (t == 0) mbar_init(&hbar, 1);
  const bool adj = bt.mode == MODE_ADJ;
  const int N = bt.N, off = bt.off;
  const int nin = adj ? P : N, yin0 = adj ? 0 : off;
  const int nout = adj ? N : P, yout0 = adj ? off : 0;
  // peers' shared memory, mapped where it is used (an array of 2 Q pointers would hold 4 Q registers)
  auto rsm = [&](int k) { return cl.map_shared_rank(sm, k); };
  cluster_sync_relaxed();
  // decimation-in-frequency split of the TC columns over the row chunks y = y1 L + y2; each
  // thread takes the adjacent pair (y2, y2 + 1) so its shared-memory writes are 16 bytes
#pragma unroll
  for (int it = 0; it < SH / (2 * T); ++it) {
    const int y2 = rank * SH + 2 * t + it * 2 * T;
    float2 col[2][TC][Q];
    // this cluster's TC columns inside the buffer's 4-wide tiles (TC = 4: the whole tile row;
    // TC = 2, 1: part of it, the rest read by the neighbouring clusters at the same time)
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int y1 = 0; y1 < Q; ++y1) {
        const int y = y1 * L + y2 + u;
        if ((unsigned)(y - yin0) < (unsigned)nin) {
          const float2* src = sl.tbuf + tiled_at(y - yin0, pos0, nin, kTile);
          if (!DOE_IN(tiled_at(y - yin0, pos0, nin, kTile) + TC - 1, sl.n_tbuf)) src = sl.tbuf;  // skip: read entry 0
          if constexpr (TC >= 2) {
#pragma unroll
            for (int f = 0; f < TC / 2; ++f) {
              const float4 q4 = __ldcs(reinterpret_cast<const float4*>(src) + f);
              col[u][2 * f][y1] = make_float2(q4.x, q4.y);
              col[u][2 * f + 1][y1] = make_float2(q4.z, q4.w);
            }
          } else {
            col[u][0][y1] = __ldcs(src);
          }
        } else {
#pragma unroll
          for (int cc = 0; cc < TC; ++cc) col[u][cc][y1] = make_float2(0.f, 0.f);
        }
      }
#pragma unroll
    for (int cc = 0; cc < TC; ++cc) {
      dft<Q, false>(col[0][cc]);
      dft<Q, false>(col[1][cc]);
    }
#pragma unroll
    for (int sp = 0; sp < Q; ++sp) {
      const float2 w0 = wbig<P>(y2 * sp), w1 = wbig<P>((y2 + 1) * sp);  // shared by the TC columns
#pragma unroll
      for (int cc = 0; cc < TC; ++cc) {
        const float2 a = cmul(col[0][cc][sp], w0), d = cmul(col[1][cc][sp], w1);
        if (DOE_IN(swz(y2 >> 1), L / 2))
          reinterpret_cast<float4*>(rsm(cc * Q + sp))[swz(y2 >> 1)] = make_float4(a.x, a.y, d.x, d.y);
      }
    }
  }
  cl.sync();
  float2 v[32];
  stage_load<L, 32, false, 0>(v, t, sm);
  fft_run_last<L, 32, false>(v, t, sm, [&] {
    fence_proxy_async_smem();  // this thread's reads of the buffer come before the copies' writes
    __syncthreads();
    if (hcopy && t == 0) {
      mbar_arrive_expect_tx(&hbar, (unsigned)(nA + nB) * sizeof(float2));
      bulk_g2s(sm, hrow + (size_t)s * sl.hq, (unsigned)nA * sizeof(float2), &hbar);
      if (nB) bulk_g2s(sm + L / 2, hrow + (size_t)hb * sl.hq, (unsigned)nB * sizeof(float2), &hbar);
    }
  });
  const bool hok = !hcopy || mbar_wait(&hbar, 0);
  if (!hok && t == 0) raise_fault(FAULT_WAIT_TIMEOUT);
  {
#pragma unroll
    for (int b = 0; b < G::B; ++b)
#pragma unroll
      for (int r = 0; r < G::R; ++r) {
        const int k2 = G::idx(t, b, r), f = s + Q * k2;
        const int a = abs_signed(f, P);
        const int e = f < P / 2 ? k2 : s == 0 ? L - k2 : nB == 0 ? L - 1 - k2 : L / 2 + L - 1 - k2;
        float2& x = v[b * G::R + r];
        if (hcopy && hok && a <= sl.kmax && DOE_IN(e, L)) {
          const float2 hv = sm[e];
          x = adj ? cmulc(x, hv) : cmul(x, hv);
        } else {
          x = make_float2(0.f, 0.f);
        }
      }
  }
  // inverse transform; once every CTA of the cluster has loaded its last stage's inputs, the
  // exchange buffers are free and each CTA pushes its results to the CTA that combines them:
  // rows x2 in [d SH, (d + 1) SH) go to rank d, at entry rank SH + x2 mod SH of its buffer
  fft_run_last<L, 32, true>(v, t, sm, [] { cluster_arrive(); });
  cluster_wait();
  {
#pragma unroll
    for (int b = 0; b < Hh::B; b += 2)
#pragma unroll
      for (int r = 0; r < Hh::R; ++r) {
        const int x2 = Hh::idx(t, b, r);  // even: registers (b, r), (b + 1, r) hold x2, x2 + 1
        const float2 a = v[b * Hh::R + r], d = v[(b + 1) * Hh::R + r];
        const int slot = rank * SH + (x2 % SH);
        if (DOE_IN(slot >> 1, L / 2)) reinterpret_cast<float4*>(rsm(x2 / SH))[slot >> 1] = make_float4(a.x, a.y, d.x, d.y);
      }
  }
  cl.sync();
  // decimation-in-time combine over the sub-transforms, rows y = y1 L + y2 (pairs y2, y2 + 1),
  // from this CTA's own buffer
  const float4* r4 = reinterpret_cast<const float4*>(sm);
#pragma unroll
  for (int it = 0; it < SH / (2 * T); ++it) {
    const int y2l = 2 * t + it * 2 * T, y2 = rank * SH + y2l;
    float2 out[2][TC][Q];
#pragma unroll
    for (int sp = 0; sp < Q; ++sp) {
      const float2 w0 = wbig<P>(sp * y2), w1 = wbig<P>(sp * (y2 + 1));  // shared by the TC columns
#pragma unroll
      for (int cc = 0; cc < TC; ++cc) {
        const int ch = ((cc * Q + sp) * SH + y2l) >> 1;
        const float4 q4 = DOE_IN(ch, L / 2) ? r4[ch] : make_float4(0.f, 0.f, 0.f, 0.f);
        out[0][cc][sp] = cmulc(make_float2(q4.x, q4.y), w0);
        out[1][cc][sp] = cmulc(make_float2(q4.z, q4.w), w1);
      }
    }
#pragma unroll
    for (int cc = 0; cc < TC; ++cc) {
      dft<Q, true>(out[0][cc]);
      dft<Q, true>(out[1][cc]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int y1 = 0; y1 < Q; ++y1) {
        const int y = y1 * L + y2 + u;
        if ((unsigned)(y - yout0) < (unsigned)nout && DOE_IN((size_t)(y - yout0) * sl.wp + pos0 + TC - 1, sl.n_buf)) {
          if constexpr (TC >= 2) {
            float4* dst = reinterpret_cast<float4*>(sl.buf + (size_t)(y - yout0) * sl.wp + pos0);
#pragma unroll
            for (int f = 0; f < TC / 2; ++f)
              __stcs(dst + f, make_float4(out[u][2 * f][y1].x, out[u][2 * f][y1].y, out[u][2 * f + 1][y1].x,
                                          out[u][2 * f + 1][y1].y));
          } else {
            __stcs(sl.buf + (size_t)(y - yout0) * sl.wp + pos0, out[u][0][y1]);
          }
        }
      }
  }
  // no closing barrier: after the last cluster barrier no CTA touches another's shared memory
}

// ------------------------------------------------------------------ rows, adjoint (pass C')
template <int Q>
__global__ void __launch_bounds__(kBigL / 32, min_blocks(kBigL)) pass_c_adj_big_kernel(const __grid_constant__ Batch bt) {
  constexpr int L = kBigL, T = L / 32, P = L * Q, SH = L / Q, IT = SH / (2 * T);
  using G = Last<L, false>;
  extern __shared__ float2 sm[];
  __shared__ double red[32];
  cg::cluster_group cl = cg::this_cluster();
  const int s = (int)cl.block_rank();
  const int y = blockIdx.x / Q;
  const Slice& sl = bt.s[blockIdx.y];
  const int t = threadIdx.x;
  float4* rsm[Q];
#pragma unroll
  for (int c = 0; c < Q; ++c) rsm[c] = reinterpret_cast<float4*>(cl.map_shared_rank(sm, c));
  big_row_inverse_to_smem<Q>(sl, y, s, t, sm);
  cl.sync();
  float2 ga[IT][Q], gb[IT][Q];
#pragma unroll
  for (int it = 0; it < IT; ++it) big_combine<Q>(rsm, s * SH + 2 * t + it * 2 * T, ga[it], gb[it]);
  cl.sync();  // all reads of the inverse sub-transforms are done before they are overwritten
  const float sc = bt.inv_p2;
  const float* trow = sl.tgt + (size_t)y * P;
  float acc = 0.f;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int x2 = s * SH + 2 * t + it * 2 * T;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float2 tv = DOE_IN((size_t)y * P + (size_t)q * L + x2 + 1, sl.n_tgt)
                            ? __ldcs(reinterpret_cast<const float2*>(trow + (size_t)q * L + x2)) : make_float2(0.f, 0.f);
      const float2 ea = cscale(ga[it][q], sc), eb = cscale(gb[it][q], sc);
      float wa, wb;
      if (bt.mode == GRAD_L2) {
        const float da = fmaf(ea.x, ea.x, ea.y * ea.y) - tv.x, db = fmaf(eb.x, eb.x, eb.y * eb.y) - tv.y;
        acc = fmaf(da, da, fmaf(db, db, acc));
        wa = 2.f * da;
        wb = 2.f * db;
      } else {
        wa = tv.x;
        wb = tv.y;
      }
      ga[it][q] = cscale(ea, wa);
      gb[it][q] = cscale(eb, wb);
    }
    // forward decimation-in-frequency split of g over the chunks q
    dft<Q, false>(ga[it]);
    dft<Q, false>(gb[it]);
#pragma unroll
    for (int sp = 0; sp < Q; ++sp) {
      const float2 a = cmul(ga[it][sp], wbig<P>(x2 * sp)), b = cmul(gb[it][sp], wbig<P>((x2 + 1) * sp));
      if (DOE_IN(swz(x2 >> 1), L / 2)) rsm[sp][swz(x2 >> 1)] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  cl.sync();
  float2 v[32];
  stage_load<L, 32, false, 0>(v, t, sm);
  fft_run<L, 32, false>(v, t, sm);
#pragma unroll
  for (int b = 0; b < G::B; b += 2)
#pragma unroll
    for (int r = 0; r < G::R; ++r) {
      const float2 a = v[b * G::R + r], c = v[(b + 1) * G::R + r];
      const int pos = s * L + G::idx(t, b, r);  // J1 row y of the column-tiled buffer (P rows)
      if (DOE_IN(tiled_at(y, pos, P, kTile) + 1, sl.n_tbuf))
        __stcs(reinterpret_cast<float4*>(sl.tbuf + tiled_at(y, pos, P, kTile)), make_float4(a.x, a.y, c.x, c.y));
    }
  const double tot = block_sum<T>((double)acc, red);
  if (t == 0 && sl.loss_part && DOE_IN((size_t)y * Q + s, sl.n_loss)) sl.loss_part[(size_t)y * Q + s] = tot;
}

// ------------------------------------------------------------------ DOE rows, adjoint (pass A*)
template <int Q, bool ILLUM>
__global__ void __launch_bounds__(kBigL / 32, min_blocks(kBigL)) pass_a_adj_big_kernel(const __grid_constant__ Batch bt) {
  constexpr int L = kBigL, T = L / 32, SH = L / Q, IT = SH / (2 * T);
  extern __shared__ float2 sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int s = (int)cl.block_rank();
  const int i = blockIdx.x / Q;
  const int t = threadIdx.x, N = bt.N, off = bt.off;
  float4* rsm[Q];
#pragma unroll
  for (int c = 0; c < Q; ++c) rsm[c] = reinterpret_cast<float4*>(cl.map_shared_rank(sm, c));
  float acc[IT][Q][2];
#pragma unroll
  for (int it = 0; it < IT; ++it)
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[it][q][0] = acc[it][q][1] = 0.f;
  for (int j = 0; j < bt.S; ++j) {
    const Slice& sl = bt.s[j];
    if (j > 0) cl.sync();  // peers finished reading the previous slice's sub-transforms
    big_row_inverse_to_smem<Q>(sl, i, s, t, sm);
    cl.sync();
    const bool erow = sl.e_in != nullptr;
    const float k2 = -2.f * sl.kp_hi;
    IncRow ir = {0.f, 0u};
    if constexpr (ILLUM) ir = incident_row(sl, i - N / 2);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int x2 = s * SH + 2 * t + it * 2 * T;
      float2 oa[Q], ob[Q];
      big_combine<Q>(rsm, x2, oa, ob);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int x = q * L + x2 - off;  // even
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
          const float2 g0 = cscale(oa[q], bt.inv_p2), g1 = cscale(ob[q], bt.inv_p2);
          acc[it][q][0] = fmaf(k2, fmaf(g0.x, e0.y, -g0.y * e0.x), acc[it][q][0]);
          acc[it][q][1] = fmaf(k2, fmaf(g1.x, e1.y, -g1.y * e1.x), acc[it][q][1]);
        }
      }
    }
  }
  cl.sync();  // peers finished reading the last slice's sub-transforms
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int x2 = s * SH + 2 * t + it * 2 * T;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int x = q * L + x2 - off;
      if ((unsigned)x < (unsigned)N)
        if (DOE_IN((size_t)i * N + x + 1, bt.n_grad))
          *reinterpret_cast<float2*>(bt.grad + (size_t)i * N + x) = make_float2(acc[it][q][0], acc[it][q][1]);
    }
  }
}

}  // namespace doe
