// doe_mixed_big.cuh -- non-power-of-two sides longer than one CTA's transform, P = Q M with
// Q in {2, 3, 4, 5, 8, 16} and M <= 8192 (Table 2's 28800 = 8 x 3600 and 40000 = 8 x 5000 grids,
// and its 128640 x 85760 large-area grid, 16 x 8040 by 16 x 5360):
// every row / column transform of length P runs on a thread-block cluster of Q CTAs.
//
// Four-step split with n = M n1 + n2 (n1 < Q, n2 < M) and k = k1 + Q k2 (k1 < Q, k2 < M):
//   forward  y_k1[n2] = w_P^(n2 k1) sum_n1 x[M n1 + n2] w_Q^(n1 k1),   X[k1 + Q k2] = FFT_M(y_k1)[k2]
//   inverse  z_k1 = IFFT_M(X[k1 + Q .]),   x[M n1 + n2] = sum_k1 w_Q^(-n1 k1) w_P^(-n2 k1) z_k1[n2]
// CTA k1 of the cluster owns chunk k1 (y_k1 / z_k1) in shared memory and the n2 range
// [k1 ceil(M/Q), (k1 + 1) ceil(M/Q)) of the Q-point steps, whose inputs / outputs it exchanges
// with the other CTAs through distributed shared memory.  A row spectrum is stored in chunk
// order: position k1 M + k2 holds frequency k1 + Q k2 (rows and columns alike); the inverse
// transforms read that order back, and the transfer function is applied at the true
// frequencies.  Four-step twiddles come from a [P] table in the workspace (read through L1).
#pragma once
#include "doe_mixed.cuh"

namespace doe {

// 16-point DFT for the Q = 16 split steps, as 4 x 4 in registers (n = n1 + 4 n2, k = k2 + 4 k1):
//   X[k2 + 4 k1] = sum_n1 w_4^(n1 k1) [ w_16^(n1 k2) sum_n2 v[n1 + 4 n2] w_4^(n2 k2) ]
template <>
__device__ __forceinline__ void mr_dft<16>(float2 (&v)[16], bool inv) {
  float2 u[16];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    float2 a[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
    mr_dft<4>(a, inv);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      const float2 w = make_float2(wr_cos<16>(n1 * k2), inv ? wr_sin<16>(n1 * k2) : -wr_sin<16>(n1 * k2));
      u[n1 + 4 * k2] = (n1 && k2) ? cmul(a[k2], w) : a[k2];
    }
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 b[4] = {u[4 * k2], u[4 * k2 + 1], u[4 * k2 + 2], u[4 * k2 + 3]};
    mr_dft<4>(b, inv);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = b[k1];
  }
}

// One axis of a split transform: P = Q M points, sub-transforms of M, the [P] table w_P^m.
// Rows use the row axis (bt.P, bt.mr_M, bt.mr_twP), columns the column axis (bt.Py, bt.mr_My,
// bt.mr_twP_y); the two coincide on square grids.
struct MrqAxis {
  int P, M;
  const float2* twP;
};
__device__ __forceinline__ MrqAxis mrq_rows_axis(const Batch& bt) { return {bt.P, bt.mr_M, bt.mr_twP}; }
__device__ __forceinline__ MrqAxis mrq_cols_axis(const Batch& bt) { return {bt.Py, bt.mr_My, bt.mr_twP_y}; }

// w_P^(n2 k1) (n2 k1 < P), conjugated for the inverse
__device__ __forceinline__ float2 mrq_tw(const MrqAxis& ax, int n2, int k1, bool inv) {
  float2 w = DOE_IN(n2 * k1, ax.P) ? __ldg(ax.twP + n2 * k1) : make_float2(0.f, 0.f);
  if (inv) w.y = -w.y;
  return w;
}

// Forward Q-point step for n2: v[n1] = x[M n1 + n2] -> DFT over n1, times w_P^(n2 k1), written
// to CTA k1's buffer at n2.
template <int Q>
__device__ __forceinline__ void mrq_scatter_fwd(float2 (&v)[Q], int n2, const MrqAxis& ax, float2* const (&dst)[Q]) {
  mr_dft<Q>(v, false);
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1)
    if (DOE_IN(n2, ax.M)) dst[k1][n2] = cmul(v[k1], mrq_tw(ax, n2, k1, false));
}
// Inverse Q-point step for n2: z_k1[n2] from CTA k1, times w_P^(-n2 k1), IDFT over k1:
// v[n1] = x[M n1 + n2] (unnormalised).
template <int Q>
__device__ __forceinline__ void mrq_gather_inv(float2 (&v)[Q], int n2, const MrqAxis& ax, float2* const (&src)[Q]) {
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) v[k1] = DOE_IN(n2, ax.M) ? cmul(src[k1][n2], mrq_tw(ax, n2, k1, true)) : make_float2(0.f, 0.f);
  mr_dft<Q>(v, true);
}

// The cluster's view of one shared buffer: the same offset in every CTA.
template <int Q>
__device__ __forceinline__ void mrq_map(cg::cluster_group& cl, float2* local, float2* (&rem)[Q]) {
#pragma unroll
  for (int q = 0; q < Q; ++q) rem[q] = cl.map_shared_rank(local, q);
}

// ---- pass A (split): DOE row i -> its row spectrum in chunk order, tbuf row i.
template <int Q, bool CMP>
__global__ void __launch_bounds__(kMrT) mrq_rows_fwd_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  cg::cluster_group cl = cg::this_cluster();
  const int k1 = (int)cl.block_rank();
  const Slice& sl = bt.s[blockIdx.y];
  const int i = blockIdx.x / Q, t = threadIdx.x, N = bt.N, M = bt.mr_M, off = bt.off;
  float2* xa = mr_smem_setup<true>(sm_mr, bt, t);
  float2* xb = xa + M;
  float2* rem[Q];
  mrq_map<Q>(cl, xa, rem);
  const IncRow ir = incident_row(sl, i - bt.Ny / 2);
  const int Mc = (M + Q - 1) / Q, n2a = k1 * Mc, n2b = min(M, n2a + Mc);
  cluster_sync_relaxed();  // every CTA of the cluster runs before its shared memory is written
  for (int n2 = n2a + t; n2 < n2b; n2 += kMrT) {
    float2 v[Q];
#pragma unroll
    for (int n1 = 0; n1 < Q; ++n1) {
      const int x = M * n1 + n2 - off;
      v[n1] = (unsigned)x < (unsigned)N ? mr_doe_field(sl, i, x, N, ir) : make_float2(0.f, 0.f);
    }
    mrq_scatter_fwd<Q>(v, n2, mrq_rows_axis(bt), rem);
  }
  cl.sync();  // chunk k1 is complete in xa (and the twiddle table visible)
  const float2* y = mr_fft<CMP, false>(xa, xb, bt, mr_tws_of<true>(sm_mr, bt), false, t);
  float2* dst = sl.tbuf + (size_t)i * bt.P + (size_t)k1 * M;
  for (int c = t; c < M; c += kMrT)
    if (DOE_IN((size_t)i * bt.P + (size_t)k1 * M + c, sl.n_tbuf)) __stcs(dst + c, y[c]);
}

// ---- pass C (split): output row: chunk IFFTs, inverse Q-point step, 1/P^2, |E|^2 or E.
template <int Q, bool CMP>
__global__ void __launch_bounds__(kMrT) mrq_rows_out_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  cg::cluster_group cl = cg::this_cluster();
  const int k1 = (int)cl.block_rank();
  const Slice& sl = bt.s[blockIdx.y];
  const int row = blockIdx.x / Q, t = threadIdx.x, P = bt.P, M = bt.mr_M;
  float2* xa = mr_smem_setup<true>(sm_mr, bt, t);
  float2* xb = xa + M;
  const float2* src = sl.buf + (size_t)row * P + (size_t)k1 * M;
  for (int c = t; c < M; c += kMrT)
    xa[c] = DOE_IN((size_t)row * P + (size_t)k1 * M + c, sl.n_buf) ? __ldcs(src + c) : make_float2(0.f, 0.f);
  __syncthreads();
  float2* z = mr_fft<CMP, false>(xa, xb, bt, mr_tws_of<true>(sm_mr, bt), true, t);
  float2* rem[Q];
  mrq_map<Q>(cl, z, rem);
  cl.sync();  // every chunk is transformed
  const int Mc = (M + Q - 1) / Q, n2a = k1 * Mc, n2b = min(M, n2a + Mc);
  const float s = bt.inv_p2;
  for (int n2 = n2a + t; n2 < n2b; n2 += kMrT) {
    float2 v[Q];
    mrq_gather_inv<Q>(v, n2, mrq_rows_axis(bt), rem);
#pragma unroll
    for (int n1 = 0; n1 < Q; ++n1) {
      const float2 e = cscale(v[n1], s);
      const size_t at = (size_t)row * P + M * n1 + n2;
      if (!DOE_IN(at, sl.n_out)) continue;
      if (bt.mode == OUT_PSF) __stcs(static_cast<float*>(sl.out) + at, fmaf(e.x, e.x, e.y * e.y));
      else __stcs(static_cast<float2*>(sl.out) + at, e);
    }
  }
  cluster_sync_relaxed();  // the peers' reads of this CTA's chunk are done before it exits
}

// ---- pass C' (split): output row: E (inverse as in pass C), g = 2 (I - T) E (L2, loss partial per
// CTA) or (dL/dI) E, forward transform of g into tbuf row (chunk order).
template <int Q, bool CMP>
__global__ void __launch_bounds__(kMrT) mrq_rows_adj_c_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  __shared__ double red[32];
  cg::cluster_group cl = cg::this_cluster();
  const int k1 = (int)cl.block_rank();
  const Slice& sl = bt.s[blockIdx.y];
  const int row = blockIdx.x / Q, t = threadIdx.x, P = bt.P, M = bt.mr_M;
  float2* xa = mr_smem_setup<true>(sm_mr, bt, t);
  float2* xb = xa + M;
  const float2* src = sl.buf + (size_t)row * P + (size_t)k1 * M;
  for (int c = t; c < M; c += kMrT)
    xa[c] = DOE_IN((size_t)row * P + (size_t)k1 * M + c, sl.n_buf) ? __ldcs(src + c) : make_float2(0.f, 0.f);
  __syncthreads();
  float2* z = mr_fft<CMP, false>(xa, xb, bt, mr_tws_of<true>(sm_mr, bt), true, t);
  float2* w = z == xa ? xb : xa;  // the same buffer in every CTA (same plan)
  float2* remz[Q];
  float2* remw[Q];
  mrq_map<Q>(cl, z, remz);
  mrq_map<Q>(cl, w, remw);
  cl.sync();  // every chunk is transformed
  const int Mc = (M + Q - 1) / Q, n2a = k1 * Mc, n2b = min(M, n2a + Mc);
  const float s = bt.inv_p2;
  const float* trow = sl.tgt + (size_t)row * P;
  float acc = 0.f;
  for (int n2 = n2a + t; n2 < n2b; n2 += kMrT) {
    float2 v[Q];
    mrq_gather_inv<Q>(v, n2, mrq_rows_axis(bt), remz);
#pragma unroll
    for (int n1 = 0; n1 < Q; ++n1) {
      const float2 e = cscale(v[n1], s);
      const float tt = DOE_IN((size_t)row * P + M * n1 + n2, sl.n_tgt) ? __ldcs(trow + M * n1 + n2) : 0.f;
      float g;
      if (bt.mode == GRAD_L2) {
        const float d = fmaf(e.x, e.x, e.y * e.y) - tt;
        acc = fmaf(d, d, acc);
        g = 2.f * d;
      } else {
        g = tt;
      }
      v[n1] = cscale(e, g);
    }
    mrq_scatter_fwd<Q>(v, n2, mrq_rows_axis(bt), remw);
  }
  cl.sync();  // w holds chunk k1 of the forward step in every CTA; reads of z are done
  const float2* y = mr_fft<CMP, false>(w, z, bt, mr_tws_of<true>(sm_mr, bt), false, t);
  float2* dst = sl.tbuf + (size_t)row * P + (size_t)k1 * M;
  for (int c = t; c < M; c += kMrT)
    if (DOE_IN((size_t)row * P + (size_t)k1 * M + c, sl.n_tbuf)) __stcs(dst + c, y[c]);
  const double tot = block_sum<kMrT>((double)acc, red);
  if (t == 0 && sl.loss_part && DOE_IN((size_t)row * Q + k1, sl.n_loss)) sl.loss_part[(size_t)row * Q + k1] = tot;
}

// ---- pass A* (split): DOE row i summed over the slices: inverse of tbuf row i (chunk order),
// 1/P^2, dL/dh += -2 k' Im(conj(g_doe) E_doe) on the DOE columns this thread owns.
template <int Q, bool CMP>
__global__ void __launch_bounds__(kMrT) mrq_rows_adj_a_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  cg::cluster_group cl = cg::this_cluster();
  const int k1 = (int)cl.block_rank();
  const int i = blockIdx.x / Q, t = threadIdx.x, N = bt.N, P = bt.P, M = bt.mr_M, off = bt.off;
  float2* xa = mr_smem_setup<true>(sm_mr, bt, t);
  float2* xb = xa + M;
  const int Mc = (M + Q - 1) / Q, n2a = k1 * Mc, n2b = min(M, n2a + Mc);
  float* grow = bt.grad + (size_t)i * N;
  for (int j = 0; j < bt.S; ++j) {
    const Slice& sl = bt.s[j];
    const float2* src = sl.tbuf + (size_t)i * P + (size_t)k1 * M;
    for (int c = t; c < M; c += kMrT)
      xa[c] = DOE_IN((size_t)i * P + (size_t)k1 * M + c, sl.n_tbuf) ? __ldcs(src + c) : make_float2(0.f, 0.f);
    __syncthreads();
    float2* z = mr_fft<CMP, false>(xa, xb, bt, mr_tws_of<true>(sm_mr, bt), true, t);
    float2* rem[Q];
    mrq_map<Q>(cl, z, rem);
    cl.sync();  // every chunk of this slice is transformed
    const IncRow ir = incident_row(sl, i - bt.Ny / 2);
    const float k2 = -2.f * sl.kp_hi;
    for (int n2 = n2a + t; n2 < n2b; n2 += kMrT) {
      float2 v[Q];
      mrq_gather_inv<Q>(v, n2, mrq_rows_axis(bt), rem);
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) {
        const int x = M * n1 + n2 - off;
        if ((unsigned)x < (unsigned)N && DOE_IN((size_t)i * N + x, bt.n_grad)) {
          const float2 e = mr_doe_field(sl, i, x, N, ir);
          const float2 g = cscale(v[n1], bt.inv_p2);
          const float prev = j ? grow[x] : 0.f;
          grow[x] = fmaf(k2, fmaf(g.x, e.y, -g.y * e.x), prev);
        }
      }
    }
    cl.sync();  // the peers' reads are done before the buffers are reused (or the CTA exits)
  }
}

// ---- pass B / B* (split): TC adjacent columns c0 + cc (stored positions; true frequencies
// mrq_freq(c)) over a cluster of TC Q CTAs, rank cc Q + k1.  Forward: padded rows M n1 + n2 from
// the DOE rows of tbuf (rows off..off+N-1), forward transform, x H, inverse, all P rows to buf.
// Adjoint: all P rows of tbuf, x conj(H), rows off..off+N-1 back to tbuf rows 0..N-1 (the
// cluster owns its columns).  With TC = 2 the columns' samples of a row are read and written
// together as one 16-byte pair; the Q-point steps of each n2 are done by one CTA for both.
template <int Q, int TC, bool CMP>
__global__ void __launch_bounds__(kMrT) mrq_cols_kernel(const __grid_constant__ Batch bt) {
  static_assert(TC == 1 || TC == 2, "one or two columns per cluster");
  constexpr int CL = TC * Q;
  extern __shared__ float2 sm_mr[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), cc = rank / Q, k1 = rank % Q;
  const Slice& sl = bt.s[blockIdx.y];
  // the column axis: Py = Q M rows (Ny DOE rows at offset offy), rows of Px = bt.P samples
  const int c0 = (blockIdx.x / CL) * TC, c = c0 + cc, t = threadIdx.x, N = bt.Ny, Px = bt.P, P = bt.Py, M = bt.mr_My,
            off = bt.offy;
  const bool adj = bt.mode == MODE_ADJ;
  float2* xa = mr_smem_setup<true>(sm_mr, bt, t, true);
  float2* xb = xa + M;
  const int Mc = (M + CL - 1) / CL, n2a = rank * Mc, n2b = min(M, n2a + Mc);
  cluster_sync_relaxed();  // every CTA of the cluster runs before its shared memory is written
  {
    float2* rem[TC][Q];
#pragma unroll
    for (int u = 0; u < TC; ++u)
#pragma unroll
      for (int q = 0; q < Q; ++q) rem[u][q] = cl.map_shared_rank(xa, u * Q + q);
    for (int n2 = n2a + t; n2 < n2b; n2 += kMrT) {
      float2 v[TC][Q];
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) {
        const int r = M * n1 + n2 - (adj ? 0 : off);
        const bool in = (unsigned)r < (unsigned)(adj ? P : N) && DOE_IN((size_t)r * Px + c0 + TC - 1, sl.n_tbuf);
        if constexpr (TC == 2) {
          const float4 w = in ? __ldcs(reinterpret_cast<const float4*>(sl.tbuf + (size_t)r * Px + c0))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
          v[0][n1] = make_float2(w.x, w.y);
          v[1][n1] = make_float2(w.z, w.w);
        } else {
          v[0][n1] = in ? __ldcs(sl.tbuf + (size_t)r * Px + c0) : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < TC; ++u) mrq_scatter_fwd<Q>(v[u], n2, mrq_cols_axis(bt), rem[u]);
    }
  }
  cl.sync();  // chunk k1 of column c is complete in xa
  float2* y = mr_fft<CMP, false>(xa, xb, bt, mr_tws_of<true>(sm_mr, bt), false, t, true);
  // the column's frequency: rows are stored in chunk order when the row transform is split
  const int kc = bt.mr_Q > 1 ? mrq_freq(c, bt.mr_Q, bt.mr_M) : c;
  for (int k2 = t; k2 < M; k2 += kMrT) y[k2] = cmul(y[k2], mr_transfer(sl, kc, k1 + Q * k2, Px, P, adj));
  __syncthreads();
  float2* z = mr_fft<CMP, false>(y, y == xa ? xb : xa, bt, mr_tws_of<true>(sm_mr, bt), true, t, true);
  cl.sync();  // every chunk is back in the row domain
  {
    float2* remz[TC][Q];
#pragma unroll
    for (int u = 0; u < TC; ++u)
#pragma unroll
      for (int q = 0; q < Q; ++q) remz[u][q] = cl.map_shared_rank(z, u * Q + q);
    for (int n2 = n2a + t; n2 < n2b; n2 += kMrT) {
      float2 v[TC][Q];
#pragma unroll
      for (int u = 0; u < TC; ++u) mrq_gather_inv<Q>(v[u], n2, mrq_cols_axis(bt), remz[u]);
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) {
        const int r = M * n1 + n2;
        const int ro = adj ? r - off : r;  // output row
        if (adj ? (unsigned)ro >= (unsigned)N : false) continue;
        float2* dst = adj ? sl.tbuf : sl.buf;
        if (!DOE_IN((size_t)ro * Px + c0 + TC - 1, adj ? sl.n_tbuf : sl.n_buf)) continue;
        if constexpr (TC == 2)
          __stcs(reinterpret_cast<float4*>(dst + (size_t)ro * Px + c0), make_float4(v[0][n1].x, v[0][n1].y, v[1][n1].x, v[1][n1].y));
        else
          __stcs(dst + (size_t)ro * Px + c0, v[0][n1]);
      }
    }
  }
  cl.sync();  // the peers' reads of this CTA's chunk are done before it exits
}

}  // namespace doe
