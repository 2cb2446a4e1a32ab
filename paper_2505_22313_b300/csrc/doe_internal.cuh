// doe_internal.cuh -- kernel parameter blocks and device helpers shared by the passes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "doe_async.cuh"
#include "doe_fft.cuh"
#include "doe_plan.h"

namespace doe {

// ------------------------------------------------------------------ double-float arithmetic
// A value is hi + lo with |lo| <= ulp(hi) / 2 (about 48 significant bits).  Error-free
// transformations: Knuth's two-sum, and the FMA two-product.  B300 runs FP64 at 1/64 of the
// FP32 rate, so the transfer-function phase (up to ~1e6 rad) is evaluated in this format.
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = two_sum(x.hi, y.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  dfl p = two_prod(x.hi, y.hi);
  float e = __fadd_rn(p.lo, fmaf(x.hi, y.lo, __fmul_rn(x.lo, y.hi)));
  return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dfl df_mul_f(dfl x, float f) {
  dfl p = two_prod(x.hi, f);
  float e = fmaf(x.lo, f, p.lo);
  return fast_two_sum(p.hi, e);
}

constexpr float kTwoPiHi = 6.28318548202514648438f;        // float(2 pi)
constexpr float kTwoPiLo = -1.7484555314695172e-07f;       // 2 pi - float(2 pi)
constexpr float kInvTwoPi = 0.15915494309189533577f;

// Transfer function H at integer frequencies with m = kt^2 + lt^2 (Eq. 3's H_lambda, the
// band-limited angular spectrum: exp(+i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2))).  Written as
// phi = phi0 sqrt(1 - q), q = c m, and evaluated as phi0 - phi0 q / (1 + sqrt(1 - q)) so that
// no large phase is ever rounded to FP32: the drop phi0 g (g = q / (1 + sqrt(1 - q))) is kept
// in double-float, reduced mod 2 pi in double-float, and subtracted from phi0 mod 2 pi
// (computed on the host in FP64).  The caller has checked m < mev (propagating sample).
// The phase from q = c m in double-float (the steps below transfer_value's product).
__device__ __forceinline__ float2 transfer_from_q(dfl q, const Slice& s);
__device__ __forceinline__ float2 transfer_value(unsigned int m, const Slice& s) {
  const float m_hi = (float)(m & 0xFFFFF000u);  // exact: at most 20 significant bits
  const float m_lo = (float)(m & 0x00000FFFu);  // exact
  const dfl c = {s.c_hi, s.c_lo};
  return transfer_from_q(df_add(df_mul_f(c, m_hi), df_mul_f(c, m_lo)), s);
}
// Rectangular grids: m = kt^2 sqb + lt^2 sqa < 2^50, split into three exactly representable
// 24-bit parts.
__device__ __forceinline__ float2 transfer_value64(unsigned long long m, const Slice& s) {
  const float m0 = (float)(m & 0xFFFFFFull);                // exact: 24 bits
  const float m1 = (float)(m & 0xFFFFFF000000ull);          // exact: 24 significant bits
  const float m2 = (float)(m & 0xFFFF000000000000ull);      // exact
  const dfl c = {s.c_hi, s.c_lo};
  return transfer_from_q(df_add(df_add(df_mul_f(c, m2), df_mul_f(c, m1)), df_mul_f(c, m0)), s);
}
__device__ __forceinline__ float2 transfer_from_q(dfl q, const Slice& s) {
  const dfl u = df_add({1.f, 0.f}, df_neg(q));  // 1 - q in (0, 1]
  // sqrt(u): one Newton step from the FP32 root doubles the precision
  const float s0 = sqrtf(u.hi);
  const dfl s0sq = two_prod(s0, s0);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(u.hi, s0sq.hi), s0sq.lo), u.lo);
  const dfl sq = fast_two_sum(s0, __fmul_rn(r, __fdiv_rn(0.5f, s0)));
  const dfl d = df_add({1.f, 0.f}, sq);  // in [1, 2]
  // g = q / d: FP32 quotient corrected by one residual step
  const float g0 = __fdiv_rn(q.hi, d.hi);
  const dfl res = df_add(q, df_neg(df_mul_f(d, g0)));
  const dfl g = fast_two_sum(g0, __fdiv_rn(res.hi, d.hi));
  const dfl dphi = df_mul({s.phi0_hi, s.phi0_lo}, g);  // phase drop below the on-axis phase
  const float n = rintf(__fmul_rn(dphi.hi, kInvTwoPi));
  const dfl t = df_add(dphi, df_mul_f({-kTwoPiHi, -kTwoPiLo}, n));  // dphi mod 2 pi
  const float th = __fadd_rn(__fsub_rn(s.th0_hi, t.hi), __fsub_rn(s.th0_lo, t.lo));
  float sn, cs;
  sincosf(th, &sn, &cs);
  return make_float2(cs, sn);
}

// Phase of the transmittance exp(+i k' h) (Eq. 1-2).  k' h is formed exactly as a float pair
// (FMA two-product) and wrapped to (-pi, pi] in that format, then rounded once.
__device__ __forceinline__ float trans_phase(float hv, float kp_hi, float kp_lo) {
  const dfl p = two_prod(kp_hi, hv);
  const float e = fmaf(kp_lo, hv, p.lo);
  const float n = rintf(__fmul_rn(p.hi, kInvTwoPi));
  const float r = fmaf(-n, kTwoPiHi, p.hi);  // exact (Sterbenz): |p.hi - n 2pi_hi| is small
  return __fadd_rn(r, fmaf(-n, kTwoPiLo, e));
}
__device__ __forceinline__ float2 transmittance(float hv, float kp_hi, float kp_lo) {
  float sn, cs;
  sincosf(trans_phase(hv, kp_hi, kp_lo), &sn, &cs);
  return make_float2(cs, sn);
}

// ------------------------------------------------------------------ parametric incident field
// E_in of Eq. 2 as a tilted plane wave times an on-axis spherical wave, at DOE sample
// (yy, xx) = (i - N/2, x - N/2) (the optical axis at padded index P/2):
//   tilt:   exp(+i 2 pi (a xx + b yy)),  a = dx sin(theta_x) / lambda, b = dx sin(theta_y) / lambda
//   sphere: (|d| / r) exp(+i sgn(d) 2 pi (r - |d|) / lambda),  r = sqrt(rho^2 + d^2)
// Phases are kept in cycles and reduced to their fractional parts in double-float, so that
// tens of thousands of cycles across a large aperture cost no accuracy.

// Fractional part of a n (a = a_hi + a_lo, n an integer with |n| <= 2^24), in cycles,
// |result| <= 1/2 + |a_lo n|.
__device__ __forceinline__ float frac_cycles(float a_hi, float a_lo, float n) {
  const dfl p = two_prod(a_hi, n);
  const float r = __fsub_rn(p.hi, rintf(p.hi));  // exact: p.hi and its nearest integer share a binade grid
  return __fadd_rn(r, fmaf(a_lo, n, p.lo));
}

// The part of the incident field shared by DOE row yy: its tilt cycles and yy^2.
struct IncRow {
  float cy;
  unsigned int yy2;
};
__device__ __forceinline__ IncRow incident_row(const Slice& s, int yy) {
  IncRow r;
  r.cy = (s.illum & ILLUM_TILT) ? frac_cycles(s.tb_hi, s.tb_lo, (float)yy) : 0.f;
  r.yy2 = (unsigned int)(yy * yy);
  return r;
}

// Phase (radians, |th| <= pi) and amplitude of the incident field at column xx of row r.
// Spherical term: with u = (dx / d)^2 (xx^2 + yy^2) = rho^2 / d^2, (r - |d|) / lambda =
// (|d| / lambda) u / (1 + sqrt(1 + u)) (no cancellation), evaluated in double-float.
__device__ __forceinline__ float incident_phase(const Slice& s, IncRow r, int xx, float& amp) {
  float cyc = r.cy;
  if (s.illum & ILLUM_TILT) cyc = __fadd_rn(cyc, frac_cycles(s.ta_hi, s.ta_lo, (float)xx));
  amp = 1.f;
  if (s.illum & ILLUM_SPHERE) {
    const unsigned int m = r.yy2 + (unsigned int)(xx * xx);  // < 2^31 + 2^30
    const float m_hi = (float)(m & 0xFFFFF000u);                // exact: at most 20 significant bits
    const float m_lo = (float)(m & 0x00000FFFu);                // exact
    const dfl c = {s.sc_hi, s.sc_lo};
    const dfl u = df_add(df_mul_f(c, m_hi), df_mul_f(c, m_lo));
    const dfl w = df_add({1.f, 0.f}, u);  // 1 + u
    // sqrt(1 + u): one Newton step from the approximate root w rsqrt(w); the step squares the
    // starting error (a few ulp), so approximate reciprocals suffice in the corrections
    const float rs = rsqrtf(w.hi);
    const float s0 = __fmul_rn(w.hi, rs);
    const dfl s0sq = two_prod(s0, s0);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(w.hi, s0sq.hi), s0sq.lo), w.lo);
    const dfl sq = fast_two_sum(s0, __fmul_rn(res, __fmul_rn(0.5f, rs)));
    const dfl den = df_add({1.f, 0.f}, sq);  // >= 2
    // q = u / (1 + sqrt(1 + u)): approximate quotient corrected by one residual step
    const float inv = __fdividef(1.f, den.hi);
    const float q0 = __fmul_rn(u.hi, inv);
    const dfl rq = df_add(u, df_neg(df_mul_f(den, q0)));
    const dfl q = fast_two_sum(q0, __fmul_rn(rq.hi, inv));
    const dfl t = df_mul({s.sk_hi, s.sk_lo}, q);  // (r - |d|) / lambda, cycles
    const float f = __fadd_rn(__fsub_rn(t.hi, rintf(t.hi)), t.lo);
    cyc = fmaf(s.ssgn, f, cyc);
    amp = rs;  // |d| / r = 1 / sqrt(1 + u), to a few ulp
  }
  cyc = __fsub_rn(cyc, rintf(cyc));  // exact
  return fmaf(cyc, kTwoPiHi, __fmul_rn(cyc, kTwoPiLo));
}

// Transmittance times the parametric incident field, one sincosf for both phases.
__device__ __forceinline__ float2 transmittance_inc(float hv, const Slice& s, IncRow r, int xx) {
  float amp;
  const float th = __fadd_rn(trans_phase(hv, s.kp_hi, s.kp_lo), incident_phase(s, r, xx, amp));
  float sn, cs;
  sincosf(th, &sn, &cs);
  return make_float2(amp * cs, amp * sn);
}

// Heights of the adjacent simulation samples (x, x + 1), x even, of DOE row i: without
// upsampling one 8-byte load; with nearest upsampling by 2^uf (uf >= 1) both samples lie in the
// same layout cell x >> uf.
__device__ __forceinline__ float2 heights_pair(const Slice& s, int N, int i, int x) {
  const size_t o = (size_t)(i >> s.uf) * (N >> s.uf) + (x >> s.uf);  // layout cell of DOE row i
  if (s.uf == 0)
    return DOE_IN(o + 1, s.n_h) ? __ldcs(reinterpret_cast<const float2*>(s.h + o)) : make_float2(0.f, 0.f);
  const float h = DOE_IN(o, s.n_h) ? __ldcs(s.h + o) : 0.f;
  return make_float2(h, h);
}
// Incident field array values at DOE samples (x, x + 1) of row i (x even): one 16-byte load.
__device__ __forceinline__ float4 ein_pair(const Slice& s, int N, int i, int x) {
  const size_t o = (size_t)i * N + x;
  return DOE_IN(o + 1, s.n_ein) ? __ldcs(reinterpret_cast<const float4*>(s.e_in + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Cluster barrier without memory ordering, for a point where no CTA publishes data: the
// arriving CTA's reads of its peers' shared memory have all been consumed (their values are
// already used by its later instructions), and the barrier only keeps a peer from reusing or
// releasing that memory early.  Unlike the default (release / acquire) barrier it does not
// wait for the CTA's outstanding global stores.
__device__ __forceinline__ void cluster_sync_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}
// The two halves of a cluster barrier, for work placed between them: the arrival releases this
// thread's earlier memory accesses (shared-memory reads included), the wait acquires every
// other thread's.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

// Position of entry a (= |lt|) in a row of the transfer-function table.  Split grids group a
// row by residue mod Q (the cluster size of their column pass): entry a at (a mod Q) hq + a / Q,
// so CTA s of a column cluster, which needs the frequencies s + Q k2, reads a contiguous run.
__device__ __forceinline__ int htab_col(const Slice& s, int a) {
  return s.hqs ? (a & ((1 << s.hqs) - 1)) * s.hq + (a >> s.hqs) : a;
}

// Stored (band-compacted) spectrum rows.  With the band limit active a row keeps the two
// FFT-order segments [0, seg_a) and [P - (w - seg_a), P), seg_a = kmax + 1 and
// w - seg_a = kmax, each rounded up to even length so that pairs of adjacent frequencies
// (k, k + 1), k even, are always stored together at an even (16-byte aligned) position.  The
// at most two stored entries outside the band (|kt| > kmax) hold zeros.  Without the band
// limit w = P and positions equal frequency indices.
__device__ __forceinline__ int band_pos(int k, int P, int seg_a, int w) {
  if (k < seg_a) return k;
  if (k >= P - (w - seg_a)) return k - (P - w);
  return -1;
}
__device__ __forceinline__ int pos_to_k(int pos, int P, int seg_a, int w) {
  return pos < seg_a ? pos : pos + (P - w);
}
__device__ __forceinline__ int abs_signed(int k, int P) { return k < P / 2 ? k : P - k; }

// Column-tiled layout of a spectrum with R rows: stored positions are grouped in tiles of TC
// adjacent positions, and each tile holds its R rows contiguously (TC samples per row), so
// the column pass reads one tile as a single contiguous block.  float2 index of (row, pos):
__device__ __forceinline__ size_t tiled_at(int row, int pos, int R, int TC) {
  return ((size_t)(pos / TC) * R + row) * TC + (pos % TC);
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

}  // namespace doe
