// doe_mixed.cuh -- grids whose side P is not a power of two (P <= 8192 even, with factors 2, 3, 5
// and primes up to 127, e.g. the 67 of Table 2's large-area grid):
// the same propagation, PSF and adjoint as the power-of-two passes (Eq. 1-4), on a generic
// mixed-radix FFT held in shared memory.  Table 2's 3600 x 3600 grid is of this kind.
//
// FFT: Stockham autosort, one stage per radix of the host plan: 2, 3, 4, 5, 8, the composites
// 9, 15, 16, 25 (split in registers), and a direct-DFT stage for each larger prime factor.  Stage
// with Ns = product of the earlier radices: butterfly j < P/R reads x[j + r P/R] (r < R),
// multiplies input r by w_P^(r k P/(Ns R)) (k = j mod Ns), takes the R-point DFT and writes
// output r to y[(j - k) R + k + r Ns].  The stage twiddles w_(Ns R)^(r k) come from a per-stage
// table laid out [stage][r][k] (mr_stage_twiddle_kernel; M - 1 entries in all, since the stages'
// (R - 1) Ns sum to M - 1): the lanes of a warp, which hold consecutive k, read consecutive
// entries (one 256-byte run per warp and radix term), through L1 in the one-CTA passes and from
// a shared copy in the cluster-split passes of doe_mixed_big.cuh.  The composite stages' inner
// twiddles w_R^m are compile-time constants; the direct-DFT stages of larger primes read the
// table of all P powers w_P^m from global memory.  Both tables are built per call in FP64.
// Stages go out of place between two shared buffers (one barrier per stage), one butterfly in
// registers at a time.
//
// Buffers (natural row-major layout, rows of Px samples): tbuf holds the row spectra of the Ny
// DOE rows (forward) or of all Py rows (adjoint), buf the field after the column pass.  Square
// grids have Px = Py; rectangles use a row plan (Px) and a column plan (Py).  The column pass
// runs on clusters of 4 CTAs when Px is a multiple of 4 (mr_cols4_kernel), else one CTA per
// column (mr_cols_kernel).
#pragma once
#include "doe_kernels.cuh"

namespace doe {


// frequency index of the stored position p = k1 M + k2 of a spectrum split over Q sub-transforms
// of M points (stored in chunk order)
__device__ __forceinline__ int mrq_freq(int p, int Q, int M) { return p / M + Q * (p % M); }

struct MrRadices {  // a plan's radices, by value (kernel argument)
  int r[kMrMaxStages];
};

// Twiddle table w_P^m, m < P, from FP64 sincospi of the exact ratio 2 m / P.
__global__ void __launch_bounds__(256) mr_twiddle_kernel(float2* __restrict__ tw, int P) {
  const int m = blockIdx.x * 256 + threadIdx.x;
  if (m >= P) return;
  double s, c;
  sincospi(-2.0 * (double)m / (double)P, &s, &c);
  tw[m] = make_float2((float)c, (float)s);
}

// Per-stage twiddles of a plan of M (radices R_s): stage s with sub-transform size Ns holds
// w_(Ns R)^(r k) = exp(-2 pi i r k / (Ns R)) at (Ns - 1) + (r - 1) Ns + k (1 <= r < R, k < Ns),
// from FP64 sincospi of the exact ratio.  One thread per entry, e < M - 1.
__global__ void __launch_bounds__(256) mr_stage_twiddle_kernel(float2* __restrict__ tws, int M, int nst,
                                                               MrRadices rad) {
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e >= M - 1) return;
  int Ns = 1, s = 0;
  while (s + 1 < nst && e >= Ns * rad.r[s] - 1) Ns *= rad.r[s++];  // stage s covers [Ns - 1, Ns R - 1)
  const int R = rad.r[s], o = e - (Ns - 1);
  const int r = 1 + o / Ns, k = o % Ns;
  double sn, cs;
  sincospi(-2.0 * (double)((long long)r * k) / ((double)Ns * R), &sn, &cs);
  tws[e] = make_float2((float)cs, (float)sn);
}

// R-point DFTs (forward kernel exp(-2 pi i n k / R); inv: exp(+...)), written from the
// definition with the symmetric pairs folded.
__device__ __forceinline__ float2 mr_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 mr_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// -i s a (s = +1) or +i a (s = -1): the rotation shared by every odd-order term
__device__ __forceinline__ float2 mr_rot(float2 a, float s) { return make_float2(s * a.y, -s * a.x); }

template <int R>
__device__ __forceinline__ void mr_dft(float2 (&v)[R], bool inv);

template <>
__device__ __forceinline__ void mr_dft<2>(float2 (&v)[2], bool) {
  const float2 a = v[0], b = v[1];
  v[0] = mr_add(a, b);
  v[1] = mr_sub(a, b);
}

template <>
__device__ __forceinline__ void mr_dft<3>(float2 (&v)[3], bool inv) {
  const float s = inv ? -1.f : 1.f;
  const float kS3 = 0.86602540378443864676f;  // sin(2 pi / 3)
  const float2 t1 = mr_add(v[1], v[2]);
  const float2 t2 = make_float2(fmaf(-0.5f, t1.x, v[0].x), fmaf(-0.5f, t1.y, v[0].y));
  const float2 d = mr_rot(mr_sub(v[1], v[2]), s);  // -i s (v1 - v2)
  v[0] = mr_add(v[0], t1);
  v[1] = make_float2(fmaf(kS3, d.x, t2.x), fmaf(kS3, d.y, t2.y));
  v[2] = make_float2(fmaf(-kS3, d.x, t2.x), fmaf(-kS3, d.y, t2.y));
}

template <>
__device__ __forceinline__ void mr_dft<4>(float2 (&v)[4], bool inv) {
  const float s = inv ? -1.f : 1.f;
  const float2 t0 = mr_add(v[0], v[2]), t1 = mr_sub(v[0], v[2]);
  const float2 t2 = mr_add(v[1], v[3]), t3 = mr_rot(mr_sub(v[1], v[3]), s);
  v[0] = mr_add(t0, t2);
  v[2] = mr_sub(t0, t2);
  v[1] = mr_add(t1, t3);
  v[3] = mr_sub(t1, t3);
}

template <>
__device__ __forceinline__ void mr_dft<5>(float2 (&v)[5], bool inv) {
  const float s = inv ? -1.f : 1.f;
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;  // cos(2 pi / 5), cos(4 pi / 5)
  const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;   // sin(2 pi / 5), sin(4 pi / 5)
  const float2 a1 = mr_add(v[1], v[4]), b1 = mr_sub(v[1], v[4]);
  const float2 a2 = mr_add(v[2], v[3]), b2 = mr_sub(v[2], v[3]);
  const float2 x0 = v[0];
  // X1, X4 = x0 + c1 a1 + c2 a2 -+ i s (s1 b1 + s2 b2); X2, X3 = x0 + c2 a1 + c1 a2 -+ i s (s2 b1 - s1 b2)
  const float2 p1 = make_float2(fmaf(c2, a2.x, fmaf(c1, a1.x, x0.x)), fmaf(c2, a2.y, fmaf(c1, a1.y, x0.y)));
  const float2 p2 = make_float2(fmaf(c1, a2.x, fmaf(c2, a1.x, x0.x)), fmaf(c1, a2.y, fmaf(c2, a1.y, x0.y)));
  const float2 q1 = mr_rot(make_float2(fmaf(s2, b2.x, s1 * b1.x), fmaf(s2, b2.y, s1 * b1.y)), s);
  const float2 q2 = mr_rot(make_float2(fmaf(-s1, b2.x, s2 * b1.x), fmaf(-s1, b2.y, s2 * b1.y)), s);
  v[0] = mr_add(x0, mr_add(a1, a2));
  v[1] = mr_add(p1, q1);
  v[4] = mr_sub(p1, q1);
  v[2] = mr_add(p2, q2);
  v[3] = mr_sub(p2, q2);
}

template <>
__device__ __forceinline__ void mr_dft<8>(float2 (&v)[8], bool inv) {
  // two 4-point DFTs (even and odd inputs), combined with w_8^k
  const float s = inv ? -1.f : 1.f;
  const float kH = 0.70710678118654752440f;  // sqrt(1/2)
  float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  mr_dft<4>(e, inv);
  mr_dft<4>(o, inv);
  // w_8 = sqrt(1/2) (1 - i s), w_8^2 = -i s, w_8^3 = sqrt(1/2) (-1 - i s)
  const float2 o1 = make_float2(kH * (o[1].x + s * o[1].y), kH * (o[1].y - s * o[1].x));
  const float2 o2 = mr_rot(o[2], s);
  const float2 o3 = make_float2(kH * (-o[3].x + s * o[3].y), kH * (-o[3].y - s * o[3].x));
  v[0] = mr_add(e[0], o[0]);
  v[4] = mr_sub(e[0], o[0]);
  v[1] = mr_add(e[1], o1);
  v[5] = mr_sub(e[1], o1);
  v[2] = mr_add(e[2], o2);
  v[6] = mr_sub(e[2], o2);
  v[3] = mr_add(e[3], o3);
  v[7] = mr_sub(e[3], o3);
}

// One Stockham stage of radix R: src -> dst (both P samples of shared memory), see the file
// comment; ends with a barrier so that dst is visible.  One butterfly in registers at a time.
// tws: this stage's twiddle rows, w_(Ns R)^(r k) at (r - 1) Ns + k (GTW: in global memory, read
// through L1; else in shared memory).
template <int R, bool GTW>
__device__ __forceinline__ void mr_stage(const float2* src, float2* dst, int P, int Ns, const float2* tws, bool inv,
                                         int t) {
  const int nb = P / R;
#pragma unroll 2
  for (int j = t; j < nb; j += kMrT) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = DOE_IN(j + r * nb, P) ? src[j + r * nb] : make_float2(0.f, 0.f);
    const int k = j % Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = DOE_IN((Ns - 1) + (r - 1) * Ns + k, P) ? (GTW ? __ldg(tws + (r - 1) * Ns + k) : tws[(r - 1) * Ns + k]) : make_float2(0.f, 0.f);
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    mr_dft<R>(v, inv);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (DOE_IN(base + r * Ns, P)) dst[base + r * Ns] = v[r];
  }
  __syncthreads();
}

// cos and sin of 2 pi m / R (m < R): the inner twiddles w_R^m = cos - i sin of the composite
// radices 9, 15, 16, 25 (mathematical constants, rounded to FP32).
template <int R>
__host__ __device__ constexpr float wr_cos(int m) {
  if constexpr (R == 9) {
    constexpr float c[9] = {1.000000000f, 7.660444431e-1f, 1.736481777e-1f, -5.000000000e-1f, -9.396926208e-1f, -9.396926208e-1f, -5.000000000e-1f, 1.736481777e-1f, 7.660444431e-1f};
    return c[m];
  } else if constexpr (R == 15) {
    constexpr float c[15] = {1.000000000f, 9.135454576e-1f, 6.691306064e-1f, 3.090169944e-1f, -1.045284633e-1f, -5.000000000e-1f, -8.090169944e-1f, -9.781476007e-1f, -9.781476007e-1f, -8.090169944e-1f, -5.000000000e-1f, -1.045284633e-1f, 3.090169944e-1f, 6.691306064e-1f, 9.135454576e-1f};
    return c[m];
  } else if constexpr (R == 16) {
    constexpr float c[16] = {1.000000000f, 9.238795325e-1f, 7.071067812e-1f, 3.826834324e-1f, 0.f, -3.826834324e-1f, -7.071067812e-1f, -9.238795325e-1f, -1.000000000f, -9.238795325e-1f, -7.071067812e-1f, -3.826834324e-1f, 0.f, 3.826834324e-1f, 7.071067812e-1f, 9.238795325e-1f};
    return c[m];
  } else if constexpr (R == 25) {
    constexpr float c[25] = {1.000000000f, 9.685831611e-1f, 8.763066800e-1f, 7.289686274e-1f, 5.358267950e-1f, 3.090169944e-1f, 6.279051953e-2f, -1.873813146e-1f, -4.257792916e-1f, -6.374239897e-1f, -8.090169944e-1f, -9.297764859e-1f, -9.921147013e-1f, -9.921147013e-1f, -9.297764859e-1f, -8.090169944e-1f, -6.374239897e-1f, -4.257792916e-1f, -1.873813146e-1f, 6.279051953e-2f, 3.090169944e-1f, 5.358267950e-1f, 7.289686274e-1f, 8.763066800e-1f, 9.685831611e-1f};
    return c[m];
  } else {
    return 1.f;
  }
}
template <int R>
__host__ __device__ constexpr float wr_sin(int m) {
  if constexpr (R == 9) {
    constexpr float s[9] = {0.f, 6.427876097e-1f, 9.848077530e-1f, 8.660254038e-1f, 3.420201433e-1f, -3.420201433e-1f, -8.660254038e-1f, -9.848077530e-1f, -6.427876097e-1f};
    return s[m];
  } else if constexpr (R == 15) {
    constexpr float s[15] = {0.f, 4.067366431e-1f, 7.431448255e-1f, 9.510565163e-1f, 9.945218954e-1f, 8.660254038e-1f, 5.877852523e-1f, 2.079116908e-1f, -2.079116908e-1f, -5.877852523e-1f, -8.660254038e-1f, -9.945218954e-1f, -9.510565163e-1f, -7.431448255e-1f, -4.067366431e-1f};
    return s[m];
  } else if constexpr (R == 16) {
    constexpr float s[16] = {0.f, 3.826834324e-1f, 7.071067812e-1f, 9.238795325e-1f, 1.000000000f, 9.238795325e-1f, 7.071067812e-1f, 3.826834324e-1f, 0.f, -3.826834324e-1f, -7.071067812e-1f, -9.238795325e-1f, -1.000000000f, -9.238795325e-1f, -7.071067812e-1f, -3.826834324e-1f};
    return s[m];
  } else if constexpr (R == 25) {
    constexpr float s[25] = {0.f, 2.486898872e-1f, 4.817536741e-1f, 6.845471059e-1f, 8.443279255e-1f, 9.510565163e-1f, 9.980267284e-1f, 9.822872507e-1f, 9.048270525e-1f, 7.705132428e-1f, 5.877852523e-1f, 3.681245527e-1f, 1.253332336e-1f, -1.253332336e-1f, -3.681245527e-1f, -5.877852523e-1f, -7.705132428e-1f, -9.048270525e-1f, -9.822872507e-1f, -9.980267284e-1f, -9.510565163e-1f, -8.443279255e-1f, -6.845471059e-1f, -4.817536741e-1f, -2.486898872e-1f};
    return s[m];
  } else {
    return 0.f;
  }
}

// One Stockham stage of a composite radix R = R1 R2 (16 = 4 x 4, 25 = 5 x 5, 9 = 3 x 3, 15 = 3 x 5):
// the R-point DFT of each butterfly is split in registers (n = n1 + R1 n2, k = k2 + R2 k1):
//   X[k2 + R2 k1] = sum_n1 w_R1^(n1 k1) [ w_R^(n1 k2) sum_n2 v[n1 + R1 n2] w_R2^(n2 k2) ],
// which halves the shared-memory passes (and barriers) of a plan.  w_R^e = w_P^(e P/R).
// tws: this stage's twiddle rows (GTW: global memory).
template <int R1, int R2, bool GTW>
__device__ __forceinline__ void mr_stage2(const float2* src, float2* dst, int P, int Ns, const float2* tws, bool inv,
                                          int t) {
  constexpr int R = R1 * R2;
  const int nb = P / R;
  for (int j = t; j < nb; j += kMrT) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = DOE_IN(j + r * nb, P) ? src[j + r * nb] : make_float2(0.f, 0.f);
    const int k = j % Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = DOE_IN((Ns - 1) + (r - 1) * Ns + k, P) ? (GTW ? __ldg(tws + (r - 1) * Ns + k) : tws[(r - 1) * Ns + k]) : make_float2(0.f, 0.f);
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      float2 a[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) a[n2] = v[n1 + R1 * n2];
      mr_dft<R2>(a, inv);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        if (n1 && k2) {
          // w_R^(n1 k2): compile-time constants
          const float2 w = make_float2(wr_cos<R>((n1 * k2) % R), inv ? wr_sin<R>((n1 * k2) % R) : -wr_sin<R>((n1 * k2) % R));
          a[k2] = cmul(a[k2], w);
        }
        v[n1 + R1 * k2] = a[k2];
      }
    }
    const int base = (j - k) * R + k;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      float2 b[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) b[n1] = v[n1 + R1 * k2];
      mr_dft<R1>(b, inv);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1)
        if (DOE_IN(base + (k2 + R2 * k1) * Ns, P)) dst[base + (k2 + R2 * k1) * Ns] = b[k1];
    }
  }
  __syncthreads();
}

// One stage of a prime radix R > 5 (Table 2's large-area grid carries 67): one thread per
// output (butterfly j, output r), a direct R-point DFT fused with the stage twiddle:
//   dst[(j - k) R + k + r Ns] = sum_m src[j + m P/R] w_P^(m e),  e = k P/(Ns R) + r P/R
// (w_P^(m k P/(Ns R)) w_R^(m r) = w_P^(m e)); the exponents are kept reduced mod P.  With
// m = 8 q + u, w_P^(m e) = w_P^(8 q e) w_P^(u e): 8 + ceil(R / 8) table entries per output
// (17 at R = 67) and one complex product per term, instead of one table entry per term.
__device__ __forceinline__ void mr_stage_prime(const float2* src, float2* dst, int P, int Ns, int R,
                                               const float2* twg, bool inv, int t) {
  const int nb = P / R, step = P / (Ns * R);
  for (int o = t; o < P; o += kMrT) {
    const int j = o / R, r = o - j * R, k = j % Ns;
    const int e = k * step + r * nb;  // < P
    float2 lo[8];                     // w_P^(u e), u < 8
    int idx = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      lo[u] = DOE_IN(idx, P) ? __ldg(twg + idx) : make_float2(0.f, 0.f);
      idx += e;
      if (idx >= P) idx -= P;
    }
    const int e8 = idx;  // 8 e mod P
    float2 acc = make_float2(0.f, 0.f);
    int hidx = 0;        // 8 q e mod P
    for (int q = 0; 8 * q < R; ++q) {
      const float2 hi = DOE_IN(hidx, P) ? __ldg(twg + hidx) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int m = 8 * q + u;
        if (m < R) {
          float2 w = cmul(hi, lo[u]);
          if (inv) w.y = -w.y;
          const float2 v = DOE_IN(j + m * nb, P) ? src[j + m * nb] : make_float2(0.f, 0.f);
          acc.x = fmaf(v.x, w.x, fmaf(-v.y, w.y, acc.x));
          acc.y = fmaf(v.x, w.y, fmaf(v.y, w.x, acc.y));
        }
      }
      hidx += e8;
      if (hidx >= P) hidx -= P;
    }
    if (DOE_IN((j - k) * R + k + r * Ns, P)) dst[(j - k) * R + k + r * Ns] = acc;
  }
  __syncthreads();
}

// Unnormalised transform of the P samples at a (shared memory; b is a second buffer of P) with
// the batch's plan and its per-stage twiddles tws: the table in global memory, read through L1
// (GTW: the one-CTA passes), or its copy in shared memory (mr_smem_setup<true>: the split
// passes, whose L1 also serves the split's own twiddles).  The caller has made a's contents visible
// (barrier).  Returns the buffer holding the result (a or b).
// CMP: the plan has composite stages (9, 15, 16, 25); kernels are compiled both ways because
// those stages raise the register count (about 125 against 66), which costs occupancy to the
// short transforms that do not use them.
// ycol: the column (y) plan of a rectangular grid instead of the row plan.
template <bool CMP, bool GTW>
__device__ __forceinline__ float2* mr_fft(float2* a, float2* b, const Batch& bt, const float2* tws, bool inv, int t,
                                          bool ycol = false) {
  // the transform length: P (Py), or the chunk length M of a split transform
  const int P = ycol ? bt.mr_My : bt.mr_M;
  const int nst = ycol ? bt.mr_nst_y : bt.mr_nst;
  const float2* twg = ycol ? bt.mr_tw_y : bt.mr_tw;
  int Ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int R = ycol ? bt.mr_radix_y[s] : bt.mr_radix[s];
    const float2* ts = tws + (Ns - 1);  // this stage's rows
    if (CMP && R == 25) mr_stage2<5, 5, GTW>(a, b, P, Ns, ts, inv, t);
    else if (CMP && R == 16) mr_stage2<4, 4, GTW>(a, b, P, Ns, ts, inv, t);
    else if (CMP && R == 9) mr_stage2<3, 3, GTW>(a, b, P, Ns, ts, inv, t);
    else if (CMP && R == 15) mr_stage2<3, 5, GTW>(a, b, P, Ns, ts, inv, t);
    else if (R == 8) mr_stage<8, GTW>(a, b, P, Ns, ts, inv, t);
    else if (R == 5) mr_stage<5, GTW>(a, b, P, Ns, ts, inv, t);
    else if (R == 4) mr_stage<4, GTW>(a, b, P, Ns, ts, inv, t);
    else if (R == 3) mr_stage<3, GTW>(a, b, P, Ns, ts, inv, t);
    else if (R == 2) mr_stage<2, GTW>(a, b, P, Ns, ts, inv, t);
    else mr_stage_prime(a, b, P, Ns, R, twg, inv, t);
    Ns *= R;
    float2* c = a;
    a = b;
    b = c;
  }
  return a;
}

// Shared memory of a mixed-radix CTA: two transform buffers (2 M samples, M = bt.mr_M the
// length each CTA transforms, or the column length My), behind a copy of the per-stage twiddle
// table (M entries) if COPY.  Returns the first buffer; the caller's first barrier publishes
// the copy.
template <bool COPY>
__device__ __forceinline__ float2* mr_smem_setup(float2* sm, const Batch& bt, int t, bool ycol = false) {
  if constexpr (!COPY) {
    return sm;
  } else {
    const int M = ycol ? bt.mr_My : bt.mr_M;
    const float2* tws = ycol ? bt.mr_tws_y : bt.mr_tws;
    for (int m = t; m < M - 1; m += kMrT) sm[m] = __ldg(tws + m);
    return sm + M;
  }
}
// the twiddle table mr_fft reads: global (no copy) or the shared copy at sm
template <bool COPY>
__device__ __forceinline__ const float2* mr_tws_of(const float2* sm, const Batch& bt, bool ycol = false) {
  return COPY ? sm : (ycol ? bt.mr_tws_y : bt.mr_tws);
}

// E_doe of Eq. 2 at DOE sample (i, x): transmittance, parametric incident field, E_in array.
// N: the DOE's row length (its x side).
__device__ __forceinline__ float2 mr_doe_field(const Slice& sl, int i, int x, int N, IncRow ir) {
  const size_t o = (size_t)(i >> sl.uf) * (N >> sl.uf) + (x >> sl.uf);  // layout cell of DOE row i
  const float hv = DOE_IN(o, sl.n_h) ? __ldg(sl.h + o) : 0.f;
  float2 e = sl.illum ? transmittance_inc(hv, sl, ir, x - N / 2) : transmittance(hv, sl.kp_hi, sl.kp_lo);
  if (sl.e_in && DOE_IN((size_t)i * N + x, sl.n_ein)) e = cmul(e, __ldg(sl.e_in + (size_t)i * N + x));
  return e;
}

// Band-limited transfer function at column frequency index kc, row index lr (FFT order), from
// the slice's quarter table; conjugated for the adjoint.  H depends on kt^2 + lt^2 only, so
// the column's values are read along a table row (contiguous in lr).
__device__ __forceinline__ float2 mr_transfer(const Slice& sl, int kc, int lr, int Px, int Py, bool conj_h) {
  const int a = abs_signed(kc, Px), b = abs_signed(lr, Py);
  if (a > sl.kmax || b > sl.kmax_y) return make_float2(0.f, 0.f);
  if (!DOE_IN((size_t)a * sl.hp + b, sl.n_htab)) return make_float2(0.f, 0.f);
  float2 h = __ldg(sl.htab + (size_t)a * sl.hp + b);
  if (conj_h) h.y = -h.y;
  return h;
}

// Rectangular grids: rows run along x (Px = bt.P samples, the DOE's Nx = bt.N columns at offset
// bt.off), columns along y (Py = bt.Py samples, the DOE's Ny = bt.Ny rows at offset bt.offy); the
// buffers are row-major with rows of Px samples.  On square grids the two axes coincide.

// ---- pass A (mixed radix): DOE row i of slice blockIdx.y -> its row spectrum, tbuf row i.
template <bool CMP>
__global__ void __launch_bounds__(kMrT) mr_rows_fwd_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  const Slice& sl = bt.s[blockIdx.y];
  const int i = blockIdx.x, t = threadIdx.x, N = bt.N, P = bt.P, off = bt.off;
  float2* xa = mr_smem_setup<false>(sm_mr, bt, t);
  float2* xb = xa + P;
  const IncRow ir = incident_row(sl, i - bt.Ny / 2);
  for (int c = t; c < P; c += kMrT) {
    const int x = c - off;
    xa[c] = (unsigned)x < (unsigned)N ? mr_doe_field(sl, i, x, N, ir) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* y = mr_fft<CMP, true>(xa, xb, bt, mr_tws_of<false>(sm_mr, bt), false, t);
  float2* dst = sl.tbuf + (size_t)i * P;
  for (int c = t; c < P; c += kMrT)
    if (DOE_IN((size_t)i * P + c, sl.n_tbuf)) __stcs(dst + c, y[c]);
}

// ---- pass B / B* (mixed radix): one column kc per CTA.  Forward: the Ny row spectra (tbuf rows
// 0..Ny-1) placed at rows offy..offy+Ny-1, FFT, x H, IFFT, all Py rows to buf.  Adjoint
// (bt.mode == MODE_ADJ): all Py rows of tbuf, FFT, x conj(H), IFFT, rows offy..offy+Ny-1 back to
// tbuf rows 0..Ny-1 (in place: the CTA owns its column).  Neighbouring CTAs read the other
// samples of each 32-byte sector, which they find in L2.
template <bool CMP>
__global__ void __launch_bounds__(kMrT) mr_cols_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  const Slice& sl = bt.s[blockIdx.y];
  const int kc = blockIdx.x, t = threadIdx.x, Ny = bt.Ny, Px = bt.P, Py = bt.Py, offy = bt.offy;
  const bool adj = bt.mode == MODE_ADJ;
  float2* xa = mr_smem_setup<false>(sm_mr, bt, t, true);
  float2* xb = xa + Py;
  for (int l = t; l < Py; l += kMrT) {
    const int r = adj ? l : l - offy;
    xa[l] = (unsigned)r < (unsigned)(adj ? Py : Ny) && DOE_IN((size_t)r * Px + kc, sl.n_tbuf)
                ? __ldcs(sl.tbuf + (size_t)r * Px + kc) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* y = mr_fft<CMP, true>(xa, xb, bt, mr_tws_of<false>(sm_mr, bt, true), false, t, true);
  float2* z = y == xa ? xb : xa;
  const int kf = bt.mr_Q > 1 ? mrq_freq(kc, bt.mr_Q, bt.mr_M) : kc;  // rows split: stored in chunk order
  for (int l = t; l < Py; l += kMrT) y[l] = cmul(y[l], mr_transfer(sl, kf, l, Px, Py, adj));
  __syncthreads();
  y = mr_fft<CMP, true>(y, z, bt, mr_tws_of<false>(sm_mr, bt, true), true, t, true);
  if (!adj) {
    for (int l = t; l < Py; l += kMrT)
      if (DOE_IN((size_t)l * Px + kc, sl.n_buf)) __stcs(sl.buf + (size_t)l * Px + kc, y[l]);
  } else {
    for (int r = t; r < Ny; r += kMrT)
      if (DOE_IN((size_t)r * Px + kc, sl.n_tbuf)) __stcs(sl.tbuf + (size_t)r * Px + kc, y[r + offy]);
  }
}

// ---- pass B / B* (mixed radix) on clusters of 4 CTAs (Px a multiple of 4): the same
// transforms as mr_cols_kernel, one column per CTA, with the global accesses of the four
// adjacent columns kc0..kc0+3 done together as 32-byte row segments.  Each CTA loads a quarter
// of the rows (pairs of rows: two 16-byte loads per row) and pushes each column's pair of
// samples into that column's CTA (distributed shared memory, one 16-byte remote store), and
// after the inverse transform gathers a quarter of the output rows of all four columns from the
// cluster and stores them as 32-byte segments.  The column's transfer-function row arrives in
// shared memory by bulk copy while the input is exchanged and the forward transform runs.
// Shared memory: two buffers of Py samples, then the H row (hp entries).
template <bool CMP>
__global__ void __launch_bounds__(kMrT) mr_cols4_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ __align__(16) float2 sm_mr[];
  __shared__ __align__(8) uint64_t hbar;  // completion of the H-row copy
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const Slice& sl = bt.s[blockIdx.y];
  const int kc = blockIdx.x, kc0 = kc - q, t = threadIdx.x, Ny = bt.Ny, Px = bt.P, Py = bt.Py, offy = bt.offy;
  const bool adj = bt.mode == MODE_ADJ;
  float2* xa = sm_mr;
  float2* xb = xa + Py;
  float2* hs = xb + Py;
  const int ak = abs_signed(bt.mr_Q > 1 ? mrq_freq(kc, bt.mr_Q, bt.mr_M) : kc, Px);  // rows split: chunk order
  const bool hcopy = ak <= sl.kmax && sl.hp <= Py / 2 + 2 && DOE_IN((size_t)ak * sl.hp + sl.hp - 1, sl.n_htab);
  if (t == 0) {
    mbar_init(&hbar, 1);
    if (hcopy) {
      mbar_arrive_expect_tx(&hbar, (unsigned)sl.hp * sizeof(float2));
      bulk_g2s(hs, sl.htab + (size_t)ak * sl.hp, (unsigned)sl.hp * sizeof(float2), &hbar);
    }
  }
  cluster_sync_relaxed();  // every CTA of the cluster has started before its shared memory is written
  // input: sample l of the column transform is row l - offy of the Ny row spectra (forward) or
  // row l of the Py rows (adjoint); rows outside are zero.  This CTA covers the pairs
  // (l0, l0 + 1), l0 even, of its quarter and writes them into all four columns' buffers.
  const int np = Py / 2, pb = q * np / 4, pe = (q + 1) * np / 4;
  const int nin = adj ? Py : Ny, l_in = adj ? 0 : offy;
  for (int p = pb + t; p < pe; p += kMrT) {
    float4 lo[2], hi[2];  // rows l0, l0 + 1: columns (0, 1) in lo, (2, 3) in hi
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int r = 2 * p + u - l_in;
      lo[u] = hi[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((unsigned)r < (unsigned)nin && DOE_IN((size_t)r * Px + kc0 + 3, sl.n_tbuf)) {
        const float4* src = reinterpret_cast<const float4*>(sl.tbuf + (size_t)r * Px + kc0);
        lo[u] = __ldcs(src);
        hi[u] = __ldcs(src + 1);
      }
    }
    if (DOE_IN(p, Py / 2)) {
      reinterpret_cast<float4*>(cl.map_shared_rank(xa, 0))[p] = make_float4(lo[0].x, lo[0].y, lo[1].x, lo[1].y);
      reinterpret_cast<float4*>(cl.map_shared_rank(xa, 1))[p] = make_float4(lo[0].z, lo[0].w, lo[1].z, lo[1].w);
      reinterpret_cast<float4*>(cl.map_shared_rank(xa, 2))[p] = make_float4(hi[0].x, hi[0].y, hi[1].x, hi[1].y);
      reinterpret_cast<float4*>(cl.map_shared_rank(xa, 3))[p] = make_float4(hi[0].z, hi[0].w, hi[1].z, hi[1].w);
    }
  }
  cl.sync();  // every column's input is in place
  float2* y = mr_fft<CMP, true>(xa, xb, bt, mr_tws_of<false>(sm_mr, bt, true), false, t, true);
  float2* z = y == xa ? xb : xa;
  const bool hok = !hcopy || mbar_wait(&hbar, 0);
  if (!hok && t == 0) raise_fault(FAULT_WAIT_TIMEOUT);
  for (int l = t; l < Py; l += kMrT) {
    const int b = abs_signed(l, Py);
    float2 hv = make_float2(0.f, 0.f);
    if (hcopy && hok && b <= sl.kmax_y && DOE_IN(b, sl.hp)) hv = hs[b];
    if (adj) hv.y = -hv.y;
    y[l] = cmul(y[l], hv);
  }
  __syncthreads();
  y = mr_fft<CMP, true>(y, z, bt, mr_tws_of<false>(sm_mr, bt, true), true, t, true);
  cl.sync();  // every column's result is in its CTA's buffer y (the same offset in every CTA)
  // output: forward, all Py rows l to buf; adjoint, the DOE rows r = l - offy < Ny back to tbuf
  const int nout = adj ? Ny : Py, l_out = adj ? offy : 0;
  float2* dst0 = adj ? sl.tbuf : sl.buf;
  [[maybe_unused]] const long long ndst = adj ? sl.n_tbuf : sl.n_buf;
  const int op = nout / 2, ob = q * op / 4, oe = (q + 1) * op / 4;
  for (int p = ob + t; p < oe; p += kMrT) {
    float2 v[2][4];  // rows 2p, 2p + 1 (output numbering) of columns 0..3
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float2* ry = cl.map_shared_rank(y, c);
      const int l = 2 * p + l_out;
      if ((l_out & 1) == 0) {  // the pair is one 16-byte chunk of the peer's buffer
        const float4 w = DOE_IN(l + 1, Py) ? reinterpret_cast<const float4*>(ry)[l >> 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        v[0][c] = make_float2(w.x, w.y);
        v[1][c] = make_float2(w.z, w.w);
      } else {
        v[0][c] = DOE_IN(l, Py) ? ry[l] : make_float2(0.f, 0.f);
        v[1][c] = DOE_IN(l + 1, Py) ? ry[l + 1] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const size_t o = (size_t)(2 * p + u) * Px + kc0;
      if (DOE_IN(o + 3, ndst)) {
        float4* d = reinterpret_cast<float4*>(dst0 + o);
        __stcs(d, make_float4(v[u][0].x, v[u][0].y, v[u][1].x, v[u][1].y));
        __stcs(d + 1, make_float4(v[u][2].x, v[u][2].y, v[u][3].x, v[u][3].y));
      }
    }
  }
  cluster_sync_relaxed();  // the peers have read this CTA's buffer (their loads feed stores issued before)
}

// ---- pass C (mixed radix): output row y: IFFT, 1/(Px Py), then |E|^2 (OUT_PSF) or E.
template <bool CMP>
__global__ void __launch_bounds__(kMrT) mr_rows_out_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  const Slice& sl = bt.s[blockIdx.y];
  const int row = blockIdx.x, t = threadIdx.x, P = bt.P;
  float2* xa = mr_smem_setup<false>(sm_mr, bt, t);
  float2* xb = xa + P;
  const float2* src = sl.buf + (size_t)row * P;
  for (int c = t; c < P; c += kMrT) xa[c] = DOE_IN((size_t)row * P + c, sl.n_buf) ? __ldcs(src + c) : make_float2(0.f, 0.f);
  __syncthreads();
  const float2* y = mr_fft<CMP, true>(xa, xb, bt, mr_tws_of<false>(sm_mr, bt), true, t);
  const float s = bt.inv_p2;
  if (bt.mode == OUT_PSF) {
    float* dst = static_cast<float*>(sl.out) + (size_t)row * P;
    for (int c = t; c < P; c += kMrT) {
      const float2 e = cscale(y[c], s);
      if (DOE_IN((size_t)row * P + c, sl.n_out)) __stcs(dst + c, fmaf(e.x, e.x, e.y * e.y));
    }
  } else {
    float2* dst = static_cast<float2*>(sl.out) + (size_t)row * P;
    for (int c = t; c < P; c += kMrT)
      if (DOE_IN((size_t)row * P + c, sl.n_out)) __stcs(dst + c, cscale(y[c], s));
  }
}

// ---- pass C' (mixed radix): output row y: E = IFFT / (Px Py), g = 2 (I - T) E (L2, with the
// row's loss partial) or (dL/dI) E (VJP), forward FFT of g into tbuf row y.
template <bool CMP>
__global__ void __launch_bounds__(kMrT) mr_rows_adj_c_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  __shared__ double red[32];
  const Slice& sl = bt.s[blockIdx.y];
  const int row = blockIdx.x, t = threadIdx.x, P = bt.P;
  float2* xa = mr_smem_setup<false>(sm_mr, bt, t);
  float2* xb = xa + P;
  const float2* src = sl.buf + (size_t)row * P;
  for (int c = t; c < P; c += kMrT) xa[c] = DOE_IN((size_t)row * P + c, sl.n_buf) ? __ldcs(src + c) : make_float2(0.f, 0.f);
  __syncthreads();
  float2* y = mr_fft<CMP, true>(xa, xb, bt, mr_tws_of<false>(sm_mr, bt), true, t);
  const float s = bt.inv_p2;
  const float* trow = sl.tgt + (size_t)row * P;
  float acc = 0.f;
  for (int c = t; c < P; c += kMrT) {
    const float2 e = cscale(y[c], s);
    const float tt = DOE_IN((size_t)row * P + c, sl.n_tgt) ? __ldcs(trow + c) : 0.f;
    float w;
    if (bt.mode == GRAD_L2) {
      const float d = fmaf(e.x, e.x, e.y * e.y) - tt;
      acc = fmaf(d, d, acc);
      w = 2.f * d;
    } else {
      w = tt;
    }
    y[c] = cscale(e, w);
  }
  __syncthreads();
  y = mr_fft<CMP, true>(y, y == xa ? xb : xa, bt, mr_tws_of<false>(sm_mr, bt), false, t);
  float2* dst = sl.tbuf + (size_t)row * P;
  for (int c = t; c < P; c += kMrT)
    if (DOE_IN((size_t)row * P + c, sl.n_tbuf)) __stcs(dst + c, y[c]);
  const double tot = block_sum<kMrT>((double)acc, red);
  if (t == 0 && sl.loss_part && DOE_IN(row, sl.n_loss)) sl.loss_part[row] = tot;
}

// ---- pass A* (mixed radix): DOE row i, summed over the slices in order: g_doe = IFFT(tbuf
// row i) / (Px Py) on the DOE columns, dL/dh += -2 k' Im(conj(g_doe) E_doe).  Each thread owns
// its DOE columns, so the running sum lives in the gradient row itself.
template <bool CMP>
__global__ void __launch_bounds__(kMrT) mr_rows_adj_a_kernel(const __grid_constant__ Batch bt) {
  extern __shared__ float2 sm_mr[];
  const int i = blockIdx.x, t = threadIdx.x, N = bt.N, P = bt.P, off = bt.off;
  float2* xa = mr_smem_setup<false>(sm_mr, bt, t);
  float2* xb = xa + P;
  float* grow = bt.grad + (size_t)i * N;
  for (int j = 0; j < bt.S; ++j) {
    const Slice& sl = bt.s[j];
    const float2* src = sl.tbuf + (size_t)i * P;
    for (int c = t; c < P; c += kMrT) xa[c] = DOE_IN((size_t)i * P + c, sl.n_tbuf) ? __ldcs(src + c) : make_float2(0.f, 0.f);
    __syncthreads();
    const float2* y = mr_fft<CMP, true>(xa, xb, bt, mr_tws_of<false>(sm_mr, bt), true, t);
    const IncRow ir = incident_row(sl, i - bt.Ny / 2);
    const float k2 = -2.f * sl.kp_hi;
    for (int x = t; x < N; x += kMrT) {
      if (!DOE_IN((size_t)i * N + x, bt.n_grad)) continue;
      const float2 e = mr_doe_field(sl, i, x, N, ir);
      const float2 g = cscale(y[off + x], bt.inv_p2);
      const float prev = j ? grow[x] : 0.f;
      grow[x] = fmaf(k2, fmaf(g.x, e.y, -g.y * e.x), prev);
    }
    __syncthreads();  // xa / xb are reused by the next slice
  }
}

}  // namespace doe
