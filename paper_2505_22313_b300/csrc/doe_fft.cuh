// doe_fft.cuh -- in-CTA Stockham FFT engine for sm_103a.
//
// One CTA transforms one vector of L = 2^LOG complex64 samples (32 <= L <= 16384).  Each of
// the T = L / 32 threads keeps E = 32 samples in registers; a stage applies E / R radix-R
// butterflies per thread, always as pairs of adjacent butterflies (j, j + 1), so that every
// shared-memory and global access moves two samples (16 bytes) at once.  Consecutive stages
// exchange data through shared memory, addressed in 16-byte chunks with an XOR swizzle
// (chunk c lives at c ^ ((c >> 4) & 7)) that keeps the strided patterns conflict-free without
// padding, so an 8192-point vector takes exactly 64 KB.  The formulation is the self-sorting
// Stockham autosort: stage s with radix R and current sub-transform size Ns reads element
//     j + r * (L / R)                        (j = butterfly index, r < R)
// multiplies element r by W_{Ns R}^{r (j mod Ns)}, takes an R-point DFT and writes it to
//     (j - j mod Ns) * R + (j mod Ns) + r * Ns,
// which leaves the result in natural order after the last stage.  Thread t owns butterflies
// j = t + b * T, b < E / R, so the first stage's reads and the last stage's writes
// (both "j + r * L/R") are contiguous across a warp and go straight to/from global memory.
//
// Radix plans: forward = [r0, 16, 16, ...], inverse = [16, ..., 16, r0] (r0 = L / 16^k <= 16).
// The forward plan ends and the inverse plan starts with radix 16, and the inverse plan ends
// with the forward plan's first radix, so a forward -> pointwise -> inverse chain (the
// transfer-function multiply) and an inverse -> pointwise -> forward chain (the adjoint row
// pass) need no shared-memory round trip in between: the registers already hold the next
// transform's first-stage inputs.
//
// Twiddles come from per-(L, direction, stage) tables in device memory, rows of R entries
// W_{Ns R}^{r k} for k < Ns (entry 0 = 1), computed on the host in FP64 and rounded to FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "doe_plan.h"

namespace doe {

// 16-byte chunk swizzle of the exchange buffer, and the float2 slot of element e.
__device__ __forceinline__ int swz(int c) { return c ^ ((c >> 4) & 7); }
__device__ __forceinline__ int phys(int e) { return (swz(e >> 1) << 1) | (e & 1); }

// Tables live in static device memory, filled once per device at library set-up.  Every
// translation unit that includes this header holds its own copy (internal linkage, so the
// kernel TUs compile separately without device linking) and registers an uploader for it;
// the set-up fills every registered copy.
static __device__ __align__(16) float2 g_tw[kTwTotal];
// W_65536^n = W_65536^(256 hi) W_65536^lo for n = 256 hi + lo: entries [0, 256) hold
// W_65536^lo, entries [256, 512) W_65536^(256 hi) (4 KB, L1-resident)
static __device__ __align__(16) float2 g_tw_big[kBigTab];

using TableUpload = cudaError_t (*)(const float2* stage_tw, size_t n_stage, const float2* big_tw, size_t n_big);
int register_table_upload(TableUpload fn);  // defined once, in doe_launch.cu
static cudaError_t upload_tables_of_this_unit(const float2* stage_tw, size_t n_stage, const float2* big_tw,
                                              size_t n_big) {
  cudaError_t e = cudaMemcpyToSymbol(g_tw, stage_tw, n_stage * sizeof(float2));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_tw_big, big_tw, n_big * sizeof(float2));
}
[[maybe_unused]] static const int g_tables_registered = register_table_upload(upload_tables_of_this_unit);

// Fault word of this translation unit's kernels (bits DOE_FAULT_*): a bounded wait that ran
// out, or (in the bounds-checked build) an index outside its buffer.  Kernels set bits and
// carry on without the faulting access; doe_fault_status() reads and clears every unit's word.
static __device__ unsigned int g_fault_word;
using FaultRead = cudaError_t (*)(unsigned int* word);
int register_fault_reader(FaultRead fn);  // defined once, in doe_launch.cu
static cudaError_t read_fault_of_this_unit(unsigned int* word) {
  const unsigned int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(word, g_fault_word, sizeof(unsigned int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_fault_word, &zero, sizeof(unsigned int));
}
[[maybe_unused]] static const int g_fault_registered = register_fault_reader(read_fault_of_this_unit);
enum : unsigned int { FAULT_WAIT_TIMEOUT = 1u, FAULT_BOUNDS = 2u };
__device__ __forceinline__ void raise_fault(unsigned int bits) { atomicOr(&g_fault_word, bits); }

// Bounds checks of the DOE_DEBUG build: DOE_IN(i, n) is true when 0 <= i < n; otherwise it sets
// FAULT_BOUNDS and is false, and the access it guards is skipped (a load then yields zero).  In
// the release build it is the constant true and the checks compile away.
#ifdef DOE_DEBUG
__device__ __forceinline__ bool doe_in(long long i, long long n) {
  if (i >= 0 && i < n) return true;
  raise_fault(FAULT_BOUNDS);
  return false;
}
#define DOE_IN(i, n) ::doe::doe_in((long long)(i), (long long)(n))
#else
#define DOE_IN(i, n) true
#endif

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
template <bool INV>
__device__ __forceinline__ float2 ctw(float2 a, float2 w) { return INV ? cmulc(a, w) : cmul(a, w); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 cmi(float2 a) { return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ------------------------------------------------------------------ small DFTs in registers
// Forward kernels use W_R = exp(-2 pi i / R); INV uses the conjugates.  In and out in place,
// natural order.
template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = cmi<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}
constexpr float kR2 = 0.70710678118654752440f;  // 1/sqrt(2)
constexpr float kC8 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kS8 = 0.38268343236508977173f;  // sin(pi/8)

template <bool INV>
__device__ __forceinline__ float2 w8(float2 a, int q) {  // a * W_8^q, q in 1..3
  const float sg = INV ? 1.f : -1.f;
  if (q == 1) return make_float2(kR2 * (a.x - sg * a.y), kR2 * (a.y + sg * a.x));
  if (q == 2) return cmi<INV>(a);
  return make_float2(kR2 * (-a.x - sg * a.y), kR2 * (-a.y + sg * a.x));
}
template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  dft4<INV>(v[0], v[2], v[4], v[6]);
  dft4<INV>(v[1], v[3], v[5], v[7]);
  v[3] = w8<INV>(v[3], 1);
  v[5] = w8<INV>(v[5], 2);
  v[7] = w8<INV>(v[7], 3);
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}
// a * W_16^m for the m that occur in the 4 x 4 split: 1, 2, 3, 4, 6, 9
template <bool INV>
__device__ __forceinline__ float2 w16(float2 a, int m) {
  const float sg = INV ? 1.f : -1.f;  // W_16^m = cos(2 pi m/16) + sg i sin(2 pi m/16)
  float c, s;
  switch (m) {
    case 1: c = kC8; s = kS8; break;
    case 2: c = kR2; s = kR2; break;
    case 3: c = kS8; s = kC8; break;
    case 4: return cmi<INV>(a);
    case 6: c = -kR2; s = kR2; break;
    default: c = -kC8; s = -kS8; break;  // m = 9
  }
  s *= sg;
  return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  // n = 4 n1 + n2, q = q1 + 4 q2
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // now v[4 q1 + n2] = A_{n2}[q1]; twiddle by W_16^{n2 q1}
  v[5] = w16<INV>(v[5], 1);
  v[6] = w16<INV>(v[6], 2);
  v[7] = w16<INV>(v[7], 3);
  v[9] = w16<INV>(v[9], 2);
  v[10] = w16<INV>(v[10], 4);
  v[11] = w16<INV>(v[11], 6);
  v[13] = w16<INV>(v[13], 3);
  v[14] = w16<INV>(v[14], 6);
  v[15] = w16<INV>(v[15], 9);
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1) dft4<INV>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
  // v[4 q1 + q2] = y[q1 + 4 q2]: transpose the 4 x 4 index
  float2 t;
  t = v[1]; v[1] = v[4]; v[4] = t;
  t = v[2]; v[2] = v[8]; v[8] = t;
  t = v[3]; v[3] = v[12]; v[12] = t;
  t = v[6]; v[6] = v[9]; v[9] = t;
  t = v[7]; v[7] = v[13]; v[13] = t;
  t = v[11]; v[11] = v[14]; v[14] = t;
}
// cos and sin of 2 pi k / 32, k < 16
__host__ __device__ constexpr float w32c(int k) {
  constexpr float c[16] = {1.00000000000000000000f, 0.98078528040323043058f, 0.92387953251128673848f,
                             0.83146961230254523567f, 0.70710678118654757274f, 0.55557023301960228867f,
                             0.38268343236508983729f, 0.19509032201612833135f, 0.f, -0.19509032201612819257f,
                             -0.38268343236508972627f, -0.55557023301960195560f, -0.70710678118654746172f,
                             -0.83146961230254534669f, -0.92387953251128673848f, -0.98078528040323043058f};
  return c[k];
}
__host__ __device__ constexpr float w32s(int k) {
  constexpr float c[16] = {0.f, 0.19509032201612824808f, 0.38268343236508978178f, 0.55557023301960217765f,
                             0.70710678118654746172f, 0.83146961230254523567f, 0.92387953251128673848f,
                             0.98078528040323043058f, 1.f, 0.98078528040323043058f, 0.92387953251128673848f,
                             0.83146961230254545772f, 0.70710678118654757274f, 0.55557023301960217765f,
                             0.38268343236508989280f, 0.19509032201612860891f};
  return c[k];
}
// 32-point DFT: two 16-point DFTs of the even and odd samples, then one radix-2 step with
// W_32^k (decimation in time).
template <bool INV>
__device__ __forceinline__ void dft32(float2* v) {
  float2 e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float c = w32c(k), s = INV ? w32s(k) : -w32s(k);  // W_32^k = c + i s
    const float2 t = k == 0 ? o[k] : (k == 8 ? cmi<INV>(o[k]) : make_float2(fmaf(o[k].x, c, -o[k].y * s), fmaf(o[k].x, s, o[k].y * c)));
    v[k] = cadd(e[k], t);
    v[k + 16] = csub(e[k], t);
  }
}
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else dft32<INV>(v);
}

// ------------------------------------------------------------------ stages
template <int L, int E, bool INV, int S>
struct St {
  static constexpr int LOG = ilog2c(L);
  static constexpr int T = L / E;
  static constexpr int NST = plan_nst(LOG);
  static constexpr int R = plan_radix(LOG, INV, S);
  static constexpr int NS = plan_ns(LOG, INV, S);
  static constexpr int B = E / R;  // butterflies per thread: even (adjacent pairs) or 1
  static constexpr bool PAIRED = B >= 2;
  static_assert(L >= 32 && L <= (1 << kMaxLog) && (L & (L - 1)) == 0, "L must be a power of two in [32, 16384]");
  static_assert(E == 32 && (B % 2 == 0 || B == 1), "butterflies are processed in adjacent pairs, or one per thread");
  // butterfly index of register group b (b even: first of a pair)
  __device__ static __forceinline__ int j(int t, int b) { return PAIRED ? 2 * (t + (b >> 1) * T) + (b & 1) : t; }
  // transform index of register b*R + r in this stage's input layout (and, for the last
  // stage, in its output layout)
  __device__ static __forceinline__ int idx(int t, int b, int r) { return j(t, b) + r * (L / R); }
};

// Twiddle + DFT of stage S on registers (inputs already in place).
template <int L, int E, bool INV, int S>
__device__ __forceinline__ void stage_compute(float2 (&v)[E], int t) {
  using X = St<L, E, INV, S>;
  constexpr int R = X::R;
#pragma unroll
  for (int b = 0; b < X::B; ++b) {
    if constexpr (S > 0) {
      const int k = X::j(t, b) & (X::NS - 1);
      const float4* tw = reinterpret_cast<const float4*>(g_tw + tw_offset(X::LOG, INV && !tw_shared_dirs(X::LOG), S));
#pragma unroll
      for (int r = 0; r < R; r += 2) {
        const long q = tw_quad(R, X::NS, k, r);
        const float4 w = DOE_IN(2 * (tw_offset(X::LOG, INV && !tw_shared_dirs(X::LOG), S) + 2 * q) + 3, 2 * kTwTotal)
                             ? __ldg(tw + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (r > 0) v[b * R + r] = ctw<INV>(v[b * R + r], make_float2(w.x, w.y));
        v[b * R + r + 1] = ctw<INV>(v[b * R + r + 1], make_float2(w.z, w.w));
      }
    }
    dft<R, INV>(&v[b * R]);
  }
}

// Write stage S's outputs to shared memory in Stockham order, 16 bytes per access.
template <int L, int E, bool INV, int S>
__device__ __forceinline__ void stage_store(const float2 (&v)[E], int t, float2* sm) {
  using X = St<L, E, INV, S>;
  constexpr int R = X::R, NS = X::NS;
  float4* s4 = reinterpret_cast<float4*>(sm);
  if constexpr (!X::PAIRED && NS == 16) {
    // one butterfly per thread (the radix-32 stage of 8192 points): outputs base + 16 r, chunk
    // c0 + 8 r with c0 = base / 2 and c0 mod 16 < 8, so the swizzle term ((c0 + 8 r) >> 4) & 7
    // = ((c0 >> 4) + (r >> 1)) & 7 is shared by r = 2q, 2q + 1 and only touches the low 3 bits
    const int jj = X::j(t, 0);
    const int k = jj & (NS - 1);
    const int base = (jj - k) * R + k;
    const int c0 = base >> 1, odd = base & 1;
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
      const int ch = (c0 & ~7) + 16 * q + ((c0 & 7) ^ (((c0 >> 4) + q) & 7));
      if (DOE_IN((ch << 1) | odd, L)) sm[(ch << 1) | odd] = v[2 * q];
      if (DOE_IN(((ch + 8) << 1) | odd, L)) sm[((ch + 8) << 1) | odd] = v[2 * q + 1];
    }
  } else if constexpr (!X::PAIRED && NS > 1) {
    // one butterfly per thread: its outputs base + r Ns are not adjacent, 8-byte accesses
    const int jj = X::j(t, 0);
    const int k = jj & (NS - 1);
    const int base = (jj - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (DOE_IN(phys(base + r * NS), L)) sm[phys(base + r * NS)] = v[r];
  } else if constexpr (NS == 1) {
    // butterfly j's outputs are the contiguous elements j R + r: chunks c0 + d, d < R / 2, all
    // inside one 16-chunk row of the swizzle (c0 = j R / 2), so the swizzle term is fixed
#pragma unroll
    for (int b = 0; b < X::B; ++b) {
      const int c0 = X::j(t, b) * (R / 2), x = (c0 >> 4) & 7;
#pragma unroll
      for (int r = 0; r < R; r += 2)
        if (DOE_IN((c0 + r / 2) ^ x, L / 2))
          s4[(c0 + r / 2) ^ x] = make_float4(v[b * R + r].x, v[b * R + r].y, v[b * R + r + 1].x, v[b * R + r + 1].y);
    }
  } else {
    // the pair (j, j + 1) writes adjacent elements base + r Ns, base + 1 + r Ns: chunks c0 + C r,
    // C = Ns / 2.  Closed forms of swz(c0 + C r): C a multiple of 128 leaves the swizzle term
    // unchanged; C = 16 a adds a r to it; C = 8 (c0 mod 16 < 8 here) adds r >> 1.
    constexpr int C = NS / 2;
#pragma unroll
    for (int b = 0; b < X::B; b += 2) {
      const int jj = X::j(t, b);
      const int k = jj & (NS - 1);
      const int c0 = ((jj - k) * R + k) >> 1, x0 = c0 >> 4, q0 = swz(c0);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int ch;
        if constexpr (C % 128 == 0) ch = q0 + C * r;
        else if constexpr (C % 16 == 0) ch = (c0 ^ ((x0 + (C / 16) * r) & 7)) + C * r;
        else if constexpr (C == 8) ch = (c0 & ~7) + 8 * r + ((c0 & 7) ^ ((x0 + (r >> 1)) & 7));
        else ch = swz(c0 + C * r);
        if (DOE_IN(ch, L / 2))
          s4[ch] = make_float4(v[b * R + r].x, v[b * R + r].y, v[(b + 1) * R + r].x, v[(b + 1) * R + r].y);
      }
    }
  }
}

// Read stage S's inputs ("j + r L/R") from shared memory, 16 bytes per access.
template <int L, int E, bool INV, int S>
__device__ __forceinline__ void stage_load(float2 (&v)[E], int t, const float2* sm) {
  using X = St<L, E, INV, S>;
  constexpr int R = X::R;
  const float4* s4 = reinterpret_cast<const float4*>(sm);
  // with a stride of a multiple of 128 chunks the swizzle term is the same for every r, so
  // the addresses are the first one plus constants
  constexpr bool kFlat = (L / R / 2) % 128 == 0;
  if constexpr (!X::PAIRED) {
    const int p0 = phys(X::j(t, 0));
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = kFlat ? p0 + r * (L / R) : phys(X::j(t, 0) + r * (L / R));
      v[r] = DOE_IN(e, L) ? sm[e] : make_float2(0.f, 0.f);
    }
  } else {
#pragma unroll
    for (int b = 0; b < X::B; b += 2) {
      const int c0 = X::j(t, b) >> 1, q0 = swz(c0);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int ch = kFlat ? q0 + r * (L / R / 2) : swz(c0 + r * (L / R / 2));
        const float4 q = DOE_IN(ch, L / 2) ? s4[ch] : make_float4(0.f, 0.f, 0.f, 0.f);
        v[b * R + r] = make_float2(q.x, q.y);
        v[(b + 1) * R + r] = make_float2(q.z, q.w);
      }
    }
  }
}

// Runs stages S..NST-1: on entry v holds stage S's inputs; on exit v holds the final outputs
// in the last stage's layout (element St<...,NST-1>::idx(t, b, r) of the transform).  Stages
// exchange through sm, each exchange preceded by a barrier, so sm may still be read by other
// threads on entry.
template <int L, int E, bool INV, int S = 0>
__device__ __forceinline__ void fft_run(float2 (&v)[E], int t, float2* sm) {
  stage_compute<L, E, INV, S>(v, t);
  if constexpr (S + 1 < St<L, E, INV, S>::NST) {
    __syncthreads();
    stage_store<L, E, INV, S>(v, t, sm);
    __syncthreads();
    stage_load<L, E, INV, S + 1>(v, t, sm);
    fft_run<L, E, INV, S + 1>(v, t, sm);
  }
}

// fft_run with a callback at the last stage: at_last() runs after the last stage's inputs are
// loaded from shared memory and before its butterflies (which need no shared memory), so a
// callback that starts with a barrier finds the exchange buffer free for other uses.
template <int L, int E, bool INV, int S = 0, class F>
__device__ __forceinline__ void fft_run_last(float2 (&v)[E], int t, float2* sm, F&& at_last) {
  if constexpr (S + 1 < St<L, E, INV, S>::NST) {
    stage_compute<L, E, INV, S>(v, t);
    __syncthreads();
    stage_store<L, E, INV, S>(v, t, sm);
    __syncthreads();
    stage_load<L, E, INV, S + 1>(v, t, sm);
    fft_run_last<L, E, INV, S + 1>(v, t, sm, at_last);
  } else {
    at_last();
    stage_compute<L, E, INV, S>(v, t);
  }
}

// Layout helpers for the kernels: the first stage's input layout and the last stage's output
// layout.  Register b*R + r holds transform element idx(t, b, r); registers (b, r) and
// (b + 1, r) for even b hold the adjacent elements e, e + 1.
template <int L, bool INV>
using First = St<L, 32, INV, 0>;
template <int L, bool INV>
using Last = St<L, 32, INV, plan_nst(ilog2c(L)) - 1>;

}  // namespace doe
