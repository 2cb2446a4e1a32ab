// doe_plan.h -- compile-time FFT plans and the launch parameter blocks, usable from host
// and device code.  Holds no device symbols.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace doe {


constexpr int kMinLog = 5;   // L = 32
constexpr int kMaxLog = 14;  // L = 16384 (one CTA)
constexpr int kBigLog = 16;  // longest transform: 65536 points, split across a cluster
constexpr int kBigTab = 512;  // cross-CTA (four-step) twiddle tables: W_65536^lo and W_65536^(256 hi)

__host__ __device__ constexpr int plan_r0(int lg) { return (lg % 4 == 0) ? 16 : (1 << (lg % 4)); }
// 8192 points use the three-stage plan 16 x 32 x 16 (two exchanges); other lengths radix-16
// stages plus one radix-2/4/8 stage.
__host__ __device__ constexpr int plan_nst(int lg) { return lg == 13 ? 3 : (lg + 3) / 4; }
__host__ __device__ constexpr int plan_radix(int lg, bool inv, int s) {
  if (lg == 13) return s == 1 ? 32 : 16;
  return inv ? (s == plan_nst(lg) - 1 ? plan_r0(lg) : 16) : (s == 0 ? plan_r0(lg) : 16);
}
__host__ __device__ constexpr int plan_ns(int lg, bool inv, int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= plan_radix(lg, inv, i);
  return p;
}
__host__ __device__ constexpr long tw_plan_size(int lg, bool inv) {
  long n = 0;
  for (int s = 0; s < plan_nst(lg); ++s) n += (long)plan_ns(lg, inv, s) * plan_radix(lg, inv, s);
  return n;
}
__host__ __device__ constexpr long tw_offset(int lg, bool inv, int s) {
  long off = 0;
  for (int l = kMinLog; l < lg; ++l) off += tw_plan_size(l, false) + tw_plan_size(l, true);
  if (inv) off += tw_plan_size(lg, false);
  for (int i = 0; i < s; ++i) off += (long)plan_ns(lg, inv, i) * plan_radix(lg, inv, i);
  return off;
}
constexpr long kTwTotal = tw_offset(kMaxLog + 1, false, 0);
// Forward and inverse plans of 8192 points are the same 16 x 32 x 16, so both directions read
// the forward table (the inverse applies the conjugate): one 68 KB table stays in L1.
__host__ __device__ constexpr bool tw_shared_dirs(int lg) { return lg == 13; }
// Stage table layout, float4 units: entry (k, r) for even r holds (W^{k r}, W^{k (r + 1)}),
// W = W_{Ns R}.  Stages with two butterflies per thread (R <= 16) hand lane t the butterflies
// k = 2 t' + p, so their table is ordered (r / 2, p, k / 2); one-butterfly stages (R = 32)
// hand lane t the butterfly k = t mod Ns, ordered (r / 2, k).  Either way the lanes of a warp
// read one contiguous 512-byte run per load.
__host__ __device__ constexpr long tw_quad(int R, int ns, int k, int r) {
  return R <= 16 ? ((long)(r >> 1) * 2 + (k & 1)) * (ns >> 1) + (k >> 1) : (long)(r >> 1) * ns + k;
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ constexpr int smem_words(int L) { return L; }

// Resident CTAs per SM requested from the register allocator for a row/column pass of length L
// (L / 32 threads): at most 128 registers per thread.  Registers are allocated per warp, so a
// CTA of fewer than 32 threads still takes a whole warp's share.
__host__ __device__ constexpr int min_blocks(int L) {
  return 65536 / (((L / 32) < 32 ? 32 : (L / 32)) * 128) > 1 ? 65536 / (((L / 32) < 32 ? 32 : (L / 32)) * 128) : 1;
}

// Elements per thread used for a transform of length L.
__host__ __device__ constexpr int elems_for(int) { return 32; }
template <int L, bool INV>
__host__ __device__ constexpr int first_radix() { return plan_radix(ilog2c(L), INV, 0); }
template <int L, bool INV>
__host__ __device__ constexpr int last_radix() { return plan_radix(ilog2c(L), INV, plan_nst(ilog2c(L)) - 1); }

constexpr int kMaxSlices = 64;  // wavelengths (over all requests) per launch
constexpr int kRenderColsMax = 8192;  // render column transform length limit (2 buffers of 64 KB)
constexpr int kTile = 4;    // tile width of the column-tiled buffer (4 x 8 B = one 32-byte sector); columns per cluster for P <= 8192
constexpr int kMaxQf = 16;  // sub-transforms per row at the longest split side (rectangles: 16 x 8192)
constexpr int kMrMax = 8192;        // longest mixed-radix (non-power-of-two) transform, one CTA
constexpr int kMrMaxStages = 16;    // radix stages of a mixed-radix plan
constexpr int kMrMaxPrime = 127;    // largest prime factor taken as a direct-DFT stage
constexpr int kMrT = 256;           // threads per CTA of every mixed-radix pass
constexpr int kMaxRadial = 9;       // coefficients of the radial height polynomial (degree 16 in rho / R)
constexpr int kRadialBlocks = 592;  // CTAs of the radial gradient reduction (4 per SM)

// One (request, wavelength) slice of a batched launch.  Everything a pass needs that is not
// shared by the whole launch.
struct Slice {
  const float* h;        // [N >> uf][N >> uf] heights (m): the layout at pitch 2^uf dx
  const float2* e_in;    // [N][N] incident field or nullptr
  float2* buf;           // [P][wp] natural-layout field buffer: I2 (rows < P), J2 (rows < N)
  float2* tbuf;          // column-tiled buffer read by the column pass: I1 (N rows), J1 (P rows)
  float2* htab;          // [kmax + 1][hp] transfer function quarter table H(|kt|, |lt|)
  const float* tgt;      // [P][P] target T or dL/dI (gradient)
  void* out;             // [P][P] float PSF or float2 field
  double* loss_part;     // [Py] per-row loss partial sums (gradient)
  float kp_hi, kp_lo;    // k' = 2 pi (n - 1) / lambda as a float pair
  float c_hi, c_lo;      // q = lambda^2 (fx^2 + fy^2) = c m: c = (lambda du)^2, (lambda g / (Px Py dx))^2 on rectangles
  float phi0_hi, phi0_lo;  // 2 pi z / lambda
  float th0_hi, th0_lo;    // (2 pi z / lambda) mod 2 pi
  long long mev;         // propagating iff m = kt^2 sqb + lt^2 sqa < mev
  long long sqa, sqb;    // (Px / g)^2, (Py / g)^2 with g = gcd(Px, Py): 1, 1 on square grids
  int kmax;              // band limit index of the row (x) frequencies kt
  int kmax_y;            // band limit index of the column (y) frequencies lt (= kmax on square grids)
  int seg_a;             // length of the stored non-negative-frequency segment (even)
  int w;                 // stored columns: P if the band limit is inactive, else seg_a + even(kmax)
  int wp;                // row pitch of buf (w rounded up to kTile)
  int hp;                // row pitch of htab: kmax + 1 rounded up to even, or hq << hqs
  int hqs;               // split grids: row entries grouped by residue mod 2^hqs (0: natural order)
  int hq;                // split grids: entries per residue class of a row (even)
  int tile_begin;        // first global column-tile index of this slice (column pass)
  int uf;                // log2 of the nearest-upsampling factor of the heights (0: none)
  int illum;             // parametric incident field: ILLUM_TILT | ILLUM_SPHERE (0: none)
  float ta_hi, ta_lo;    // tilt: cycles per sample along x, dx sin(theta_x) / lambda
  float tb_hi, tb_lo;    // tilt: cycles per sample along y, dx sin(theta_y) / lambda
  float sc_hi, sc_lo;    // spherical wave: (dx / d)^2
  float sk_hi, sk_lo;    // spherical wave: |d| / lambda
  float ssgn;            // spherical wave: +1 diverging (d > 0), -1 converging
  // extents of the slice's buffers in elements (float2, or float for h / tgt / out as a PSF),
  // for the bounds checks of the DOE_DEBUG build
  long long n_buf, n_tbuf, n_htab, n_h, n_ein, n_tgt, n_out, n_loss;
};
enum : int { ILLUM_TILT = 1, ILLUM_SPHERE = 2 };

// Lanczos-3 interpolation of a height layout onto the simulation grid (upsampling factor f):
// simulation sample x = f xc + r reads layout cells xc + off[r] + d, d = 0..5, with weights
// w[r][d] (normalised to sum 1; cells clamped to the layout).
struct LanczosTab {
  int f, nl;          // factor, layout side
  int off[8];         // first tap relative to xc, per residue r
  float w[8][6];      // tap weights per residue r
};

enum : int { OUT_PSF = 0, OUT_FIELD = 1 };
enum : int { MODE_FWD = 0, MODE_ADJ = 1 };
enum : int { GRAD_L2 = 0, GRAD_VJP = 1 };

struct Batch {
  int S;             // slices
  int N, P, off;     // DOE side, padded side, DOE offset in the padded grid (rows: the x axis)
  int Ny, Py, offy;  // the same along the columns (y axis); equal to N, P, off on square grids
  int total_tiles;   // column tiles over all slices
  int mode;          // MODE_FWD / MODE_ADJ (column pass), OUT_* (row inverse pass), GRAD_* (adjoint row pass)
  int max_kmax;      // largest kmax over the slices (table builder grid)
  int qf;            // sub-transforms per row: P / 16384 for P > 16384, else 1
  int illum;         // some slice has a parametric incident field (selects the DOE-row kernels)
  int mr;            // P is not a power of two: the mixed-radix passes run
  int mr_Q, mr_M;    // P = Q M: Q CTAs (a cluster) per row / column, each transforming M points (Q = 1: M = P)
  int mr_cmp;        // the plan has composite stages (9, 15, 16, 25): selects the kernel build
  int mr_nst;        // mixed-radix plan of M: stages and their radices (2..8, 9, 15, 16, 25, primes)
  int mr_radix[kMrMaxStages];
  const float2* mr_tw;   // [M] twiddles exp(-2 pi i m / M) in the workspace
  int mr_My;             // rectangular grids: the column transform's length, plan and twiddles
  int mr_nst_y;          // (equal to the row's on square grids)
  int mr_radix_y[kMrMaxStages];
  const float2* mr_tw_y;
  const float2* mr_twP;  // [P] twiddles exp(-2 pi i m / P) of the split (Q > 1)
  int mr_Qy;               // the column transform's split (Py = mr_Qy mr_My; equal to mr_Q on square grids)
  const float2* mr_twP_y;  // [Py] twiddles of the column split (rectangular grids, mr_Qy > 1)
  // per-stage twiddles of the plan, lane-contiguous: stage s (sub-transform size Ns, radix R)
  // holds w_(Ns R)^(r k) at (Ns - 1) + (r - 1) Ns + k for 1 <= r < R, k < Ns (M - 1 entries in all)
  const float2* mr_tws;
  const float2* mr_tws_y;  // of the column transform of a rectangular grid
  float inv_p2;      // 1 / P^2 (inverse transform normalisation)
  float* grad;       // [N][N] gradient on the simulation grid (DOE-row adjoint pass)
  long long n_grad;  // its extent (bounds checks of the DOE_DEBUG build)
  Slice s[kMaxSlices];
};

}  // namespace doe
