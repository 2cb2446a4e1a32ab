// doe_api.cu -- host side of libdoe: argument validation, per-device set-up, workspace
// layout and launch sequencing of the passes (see doe_kernels.cuh).  Everything is
// enqueued on the caller's stream; nothing here synchronises the device.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "doe.h"
#include "doe_launch.h"

using namespace doe;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
bool g_dev_ready[kMaxDevices] = {};

// Forward twiddles exp(-2 pi i m / n) in FP64, rounded to FP32.
float2 twiddle(long m, long n) {
  const double a = -2.0 * kPi * (double)(m % n) / (double)n;
  return make_float2((float)std::cos(a), (float)std::sin(a));
}

const std::vector<float2>& host_stage_tables() {
  static std::vector<float2> tw;
  if (tw.empty()) {
    tw.assign((size_t)kTwTotal, make_float2(0.f, 0.f));
    for (int lg = kMinLog; lg <= kMaxLog; ++lg)
      for (int inv = 0; inv < 2; ++inv)
        for (int s = 0; s < plan_nst(lg); ++s) {
          const long ns = plan_ns(lg, inv, s), R = plan_radix(lg, inv, s);
          float2* p = tw.data() + tw_offset(lg, inv, s);
          for (long k = 0; k < ns; ++k)
            for (long r = 0; r < R; ++r) p[2 * tw_quad((int)R, (int)ns, (int)k, (int)r) + (r & 1)] = twiddle(r * k, ns * R);
        }
  }
  return tw;
}

const std::vector<float2>& host_big_table() {
  static std::vector<float2> tw;
  if (tw.empty()) {
    tw.resize(kBigTab);  // W_65536^lo, then W_65536^(256 hi), lo, hi < 256
    for (long n = 0; n < 256; ++n) {
      tw[n] = twiddle(n, 1L << kBigLog);
      tw[256 + n] = twiddle(256 * n, 1L << kBigLog);
    }
  }
  return tw;
}

int ensure_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DOE_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_dev_ready[dev]) return DOE_OK;
  const auto& a = host_stage_tables();
  const auto& b = host_big_table();
  if (upload_tables(a.data(), a.size(), b.data(), b.size()) != cudaSuccess) return DOE_ECUDA;
  if (prepare_kernels() != cudaSuccess) return DOE_ECUDA;
  g_dev_ready[dev] = true;
  return DOE_OK;
}

bool is_pow2(long n) { return n > 0 && (n & (n - 1)) == 0; }

// Radices of the mixed-radix plan of a length 2 <= M <= kMrMax: its prime factors above 5 (up to
// kMrMaxPrime, one direct-DFT stage each), then the 5s and 3s in pairs (25, 9; a lone 5 and 3 as
// 15), then the power of two as 16s, with 8, 4 or 2 for the rest; empty for any other M.  Below
// 2048 points a composite stage has too few butterflies for a CTA's threads (1125 / 25 = 45), so
// short transforms keep the single radices (5, 3, then 8s and 4s).
std::vector<int> mr_radices(long M) {
  std::vector<int> r;
  if (M < 2 || M > kMrMax) return r;
  long n = M;
  for (int p = 7; p <= kMrMaxPrime; p += 2) {
    bool prime = true;
    for (int d = 3; d * d <= p; d += 2)
      if (p % d == 0) prime = false;
    while (prime && n % p == 0) {
      r.push_back(p);
      n /= p;
    }
  }
  int c5 = 0, c3 = 0, a = 0;
  for (; n % 5 == 0; n /= 5) ++c5;
  for (; n % 3 == 0; n /= 3) ++c3;
  for (; n % 2 == 0; n /= 2) ++a;
  if (n != 1) return {};
  // the plan with n25 stages of 25, n9 of 9, n15 of 15, n16 of 16, then 5s, 3s and the powers
  // of two as 8s (4 4 for a remainder of 4, a single 2 only for a remainder of 1)
  auto plan = [&](int n25, int n9, int n15, int n16) {
    std::vector<int> p = r;
    p.insert(p.end(), n25, 25);
    p.insert(p.end(), n9, 9);
    p.insert(p.end(), n15, 15);
    p.insert(p.end(), n16, 16);
    p.insert(p.end(), c5 - 2 * n25 - n15, 5);
    p.insert(p.end(), c3 - 2 * n9 - n15, 3);
    for (int b = a - 4 * n16; b > 0;) {
      const int e = (b == 4 || b == 2) ? 2 : (b >= 3 ? 3 : 1);
      p.push_back(1 << e);
      b -= e;
    }
    return p;
  };
  if (M < 2048) {  // short transforms: no composite stages (their kernels keep the occupancy)
    r = plan(0, 0, 0, 0);
    return (int)r.size() > kMrMaxStages ? std::vector<int>{} : r;
  }
  // composite stages (25 = 5 x 5, 9 = 3 x 3, 15 = 3 x 5, 16 = 4 x 4, split in registers) save
  // shared-memory passes, but a stage of radix R has M / R butterflies for kMrT threads: take the
  // plan of least estimated time, each stage costing its rounds ceil(M / R / kMrT) of R-point
  // butterflies (about R (3 + log2 R) operations: loads, twiddles, DFT, stores) plus a barrier
  auto cost = [&](const std::vector<int>& p) {
    double c = 0.0;
    for (int R : p) c += (double)((M / R + kMrT - 1) / kMrT) * R * (3.0 + std::log2((double)R)) + 30.0;
    return c;
  };
  std::vector<int> best;
  double bc = 1e300;
  for (int n25 = 0; 2 * n25 <= c5; ++n25)
    for (int n9 = 0; 2 * n9 <= c3; ++n9)
      for (int n15 = 0; n15 <= c5 - 2 * n25 && n15 <= c3 - 2 * n9; ++n15)
        for (int n16 = 0; 4 * n16 <= a; ++n16) {
          const std::vector<int> p = plan(n25, n9, n15, n16);
          if ((int)p.size() > kMrMaxStages) continue;
          const double c = cost(p);
          if (c < bc - 1e-9 || (c < bc + 1e-9 && p.size() < best.size())) {
            bc = c;
            best = p;
          }
        }
  return best;
}

// Split of a non-power-of-two side P into Q CTAs of M = P / Q points: Q = 1 up to kMrMax
// (P even), else the first of Q = 8, 5, 4, 3, 2 that divides P with a supported M <= kMrMax.
// {0, 0} when P is unsupported.
struct MrSplit {
  int Q, M;
};
MrSplit mr_split(long P) {
  if (P < 2 || (P & 1) || is_pow2(P) || P > (1L << kBigLog)) return {0, 0};
  if (P <= kMrMax) return mr_radices(P).empty() ? MrSplit{0, 0} : MrSplit{1, (int)P};
  for (int q : {8, 5, 4, 3, 2})
    if (P % q == 0 && P / q <= kMrMax && !mr_radices(P / q).empty()) return {q, (int)(P / q)};
  return {0, 0};
}

int ilog2(long n) { int l = 0; while ((1L << l) < n) ++l; return l; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
void split(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// Integer band logic (see doe.h): the same FP64 expressions the specification states.
long band_kmax(double lam, double dx, long P, double z, bool bandlimit) {
  if (!bandlimit) return P / 2;
  const double du = 1.0 / ((double)P * dx);
  const double t = 2.0 * du * z;
  const double flim = 1.0 / (lam * std::sqrt(t * t + 1.0));
  long k = (long)std::ceil(flim / du) - 1;
  if (k > P / 2) k = P / 2;
  if (k < 0) k = 0;
  return k;
}
// The bound of kt^2 + lt^2 the transfer function applies: the evanescent cut, and with the
// circular band limit also the disc m < ceil((f_lim / du)^2).
long long band_mev(double lam, double dx, long P);
long long band_mlim(const doe_geom* g, double lam, long P) {
  const long long mev = band_mev(lam, g->dx, P);
  if (!(g->flags & DOE_BANDLIMIT) || !(g->flags & DOE_BANDLIMIT_CIRCULAR)) return mev;
  const double du = 1.0 / ((double)P * g->dx);
  const double t = 2.0 * du * g->z;
  const double flim = 1.0 / (lam * std::sqrt(t * t + 1.0));
  const double r = flim / du;
  const double x = r * r;
  const long long mc = x > 9.0e18 ? LLONG_MAX : (long long)std::ceil(x);
  return mc < mev ? mc : mev;
}
long long band_mev(double lam, double dx, long P) {
  const double du = 1.0 / ((double)P * dx);
  const double ld = lam * du;
  const double x = 1.0 / (ld * ld);
  if (x > 9.0e18) return LLONG_MAX;
  return (long long)std::ceil(x);
}

// Columns per column-pass tile: 4, except for rows split into Q = P / 8192 sub-transforms,
// where a cluster of 2 Q CTAs holds 2 columns.
int col_tile(long P) { return (P == 65536 || P == 32768) ? 2 : kTile; }

int upsample_log2(const doe_geom* g) { return (int)((g->flags >> DOE_UPSAMPLE_SHIFT) & 3u); }
// Lanczos-3 interpolation of the layout (a pre-pass) instead of nearest (fused into pass A)
bool lanczos(const doe_geom* g) { return (g->flags & DOE_UPSAMPLE_LANCZOS3) && upsample_log2(g) > 0; }

// Tap table of the Lanczos-3 interpolation by f = 2^u (FP64 on the host): sample x = f xc + r
// sits at layout coordinate u = xc + (r + 1/2) / f - 1/2; its taps are the cells
// floor(u) - 2 .. floor(u) + 3 with weights K(u - n), K(t) = sinc(t) sinc(t / 3), normalised.
LanczosTab lanczos_table(int N, int u) {
  LanczosTab tb;
  std::memset(&tb, 0, sizeof(tb));
  tb.f = 1 << u;
  tb.nl = N >> u;
  auto sinc = [](double x) { return x == 0.0 ? 1.0 : std::sin(kPi * x) / (kPi * x); };
  for (int r = 0; r < tb.f; ++r) {
    const double fr = (r + 0.5) / tb.f - 0.5;  // u - xc
    const int n0 = (int)std::floor(fr) - 2;
    double w[6], sum = 0.0;
    for (int d = 0; d < 6; ++d) {
      const double tt = fr - (n0 + d);
      w[d] = std::fabs(tt) < 3.0 ? sinc(tt) * sinc(tt / 3.0) : 0.0;
      sum += w[d];
    }
    tb.off[r] = n0;
    for (int d = 0; d < 6; ++d) tb.w[r][d] = (float)(w[d] / sum);
  }
  return tb;
}

bool rect(const doe_geom* g) { return g->nx != g->ny; }

// Split of one side of a rectangular grid: one CTA per transform up to kMrMax (any length with a
// plan, powers of two included), else the first of Q = 8, 5, 4, 3, 2, 16 that divides it into
// sub-transforms of at most kMrMax points with a plan (16: sides up to 131072, such as Table 2's
// 128640 = 16 x 8040 and 85760 = 16 x 5360).  {0, 0} when the side is unsupported.
MrSplit axis_split(long P) {
  if (P < 2 || (P & 1)) return {0, 0};
  if (P <= kMrMax) return mr_radices(P).empty() ? MrSplit{0, 0} : MrSplit{1, (int)P};
  for (int q : {8, 5, 4, 3, 2, 16})
    if (P % q == 0 && P / q <= kMrMax && !mr_radices(P / q).empty()) return {q, (int)(P / q)};
  return {0, 0};
}

// Rectangular grids (nx != ny) run on the mixed-radix passes with a row plan and a column plan:
// each side one CTA per transform up to kMrMax (powers of two included), or split over a
// cluster (axis_split) above.
bool rect_supported(const doe_geom* g) {
  const long px = (long)g->pad * g->nx, py = (long)g->pad * g->ny;
  return axis_split(px).Q > 0 && axis_split(py).Q > 0 && upsample_log2(g) == 0 &&
         !(g->flags & DOE_BANDLIMIT_CIRCULAR) && g->theta_x == 0.0 && g->theta_y == 0.0 && g->src_d == 0.0;
}

int check_geom(const doe_geom* g) {
  if (!g) return DOE_EINVAL;
  if (g->nx < 16 || g->ny < 16 || (g->nx & 1) || (g->ny & 1)) return DOE_EINVAL;
  if (g->pad != 1 && g->pad != 2) return DOE_EINVAL;
  if ((long)g->pad * g->nx < (1L << kMinLog) || (long)g->pad * g->ny < (1L << kMinLog)) return DOE_EUNSUPPORTED;
  if (!(g->dx > 0.0) || !(g->z > 0.0) || !std::isfinite(g->dx) || !std::isfinite(g->z)) return DOE_EINVAL;
  if (g->n_lambda < 1 || g->n_lambda > kMaxSlices || !g->lambda || !g->n_index) return DOE_EINVAL;
  for (int j = 0; j < g->n_lambda; ++j) {
    if (!(g->lambda[j] > 0.0) || !std::isfinite(g->lambda[j])) return DOE_EINVAL;
    if (!(g->n_index[j] >= 1.0) || !std::isfinite(g->n_index[j])) return DOE_EINVAL;
  }
  if (rect(g) && !rect_supported(g)) return DOE_EUNSUPPORTED;
  if (!rect(g) && (long)g->pad * g->nx > (1L << kBigLog)) return DOE_EUNSUPPORTED;  // rectangles: axis_split
  if (!rect(g) && !is_pow2((long)g->pad * g->nx) && mr_split((long)g->pad * g->nx).Q == 0) return DOE_EUNSUPPORTED;
  const int u = upsample_log2(g);
  if ((g->nx >> u) < 4 || (g->ny >> u) < 4 || (g->nx & ((1 << u) - 1)) || (g->ny & ((1 << u) - 1))) return DOE_EINVAL;
  if (!(std::fabs(g->theta_x) < 0.5 * kPi) || !(std::fabs(g->theta_y) < 0.5 * kPi) || !std::isfinite(g->src_d))
    return DOE_EINVAL;
  return DOE_OK;
}

// Rectangular evanescent rule: with g = gcd(Px, Py), A = Px / g, B = Py / g a sample (kt, lt)
// propagates iff kt^2 B^2 + lt^2 A^2 < ceil((Px Py dx / (g lambda))^2) (the same FP64
// expression the oracle writes out).
long gcdl(long a, long b) { return b ? gcdl(b, a % b) : a; }
long long rect_mev(long Px, long Py, double dx, double lam) {
  const long gg = gcdl(Px, Py);
  const double x = (double)Px * (double)Py * dx / ((double)gg * lam);
  const double x2 = x * x;
  return x2 > 9.0e18 ? LLONG_MAX : (long long)std::ceil(x2);
}

// Fills the per-slice constants of wavelength j of g.
void fill_slice(Slice& s, const doe_geom* g, int j) {
  const long P = (long)g->pad * g->nx;
  const long Py = (long)g->pad * g->ny;
  const double lam = g->lambda[j];
  const double du = 1.0 / ((double)P * g->dx);
  const long kmax = band_kmax(lam, g->dx, P, g->z, (g->flags & DOE_BANDLIMIT) != 0);
  std::memset(&s, 0, sizeof(s));
  s.uf = lanczos(g) ? 0 : upsample_log2(g);  // Lanczos: the passes read pre-interpolated heights
  s.kmax = (int)kmax;
  s.kmax_y = (int)kmax;
  s.sqa = s.sqb = 1;
  if (kmax >= P / 2 || P > (1L << kMaxLog) || !is_pow2(P) || rect(g)) {  // no compaction (split rows: sub-transform order; mixed radix: natural)
    s.seg_a = (int)P;
    s.w = (int)P;
  } else {
    s.seg_a = (int)((kmax + 2) & ~1L);  // kmax + 1 rounded up to even
    s.w = s.seg_a + (int)((kmax + 1) & ~1L);  // + kmax rounded up to even
  }
  s.wp = (s.w + kTile - 1) / kTile * kTile;
  s.hp = (int)((kmax + 2) & ~1L);  // kmax + 1 rounded up to even
  if (is_pow2(P) && P > (1L << kMaxLog) && !rect(g)) {  // split grids: rows grouped by residue mod Q = P / 8192
    s.hqs = ilog2(P / 8192);
    s.hq = (int)(((kmax >> s.hqs) + 2) & ~1L);  // (kmax >> hqs) + 1 rounded up to even: 16-byte class runs
    s.hp = s.hq << s.hqs;
  }
  s.mev = band_mlim(g, lam, P);
  const double ld = lam * du;
  split(ld * ld, s.c_hi, s.c_lo);
  if (rect(g)) {  // per-axis band limits; q = c (kt^2 B^2 + lt^2 A^2)
    const long gg = gcdl(P, Py);
    s.kmax_y = (int)band_kmax(lam, g->dx, Py, g->z, (g->flags & DOE_BANDLIMIT) != 0);
    s.hp = (int)((s.kmax_y + 2) & ~1L);
    s.sqa = (long long)(P / gg) * (P / gg);
    s.sqb = (long long)(Py / gg) * (Py / gg);
    s.mev = rect_mev(P, Py, g->dx, lam);
    const double cq = lam * (double)gg / ((double)P * (double)Py * g->dx);
    split(cq * cq, s.c_hi, s.c_lo);
  }
  const double phi0 = 2.0 * kPi * g->z / lam;
  split(phi0, s.phi0_hi, s.phi0_lo);
  split(std::fmod(phi0, 2.0 * kPi), s.th0_hi, s.th0_lo);
  split(2.0 * kPi * (g->n_index[j] - 1.0) / lam, s.kp_hi, s.kp_lo);
  // parametric incident field: tilt in cycles per sample, spherical wave as (dx/d)^2 and |d|/lambda
  if (g->theta_x != 0.0 || g->theta_y != 0.0) {
    s.illum |= ILLUM_TILT;
    split(g->dx * std::sin(g->theta_x) / lam, s.ta_hi, s.ta_lo);
    split(g->dx * std::sin(g->theta_y) / lam, s.tb_hi, s.tb_lo);
  }
  if (g->src_d != 0.0) {
    s.illum |= ILLUM_SPHERE;
    const double q = g->dx / g->src_d;
    split(q * q, s.sc_hi, s.sc_lo);
    split(std::fabs(g->src_d) / lam, s.sk_hi, s.sk_lo);
    s.ssgn = g->src_d > 0.0 ? 1.f : -1.f;
  }
}

struct Layout {
  size_t total = 0;
  std::vector<size_t> buf, htab, tbuf;
  size_t loss = 0;
  size_t gsim = 0;  // gradient on the simulation grid before the upsampling adjoint
  std::vector<size_t> hsim;  // per request, Lanczos-3: heights interpolated onto the simulation grid
  size_t ltmp = 0;           // Lanczos-3: the [N / f][N] buffer of the separable passes
  size_t mrtw = 0;           // mixed radix: the [M] twiddle table of the per-CTA transform
  size_t mrtwP = 0;          // mixed radix split over a cluster: the [P] twiddle table
  size_t mrtw_y = 0;         // rectangular grids: the [Py] twiddle table of the column transform
  size_t mrtws = 0, mrtws_y = 0;  // per-stage (lane-contiguous) twiddles of the row / column plans
  size_t mrtwP_y = 0;        // rectangular grids with a split column transform: the [Py] table
  long tbuf_rows = 0;        // rows of the column-tiled buffers (Ny forward, Py with the adjoint)
};

// Sides of a request's grid: the DOE (Nx x Ny) and its padded grid (Px x Py).
struct Grid {
  long Nx, Ny, Px, Py;
};
Grid grid_of(const doe_geom* g) {
  return {g->nx, g->ny, (long)g->pad * g->nx, (long)g->pad * g->ny};
}

// Workspace: per slice a natural-layout [P][wp] complex field buffer, then per slice a transfer
// table, then per slice a column-tiled buffer (N rows for the forward path, P rows when the
// adjoint also runs), then (gradient) the per-row loss partials.  The field buffers and tables
// sit at the same offsets in the PSF and gradient layouts, so a gradient-sized workspace used
// by doe_psf keeps the fields and tables doe_grad(recompute=0) needs.
Layout make_layout(const std::vector<Slice>& sl, int op, int n_req, const doe_geom* geoms) {
  const Grid gr = grid_of(&geoms[0]);
  const long P = gr.Px, N = gr.Nx, Py = gr.Py, Ny = gr.Ny;
  Layout L;
  size_t off = 0;
  for (const auto& s : sl) {
    L.buf.push_back(off);
    off = align256(off + (size_t)Py * s.wp * sizeof(float2));
  }
  for (const auto& s : sl) {
    L.htab.push_back(off);
    off = align256(off + (size_t)(s.kmax + 1) * s.hp * sizeof(float2));
  }
  const long R = op == DOE_OP_GRAD ? Py : Ny;
  L.tbuf_rows = R;
  for (const auto& s : sl) {
    L.tbuf.push_back(off);
    off = align256(off + (size_t)R * s.wp * sizeof(float2));
  }
  if (op == DOE_OP_GRAD) {
    L.loss = off;
    off = align256(off + sl.size() * (size_t)(P > Py ? P : Py) * kMaxQf * sizeof(double));
    if (upsample_log2(&geoms[0]) > 0) {
      L.gsim = off;
      off = align256(off + (size_t)N * N * sizeof(float));
    }
  }
  if (Py != P) {  // rectangular grid: twiddle tables of the row and of the column transform
    const MrSplit sx = axis_split(P), sy = axis_split(Py);
    L.mrtw = off;
    off = align256(off + (size_t)sx.M * sizeof(float2));
    L.mrtw_y = off;
    off = align256(off + (size_t)sy.M * sizeof(float2));
    L.mrtws = off;
    off = align256(off + (size_t)sx.M * sizeof(float2));
    L.mrtws_y = off;
    off = align256(off + (size_t)sy.M * sizeof(float2));
    if (sx.Q > 1) {
      L.mrtwP = off;
      off = align256(off + (size_t)P * sizeof(float2));
    }
    if (sy.Q > 1) {
      L.mrtwP_y = off;
      off = align256(off + (size_t)Py * sizeof(float2));
    }
  } else if (!is_pow2(P)) {
    const MrSplit sp = mr_split(P);
    L.mrtw = off;
    off = align256(off + (size_t)sp.M * sizeof(float2));
    L.mrtws = off;
    off = align256(off + (size_t)sp.M * sizeof(float2));
    if (sp.Q > 1) {
      L.mrtwP = off;
      off = align256(off + (size_t)P * sizeof(float2));
    }
  }
  long nl_max = 0;  // Lanczos-3: [N / f][N] buffer of the separable interpolation (and its adjoint)
  for (int r = 0; r < n_req; ++r)
    if (lanczos(&geoms[r]) && (N >> upsample_log2(&geoms[r])) > nl_max) nl_max = N >> upsample_log2(&geoms[r]);
  if (nl_max) {
    L.ltmp = off;
    off = align256(off + (size_t)N * nl_max * sizeof(float));
  }
  L.hsim.assign(n_req, 0);
  for (int r = 0; r < n_req; ++r)
    if (lanczos(&geoms[r])) {
      L.hsim[r] = off;
      off = align256(off + (size_t)N * N * sizeof(float));
    }
  L.total = off;
  return L;
}

int collect_slices(int n_req, const doe_geom* geoms, std::vector<Slice>& sl, std::vector<int>& req_of) {
  if (n_req < 1 || !geoms) return DOE_EINVAL;
  for (int r = 0; r < n_req; ++r) {
    const int rc = check_geom(&geoms[r]);
    if (rc != DOE_OK) return rc;
    if (geoms[r].nx != geoms[0].nx || geoms[r].ny != geoms[0].ny || geoms[r].pad != geoms[0].pad) return DOE_EINVAL;
  }
  for (int r = 0; r < n_req; ++r)
    for (int j = 0; j < geoms[r].n_lambda; ++j) {
      Slice s;
      fill_slice(s, &geoms[r], j);
      sl.push_back(s);
      req_of.push_back(r);
    }
  if ((int)sl.size() > kMaxSlices) return DOE_EUNSUPPORTED;
  return DOE_OK;
}

// The mixed-radix plan of a transform of length M into (nst, radix[]); true if it has composite
// stages (9, 15, 16, 25).
bool set_plan(long M, int& nst, int* radix) {
  const std::vector<int> pl = mr_radices(M);
  bool cmp = false;
  nst = (int)pl.size();
  for (size_t s = 0; s < pl.size(); ++s) {
    radix[s] = pl[s];
    if (pl[s] == 9 || pl[s] == 15 || pl[s] == 16 || pl[s] == 25) cmp = true;
  }
  return cmp;
}

void init_batch(Batch& bt, const std::vector<Slice>& sl, const doe_geom* g0, void* ws, const Layout& lay) {
  const Grid gr = grid_of(g0);
  std::memset(&bt, 0, sizeof(bt));
  bt.S = (int)sl.size();
  bt.N = (int)gr.Nx;
  bt.P = (int)gr.Px;
  bt.off = (bt.P - bt.N) / 2;
  bt.Ny = (int)gr.Ny;
  bt.Py = (int)gr.Py;
  bt.offy = (bt.Py - bt.Ny) / 2;
  bt.inv_p2 = (float)(1.0 / ((double)bt.P * (double)bt.Py));
  bt.qf = bt.P > (1 << kMaxLog) ? bt.P / 8192 : 1;
  const long Pl = bt.P > bt.Py ? bt.P : bt.Py;
  int tiles = 0, kmx = 0;
  for (int j = 0; j < bt.S; ++j) {
    bt.s[j] = sl[j];
    bt.s[j].buf = reinterpret_cast<float2*>(static_cast<char*>(ws) + lay.buf[j]);
    bt.s[j].htab = reinterpret_cast<float2*>(static_cast<char*>(ws) + lay.htab[j]);
    bt.s[j].tbuf = reinterpret_cast<float2*>(static_cast<char*>(ws) + lay.tbuf[j]);
    if (lay.loss) bt.s[j].loss_part = reinterpret_cast<double*>(static_cast<char*>(ws) + lay.loss) + (size_t)j * Pl * kMaxQf;
    bt.s[j].n_buf = (long long)bt.Py * sl[j].wp;
    bt.s[j].n_tbuf = (long long)lay.tbuf_rows * sl[j].wp;
    bt.s[j].n_htab = (long long)(sl[j].kmax + 1) * sl[j].hp;
    if (lay.loss) bt.s[j].n_loss = (long long)Pl * kMaxQf;
    bt.s[j].tile_begin = tiles;
    tiles += sl[j].wp / col_tile(bt.P);
    if (sl[j].kmax > kmx) kmx = sl[j].kmax;
    if (sl[j].illum) bt.illum = 1;
  }
  bt.total_tiles = tiles;
  bt.max_kmax = kmx;
  if (bt.Py != bt.P) {  // rectangular grid: one-CTA mixed-radix passes with a row and a column plan
    const MrSplit sx = axis_split(bt.P), sy = axis_split(bt.Py);
    bt.mr = 1;
    bt.mr_Q = sx.Q;
    bt.mr_M = sx.M;
    bt.mr_Qy = sy.Q;
    bt.mr_My = sy.M;
    bt.qf = sx.Q;  // split rows write one loss partial per CTA
    const bool cx = set_plan(sx.M, bt.mr_nst, bt.mr_radix), cy = set_plan(sy.M, bt.mr_nst_y, bt.mr_radix_y);
    bt.mr_cmp = (cx || cy) ? 1 : 0;
    bt.mr_tw = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtw);
    bt.mr_tw_y = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtw_y);
    bt.mr_tws = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtws);
    bt.mr_tws_y = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtws_y);
    if (sx.Q > 1) bt.mr_twP = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtwP);
    if (sy.Q > 1) bt.mr_twP_y = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtwP_y);
  } else if (!is_pow2(bt.P)) {
    const MrSplit sp = mr_split(bt.P);
    bt.mr = 1;
    bt.mr_Q = sp.Q;
    bt.mr_M = sp.M;
    bt.qf = sp.Q;  // split rows write one loss partial per CTA
    bt.mr_cmp = set_plan(sp.M, bt.mr_nst, bt.mr_radix) ? 1 : 0;
    bt.mr_tw = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtw);
    bt.mr_tws = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtws);
    if (sp.Q > 1) bt.mr_twP = reinterpret_cast<const float2*>(static_cast<char*>(ws) + lay.mrtwP);
    // square grid: the column transform is the row transform
    bt.mr_My = bt.mr_M;
    bt.mr_nst_y = bt.mr_nst;
    for (int s = 0; s < bt.mr_nst; ++s) bt.mr_radix_y[s] = bt.mr_radix[s];
    bt.mr_tw_y = bt.mr_tw;
    bt.mr_tws_y = bt.mr_tws;
    bt.mr_Qy = bt.mr_Q;
    bt.mr_twP_y = bt.mr_twP;
  }
}

int ws_ok(void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return DOE_OK;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u)) return DOE_ENOWS;
  return DOE_OK;
}

int forward_passes(Batch& bt, cudaStream_t st) {
  const int lg = ilog2(bt.P);
  if (bt.mr && launch_mr_twiddles(bt, st) != cudaSuccess) return DOE_ECUDA;
  if (launch_htab(bt, st) != cudaSuccess) return DOE_ECUDA;
  if (launch_pass_a(lg, bt, st) != cudaSuccess) return DOE_ECUDA;
  bt.mode = MODE_FWD;
  if (launch_pass_b(lg, bt, st) != cudaSuccess) return DOE_ECUDA;
  return DOE_OK;
}

int run_forward(int n_req, const doe_geom* geoms, const float* const* h, const float* const* e_in,
                void* const* out, int out_kind, void* ws, size_t ws_bytes, void* stream) {
  std::vector<Slice> sl;
  std::vector<int> req_of;
  int rc = collect_slices(n_req, geoms, sl, req_of);
  if (rc != DOE_OK) return rc;
  for (int r = 0; r < n_req; ++r)
    if (!h[r] || !out[r]) return DOE_EINVAL;
  const Grid gr = grid_of(&geoms[0]);
  const int N = geoms[0].nx;
  const long P = gr.Px;
  const Layout lay = make_layout(sl, DOE_OP_PSF, n_req, geoms);
  if ((rc = ws_ok(ws, ws_bytes, lay.total)) != DOE_OK) return rc;
  if ((rc = ensure_device()) != DOE_OK) return rc;
  static thread_local Batch bt;
  init_batch(bt, sl, &geoms[0], ws, lay);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Lanczos-3 requests: interpolate their layouts onto the simulation grid first
  std::vector<const float*> hr(h, h + n_req);
  for (int r = 0; r < n_req; ++r)
    if (lanczos(&geoms[r])) {
      float* hs = reinterpret_cast<float*>(static_cast<char*>(ws) + lay.hsim[r]);
      float* tmp = reinterpret_cast<float*>(static_cast<char*>(ws) + lay.ltmp);
      if (launch_lanczos_up(h[r], tmp, hs, N, lanczos_table(N, upsample_log2(&geoms[r])), st) != cudaSuccess)
        return DOE_ECUDA;
      hr[r] = hs;
    }
  int jr = 0, prev = -1;
  for (int j = 0; j < bt.S; ++j) {
    const int r = req_of[j];
    jr = (r == prev) ? jr + 1 : 0;
    prev = r;
    bt.s[j].h = hr[r];
    bt.s[j].e_in = e_in ? reinterpret_cast<const float2*>(e_in[r]) : nullptr;
    const size_t esz = out_kind == OUT_PSF ? sizeof(float) : sizeof(float2);
    bt.s[j].out = static_cast<char*>(out[r]) + (size_t)jr * gr.Py * gr.Px * esz;
    const int u = lanczos(&geoms[r]) ? 0 : upsample_log2(&geoms[r]);
    bt.s[j].n_h = (long long)(gr.Ny >> u) * (gr.Nx >> u);
    bt.s[j].n_ein = e_in && e_in[r] ? (long long)gr.Ny * gr.Nx : 0;
    bt.s[j].n_out = (long long)gr.Py * gr.Px;
  }
  if ((rc = forward_passes(bt, st)) != DOE_OK) return rc;
  bt.mode = out_kind;
  if (launch_pass_c(ilog2(P), bt, st) != cudaSuccess) return DOE_ECUDA;
  return DOE_OK;
}

}  // namespace

int render_ensure_device() { return ensure_device(); }

extern "C" {

int doe_init(void) { return ensure_device(); }

size_t doe_workspace_bytes_many(int n_req, const doe_geom* geoms, int op) {
  if (op != DOE_OP_PROPAGATE && op != DOE_OP_PSF && op != DOE_OP_GRAD) return 0;
  std::vector<Slice> sl;
  std::vector<int> req_of;
  if (collect_slices(n_req, geoms, sl, req_of) != DOE_OK) return 0;
  return make_layout(sl, op, n_req, geoms).total;
}

size_t doe_workspace_bytes(const doe_geom* g, int op) { return doe_workspace_bytes_many(1, g, op); }

int doe_propagate(const doe_geom* g, const float* h, const float* e_in, float* e_out, void* ws,
                  size_t ws_bytes, void* stream) {
  void* o = e_out;
  return run_forward(1, g, &h, &e_in, &o, OUT_FIELD, ws, ws_bytes, stream);
}

int doe_psf(const doe_geom* g, const float* h, const float* e_in, float* psf, void* ws, size_t ws_bytes,
            void* stream) {
  void* o = psf;
  return run_forward(1, g, &h, &e_in, &o, OUT_PSF, ws, ws_bytes, stream);
}

int doe_psf_many(int n_req, const doe_geom* geoms, const float* const* h, const float* const* e_in,
                 float* const* psf, void* ws, size_t ws_bytes, void* stream) {
  if (n_req < 1 || !h || !psf) return DOE_EINVAL;
  std::vector<void*> o(psf, psf + n_req);
  return run_forward(n_req, geoms, h, e_in, o.data(), OUT_PSF, ws, ws_bytes, stream);
}

int doe_grad(const doe_geom* g, const float* h, const float* e_in, const float* t_or_dldi, int mode,
             float* grad_h, double* loss_dev, int recompute, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g);
  if (rc != DOE_OK) return rc;
  if (!h || !t_or_dldi || !grad_h) return DOE_EINVAL;
  if (mode != DOE_GRAD_L2_TARGET && mode != DOE_GRAD_VJP) return DOE_EINVAL;
  if (recompute != 0 && recompute != 1) return DOE_EINVAL;
  std::vector<Slice> sl;
  std::vector<int> req_of;
  if ((rc = collect_slices(1, g, sl, req_of)) != DOE_OK) return rc;
  const Grid gr = grid_of(g);
  const int N = g->nx;
  const long P = gr.Px;
  const Layout lay = make_layout(sl, DOE_OP_GRAD, 1, g);
  if ((rc = ws_ok(ws, ws_bytes, lay.total)) != DOE_OK) return rc;
  if ((rc = ensure_device()) != DOE_OK) return rc;
  static thread_local Batch bt;
  init_batch(bt, sl, g, ws, lay);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool lz = lanczos(g);
  const float* hsim = lz ? reinterpret_cast<const float*>(static_cast<char*>(ws) + lay.hsim[0]) : nullptr;
  // the adjoint row pass reads the heights too, so the interpolation runs with stored fields as well
  if (lz && launch_lanczos_up(h, reinterpret_cast<float*>(static_cast<char*>(ws) + lay.ltmp), const_cast<float*>(hsim),
                             N, lanczos_table(N, upsample_log2(g)), st) != cudaSuccess)
    return DOE_ECUDA;
  const int uf = upsample_log2(g);
  for (int j = 0; j < bt.S; ++j) {
    bt.s[j].h = lz ? hsim : h;
    bt.s[j].e_in = reinterpret_cast<const float2*>(e_in);
    bt.s[j].tgt = t_or_dldi + (size_t)j * gr.Py * gr.Px;
    const int u = lz ? 0 : uf;
    bt.s[j].n_h = (long long)(gr.Ny >> u) * (gr.Nx >> u);
    bt.s[j].n_ein = e_in ? (long long)gr.Ny * gr.Nx : 0;
    bt.s[j].n_tgt = (long long)gr.Py * gr.Px;
  }
  bt.grad = uf ? reinterpret_cast<float*>(static_cast<char*>(ws) + lay.gsim) : grad_h;
  bt.n_grad = (long long)gr.Ny * gr.Nx;
  const int lg = ilog2(P);
  if (recompute && (rc = forward_passes(bt, st)) != DOE_OK) return rc;
  if (!recompute && bt.mr && launch_mr_twiddles(bt, st) != cudaSuccess) return DOE_ECUDA;
  bt.mode = mode == DOE_GRAD_L2_TARGET ? GRAD_L2 : GRAD_VJP;
  if (launch_pass_c_adj(lg, bt, st) != cudaSuccess) return DOE_ECUDA;
  const int gmode = bt.mode;
  bt.mode = MODE_ADJ;
  if (launch_pass_b(lg, bt, st) != cudaSuccess) return DOE_ECUDA;
  if (launch_pass_a_adj(lg, bt, st) != cudaSuccess) return DOE_ECUDA;
  if (lz) {
    float* tmp = reinterpret_cast<float*>(static_cast<char*>(ws) + lay.ltmp);
    if (launch_lanczos_adjoint(bt.grad, tmp, grad_h, N, lanczos_table(N, uf), st) != cudaSuccess) return DOE_ECUDA;
  } else if (uf && launch_upsample_adjoint(bt.grad, grad_h, N, uf, st) != cudaSuccess) {
    return DOE_ECUDA;
  }
  if (loss_dev) {
    bt.mode = gmode;
    if (launch_loss_reduce(bt, loss_dev, st) != cudaSuccess) return DOE_ECUDA;
  }
  return DOE_OK;
}

int doe_band_limits(const doe_geom* g, int32_t* kmax, int64_t* m_ev) {
  const int rc = check_geom(g);
  if (rc != DOE_OK && rc != DOE_EUNSUPPORTED) return rc;
  if (!kmax || !m_ev) return DOE_EINVAL;
  const long P = (long)g->pad * g->nx;
  for (int j = 0; j < g->n_lambda; ++j) {
    kmax[j] = (int32_t)band_kmax(g->lambda[j], g->dx, P, g->z, (g->flags & DOE_BANDLIMIT) != 0);
    m_ev[j] = (int64_t)(rect(g) ? rect_mev(P, (long)g->pad * g->ny, g->dx, g->lambda[j]) : band_mlim(g, g->lambda[j], P));
  }
  return DOE_OK;
}

int doe_band_limits_xy(const doe_geom* g, int32_t* kmax_x, int32_t* kmax_y, int64_t* m_ev) {
  const int rc = doe_band_limits(g, kmax_x, m_ev);
  if (rc != DOE_OK) return rc;
  if (!kmax_y) return DOE_EINVAL;
  for (int j = 0; j < g->n_lambda; ++j)
    kmax_y[j] = (int32_t)band_kmax(g->lambda[j], g->dx, (long)g->pad * g->ny, g->z, (g->flags & DOE_BANDLIMIT) != 0);
  return DOE_OK;
}

int doe_debug_band_mask(const doe_geom* g, int j, uint8_t* mask, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_geom(g);
  if (rc != DOE_OK) return rc;
  if (!mask || j < 0 || j >= g->n_lambda) return DOE_EINVAL;
  doe_geom one = *g;
  one.n_lambda = 1;
  one.lambda = g->lambda + j;
  one.n_index = g->n_index + j;
  std::vector<Slice> sl;
  std::vector<int> req_of;
  if ((rc = collect_slices(1, &one, sl, req_of)) != DOE_OK) return rc;
  const Layout lay = make_layout(sl, DOE_OP_PSF, 1, g);
  if ((rc = ws_ok(ws, ws_bytes, lay.total)) != DOE_OK) return rc;
  if ((rc = ensure_device()) != DOE_OK) return rc;
  static thread_local Batch bt;
  init_batch(bt, sl, g, ws, lay);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (launch_htab(bt, st) != cudaSuccess) return DOE_ECUDA;
  if (launch_band_mask(bt, mask, st) != cudaSuccess) return DOE_ECUDA;
  return DOE_OK;
}

int doe_render(int C, int H, int W, const float* psf, int Py, int Px, const float* img, float* out, void* ws,
               size_t ws_bytes, void* stream) {
  return render_entry(C, H, W, psf, Py, Px, img, out, ws, ws_bytes, stream);
}

size_t doe_render_workspace_bytes(int C, int H, int W) { return render_workspace(C, H, W); }

int doe_wiener(int C, int H, int W, const float* psf, int Py, int Px, const float* y, double gamma, float* out,
               void* ws, size_t ws_bytes, void* stream) {
  return wiener_entry(C, H, W, psf, Py, Px, y, gamma, out, ws, ws_bytes, stream);
}

size_t doe_wiener_workspace_bytes(int C, int H, int W) { return wiener_workspace(C, H, W); }

int doe_trace_enable(int max_records) { return trace_enable(max_records) == 0 ? DOE_OK : DOE_ECUDA; }

int doe_trace_read(int max, int* pass_ids, float* ms) {
  if (max < 0 || (max > 0 && (!pass_ids || !ms))) return DOE_EINVAL;
  const int n = trace_read(max, pass_ids, ms);
  return n < 0 ? DOE_ECUDA : n;
}

const char* doe_pass_name(int id) {
  static const char* names[TR_COUNT] = {"transfer_table", "pass_a_rows", "pass_b_columns", "pass_c_rows",
                                        "pass_c_adjoint_rows", "pass_b_adjoint_columns", "pass_a_adjoint_rows",
                                        "loss_reduce", "render_rows", "render_columns", "render_output",
                                        "band_mask", "upsample_adjoint", "adam_step", "lanczos_upsample", "lanczos_adjoint",
                                        "radial_heights", "radial_grad", "mixed_radix_twiddles"};
  return (id >= 0 && id < TR_COUNT) ? names[id] : "unknown";
}

long long doe_launch_count(void) { return launch_count(); }

int doe_fault_status(uint32_t* word) {
  if (!word) return DOE_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return DOE_ECUDA;
  unsigned int w = 0;
  if (read_faults(&w) != cudaSuccess) return DOE_ECUDA;
  *word = w;
  return DOE_OK;
}

int doe_check_wait_timeout(uint32_t polls, void* stream) {
  if (polls < 1 || polls > (1u << 20)) return DOE_EINVAL;
  return launch_wait_check(polls, static_cast<cudaStream_t>(stream)) == cudaSuccess ? DOE_OK : DOE_ECUDA;
}

int doe_debug_build(void) {
#ifdef DOE_DEBUG
  return 1;
#else
  return 0;
#endif
}

const char* doe_strerror(int code) {
  switch (code) {
    case DOE_OK: return "ok";
    case DOE_EINVAL: return "invalid argument";
    case DOE_EUNSUPPORTED: return "unsupported size or shape";
    case DOE_ENOWS: return "workspace missing, too small or misaligned";
    case DOE_ECUDA: return "CUDA runtime error";
    case DOE_ETIMEDOUT: return "timed out";
    case DOE_ESCRATCH: return "problem larger than the static no-alloc scratch (DOE_NOALLOC_SCRATCH_BYTES)";
    default: return "unknown error";
  }
}

}  // extern "C"
