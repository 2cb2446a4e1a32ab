/*
 * doe_oracle.c -- plain, slow, FP64 CPU oracle for the DOE scalar-diffraction path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (Wei et al., "Large-Area Fabrication-Aware Computational Diffractive
 * Optics", TOG 2025, Sec. 3.1):
 *   Eq. 1   Phi = 2*pi/lambda * (n_lambda - 1) * h
 *   Eq. 2   E_doe = E_in * exp(+i Phi)
 *   Eq. 3   E_dest = IFFT2( FFT2(E_doe zero-padded) (Hadamard) H_lambda )
 *           with H the band-limited angular-spectrum transfer function (the paper cites
 *           Matsushima & Shimobaba 2009 for it without writing it out; the reading used
 *           here is written next to orc_transfer_value below)
 *   Sec 3.1 I = |E_dest|^2 (the PSF)
 *   Eq. 4   gradient of sum_lambda L(I_lambda) with respect to h, derived by hand with
 *           Wirtinger calculus (the adjoint of the chain above).
 * plus the FFT convolution of an image with the PSFs used by the imaging application
 * (Sec. 5.4, Eq. 9 context) and a Rayleigh-Sommerfeld direct sum used only to pin the
 * physics.  Everything is FP64; the FFT (iterative radix-2 for powers of two, mixed-radix
 * decimation in time with direct prime-length DFTs otherwise) is written here.
 *
 * Layouts: arrays are row-major [row = y][col = x]; complex arrays are interleaved
 * (re, im) doubles, i.e. C99 double complex, the same memory layout as numpy complex128.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288

static int is_pow2(long n) { return n > 0 && (n & (n - 1)) == 0; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------
 * FFT.  Unnormalised DFT with kernel exp(sign * 2 pi i j k / n): sign = -1 is the
 * forward transform, sign = +1 the (unnormalised) inverse.  A power of two n takes the
 * iterative radix-2 path: bit-reversal permutation, then log2(n) butterfly levels with
 * twiddles taken from libm cos/sin at each level.  Any other n takes fft_any below.
 * ---------------------------------------------------------------------------------- */
static long smallest_factor(long n) {
    for (long p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Mixed-radix decimation in time, for any n.  With p the smallest prime factor of n and
 * n = p m, the p interleaved subsequences y_r[j] = x[r + p j] (r < p) are transformed
 * recursively (length m), then X[k + m q] = sum_r exp(sign 2 pi i r (k + m q) / n) Y_r[k]
 * for k < m, q < p.  A prime n (m = 1) is a direct DFT.  Twiddle angles are reduced
 * exactly in integers (r (k + m q) mod n) before libm cos/sin. */
static void fft_any(cplx *x, long n, int sign) {
    if (n <= 1) return;
    const long p = smallest_factor(n), m = n / p;
    cplx *y = (cplx *)malloc((size_t)n * sizeof(cplx));
    cplx *w = (cplx *)malloc((size_t)n * sizeof(cplx)); /* w[e] = exp(sign 2 pi i e / n) */
    for (long e = 0; e < n; ++e) {
        const double ang = (double)sign * 2.0 * ORC_PI * (double)e / (double)n;
        w[e] = cos(ang) + I * sin(ang);
    }
    for (long r = 0; r < p; ++r) {
        for (long j = 0; j < m; ++j) y[r * m + j] = x[r + p * j];
        fft_any(y + r * m, m, sign);
    }
    for (long q = 0; q < p; ++q)
        for (long k = 0; k < m; ++k) {
            const long kk = k + m * q;
            cplx s = 0;
            for (long r = 0; r < p; ++r) s += w[(r * kk) % n] * y[r * m + k];
            x[kk] = s;
        }
    free(w);
    free(y);
}

void orc_fft1d(cplx *x, long n, int sign) {
    if (n <= 1) return;
    if (!is_pow2(n)) {
        fft_any(x, n, sign);
        return;
    }
    for (long i = 1, j = 0; i < n; ++i) {
        long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (long len = 2; len <= n; len <<= 1) {
        long half = len >> 1;
        for (long k = 0; k < half; ++k) {
            double ang = (double)sign * 2.0 * ORC_PI * (double)k / (double)len;
            cplx w = cos(ang) + I * sin(ang);
            for (long s = 0; s < n; s += len) {
                cplx a = x[s + k];
                cplx b = x[s + k + half] * w;
                x[s + k] = a + b;
                x[s + k + half] = a - b;
            }
        }
    }
}

/* 2-D transform of a [ny][nx] array: 1-D transforms of every row, then of every column. */
int orc_fft2d(cplx *a, long ny, long nx, int sign) {
    if (ny < 1 || nx < 1) return -1;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < ny; ++r) orc_fft1d(a + r * nx, nx, sign);
#pragma omp parallel
    {
        cplx *col = (cplx *)malloc((size_t)ny * sizeof(cplx));
#pragma omp for schedule(static)
        for (long c = 0; c < nx; ++c) {
            for (long r = 0; r < ny; ++r) col[r] = a[r * nx + c];
            orc_fft1d(col, ny, sign);
            for (long r = 0; r < ny; ++r) a[r * nx + c] = col[r];
        }
        free(col);
    }
    return 0;
}

/* Plain O(n^2) DFT, for pinning orc_fft1d on small n. */
void orc_dft1d(const cplx *x, cplx *out, long n, int sign) {
    for (long k = 0; k < n; ++k) {
        cplx s = 0;
        for (long j = 0; j < n; ++j) {
            double ang = (double)sign * 2.0 * ORC_PI * (double)((j * k) % n) / (double)n;
            s += x[j] * (cos(ang) + I * sin(ang));
        }
        out[k] = s;
    }
}

/* ------------------------------------------------------------------------------------
 * Frequency grid and band limit.
 * Index k in [0, P) of a P-point transform is the signed frequency index
 * kt = k (k < P/2) or k - P (k >= P/2) -- numpy fftfreq order, Nyquist at -P/2 --
 * and frequency fx = kt * du with du = 1 / (P dx).
 * ---------------------------------------------------------------------------------- */
long orc_signed_index(long k, long P) { return k < P / 2 ? k : k - P; }

/* Band limit of the angular-spectrum transfer function (Matsushima & Shimobaba 2009, the
 * band-limited ASM the paper cites in Sec. 3.1 next to Eq. 3): the phase of H along one
 * frequency axis has local frequency z u / sqrt(1/lambda^2 - u^2); keeping it at or below
 * the frequency-domain Nyquist rate 1 / (2 du) gives |u| < f_lim with
 *     f_lim = 1 / (lambda * sqrt((2 du z)^2 + 1)).
 * kmax is the largest integer k with k du < f_lim (strict), i.e. ceil(f_lim/du) - 1,
 * capped at P/2 (at the cap the whole grid is kept: the band limit is inactive).  With
 * bandlimit == 0 every index is kept (kmax = P/2). */
long orc_kmax(double lambda, double dx, long P, double z, int bandlimit) {
    if (!bandlimit) return P / 2;
    double du = 1.0 / ((double)P * dx);
    double t = 2.0 * du * z;
    double flim = 1.0 / (lambda * sqrt(t * t + 1.0));
    long k = (long)ceil(flim / du) - 1;
    if (k > P / 2) k = P / 2;
    if (k < 0) k = 0;
    return k;
}

/* Evanescent cut: a sample propagates iff lambda^2 (fx^2 + fy^2) < 1.  With
 * m = kt^2 + lt^2 (an exact integer) that is m < 1/(lambda du)^2, i.e. m < m_ev with
 * m_ev = ceil(1 / (lambda du)^2) evaluated once in FP64. */
int64_t orc_mev(double lambda, double dx, long P) {
    double du = 1.0 / ((double)P * dx);
    double ld = lambda * du;
    double x = 1.0 / (ld * ld);
    if (x > 9.0e18) return INT64_MAX;
    return (int64_t)ceil(x);
}

/* Circular band limit (bandlimit == 2): the disc fx^2 + fy^2 < f_lim^2 instead of the square
 * |fx|, |fy| < f_lim (the paper cites the band-limited ASM without fixing the window's shape;
 * the disc is the rotation-invariant reading).  With m = kt^2 + lt^2 that is m < (f_lim/du)^2,
 * i.e. m < m_circ = ceil((f_lim/du)^2) evaluated once in FP64.  The disc lies inside the
 * square of kmax, so the square bounds still hold.  Returns the bound of m that the transfer
 * function applies: m_ev, or min(m_ev, m_circ) for the disc. */
int64_t orc_mlim(double lambda, double dx, long P, double z, int bandlimit) {
    int64_t mev = orc_mev(lambda, dx, P);
    if (bandlimit != 2) return mev;
    double du = 1.0 / ((double)P * dx);
    double t = 2.0 * du * z;
    double flim = 1.0 / (lambda * sqrt(t * t + 1.0));
    double r = flim / du;
    double x = r * r;
    int64_t mc = x > 9.0e18 ? INT64_MAX : (int64_t)ceil(x);
    return mc < mev ? mc : mev;
}

/* H at integer frequency indices (kt, lt):
 *   exp(+i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2))  inside the band and propagating,
 *   0 otherwise.  The e^{+i} sign matches Eq. 2's e^{+i Phi} (Goodman's convention). */
static cplx orc_transfer_value(long kt, long lt, long kmax, int64_t mev, double du, double lambda,
                               double z) {
    if (labs(kt) > kmax || labs(lt) > kmax) return 0;
    int64_t m = (int64_t)kt * kt + (int64_t)lt * lt;
    if (m >= mev) return 0;
    double fx = (double)kt * du, fy = (double)lt * du;
    double s = 1.0 / (lambda * lambda) - fx * fx - fy * fy;
    double phi = 2.0 * ORC_PI * z * sqrt(s);
    return cos(phi) + I * sin(phi);
}

/* Full [P][P] transfer function in FFT order, H[l][k]. */
void orc_transfer(cplx *H, long P, double dx, double z, double lambda, int bandlimit) {
    long kmax = orc_kmax(lambda, dx, P, z, bandlimit);
    int64_t mev = orc_mlim(lambda, dx, P, z, bandlimit);
    double du = 1.0 / ((double)P * dx);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < P; ++l)
        for (long k = 0; k < P; ++k)
            H[l * P + k] = orc_transfer_value(orc_signed_index(k, P), orc_signed_index(l, P), kmax,
                                              mev, du, lambda, z);
}

/* Band mask, 1 where H != 0 by the integer rules above ([P][P] bytes). */
void orc_band_mask(uint8_t *mask, long P, double dx, double z, double lambda, int bandlimit) {
    long kmax = orc_kmax(lambda, dx, P, z, bandlimit);
    int64_t mev = orc_mlim(lambda, dx, P, z, bandlimit);
    for (long l = 0; l < P; ++l)
        for (long k = 0; k < P; ++k) {
            long kt = orc_signed_index(k, P), lt = orc_signed_index(l, P);
            int64_t m = (int64_t)kt * kt + (int64_t)lt * lt;
            mask[l * P + k] = (labs(kt) <= kmax && labs(lt) <= kmax && m < mev) ? 1 : 0;
        }
}

/* ------------------------------------------------------------------------------------
 * Eq. 1-2: DOE field, and the 2x (or 1x) zero padding.  The N x N DOE sits at offset
 * off = (P - N)/2 in both axes of the P x P grid; every other sample is zero.  The
 * propagation keeps the grid, so output sample (y, x) is at the same physical position
 * as padded input sample (y, x).
 * ---------------------------------------------------------------------------------- */
static double orc_kprime(double lambda, double n_index) {
    return 2.0 * ORC_PI * (n_index - 1.0) / lambda;
}

static void orc_doe_field(cplx *e_doe, long N, const float *h, const cplx *e_in, double kp) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N * N; ++i) {
        double phi = kp * (double)h[i];
        cplx t = cos(phi) + I * sin(phi);
        e_doe[i] = e_in ? e_in[i] * t : t;
    }
}

static void orc_pad(cplx *pad, long P, const cplx *src, long N) {
    long off = (P - N) / 2;
    memset(pad, 0, (size_t)P * P * sizeof(cplx));
    for (long i = 0; i < N; ++i)
        memcpy(pad + (i + off) * P + off, src + i * N, (size_t)N * sizeof(cplx));
}

/* Eq. 3 on a padded field in place: a <- IFFT2( FFT2(a) * H ), numpy normalisation
 * (forward unnormalised, inverse 1/P^2).  conj_h != 0 uses conj(H) (the adjoint). */
static void orc_asm_inplace(cplx *a, long P, double dx, double z, double lambda, int bandlimit,
                            int conj_h) {
    long kmax = orc_kmax(lambda, dx, P, z, bandlimit);
    int64_t mev = orc_mlim(lambda, dx, P, z, bandlimit);
    double du = 1.0 / ((double)P * dx);
    orc_fft2d(a, P, P, -1);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < P; ++l)
        for (long k = 0; k < P; ++k) {
            cplx hv = orc_transfer_value(orc_signed_index(k, P), orc_signed_index(l, P), kmax, mev,
                                         du, lambda, z);
            a[l * P + k] *= conj_h ? conj(hv) : hv;
        }
    orc_fft2d(a, P, P, +1);
    double s = 1.0 / ((double)P * (double)P);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < P * P; ++i) a[i] *= s;
}

/* E_dest for one wavelength: e_out is [P][P], P = pad * N. */
int orc_propagate(long N, long pad, double dx, double z, double lambda, double n_index,
                  int bandlimit, const float *h, const cplx *e_in, cplx *e_out) {
    if (N < 2 || (N & 1) || (pad != 1 && pad != 2)) return -1;
    long P = pad * N;
    cplx *e_doe = (cplx *)malloc((size_t)N * N * sizeof(cplx));
    if (!e_doe) return -2;
    orc_doe_field(e_doe, N, h, e_in, orc_kprime(lambda, n_index));
    orc_pad(e_out, P, e_doe, N);
    free(e_doe);
    orc_asm_inplace(e_out, P, dx, z, lambda, bandlimit, 0);
    return 0;
}

/* PSF I = |E_dest|^2 for one wavelength, FP64 [P][P]. */
int orc_psf(long N, long pad, double dx, double z, double lambda, double n_index, int bandlimit,
            const float *h, const cplx *e_in, double *psf) {
    long P = pad * N;
    cplx *e = (cplx *)malloc((size_t)P * P * sizeof(cplx));
    if (!e) return -2;
    int rc = orc_propagate(N, pad, dx, z, lambda, n_index, bandlimit, h, e_in, e);
    if (rc == 0) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < P * P; ++i) psf[i] = creal(e[i]) * creal(e[i]) + cimag(e[i]) * cimag(e[i]);
    }
    free(e);
    return rc;
}

/* Row-subset PSF: exact FP64 output rows rows[0..nrows) only, for grids whose full FP64
 * field does not fit in host memory.  Same arithmetic as orc_psf, ordered differently:
 * row FFT of the N non-zero rows, then per column: FFT -> *H -> IFFT keeping the requested
 * rows, then the row IFFT of those rows.  Peak memory: N*P + nrows*P complex. */
int orc_psf_rows(long N, long pad, double dx, double z, double lambda, double n_index,
                 int bandlimit, const float *h, const cplx *e_in, long nrows, const long *rows,
                 double *psf_rows) {
    if (N < 2 || (N & 1) || (pad != 1 && pad != 2)) return -1;
    long P = pad * N, off = (P - N) / 2;
    long kmax = orc_kmax(lambda, dx, P, z, bandlimit);
    int64_t mev = orc_mlim(lambda, dx, P, z, bandlimit);
    double du = 1.0 / ((double)P * dx);
    double kp = orc_kprime(lambda, n_index);
    cplx *a = (cplx *)malloc((size_t)N * P * sizeof(cplx));
    cplx *out = (cplx *)calloc((size_t)nrows * P, sizeof(cplx));
    if (!a || !out) { free(a); free(out); return -2; }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        cplx *row = a + i * P;
        memset(row, 0, (size_t)P * sizeof(cplx));
        for (long j = 0; j < N; ++j) {
            double phi = kp * (double)h[i * N + j];
            cplx t = cos(phi) + I * sin(phi);
            row[off + j] = e_in ? e_in[i * N + j] * t : t;
        }
        orc_fft1d(row, P, -1);
    }
#pragma omp parallel
    {
        cplx *col = (cplx *)malloc((size_t)P * sizeof(cplx));
#pragma omp for schedule(static)
        for (long k = 0; k < P; ++k) {
            memset(col, 0, (size_t)P * sizeof(cplx));
            for (long i = 0; i < N; ++i) col[off + i] = a[i * P + k];
            orc_fft1d(col, P, -1);
            long kt = orc_signed_index(k, P);
            for (long l = 0; l < P; ++l)
                col[l] *= orc_transfer_value(kt, orc_signed_index(l, P), kmax, mev, du, lambda, z);
            orc_fft1d(col, P, +1);
            for (long r = 0; r < nrows; ++r) out[r * P + k] = col[rows[r]];
        }
        free(col);
    }
    free(a);
    double s = 1.0 / ((double)P * (double)P);
#pragma omp parallel for schedule(static)
    for (long r = 0; r < nrows; ++r) {
        orc_fft1d(out + r * P, P, +1);
        for (long x = 0; x < P; ++x) {
            cplx e = out[r * P + x] * s;
            psf_rows[r * P + x] = creal(e) * creal(e) + cimag(e) * cimag(e);
        }
    }
    free(out);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Row-masked adjoint for grids whose FP64 field does not fit host memory (Sec. 3.1, Eq. 4
 * with dL/dI non-zero only on the output rows `rows`, one wavelength).  The output rows of
 * E_out are formed as in orc_psf_rows; then
 *   g_out = G E_out on those rows (G = dL/dI, zero on every other row),
 *   g_pad = IFFT2( conj(H) FFT2(g_out) )  (numpy normalisation),
 * where the column transforms see only the non-zero rows and keep only the requested DOE rows
 * `drows` (0-based DOE row indices, padded row off + d), and
 *   dL/dh[d][x] = -2 k' Im( conj(g_pad[off + d][off + x]) E_doe[d][x] ).
 * rows must be distinct.  g_rows: float [nrows][P]; grad_rows: double [nd][N] (overwritten).
 * ---------------------------------------------------------------------------------- */
int orc_grad_rows(long N, long pad, double dx, double z, double lambda, double n_index,
                  int bandlimit, const float *h, const cplx *e_in, long nrows, const long *rows,
                  const float *g_rows, long nd, const long *drows, double *grad_rows) {
    if (N < 2 || (N & 1) || (pad != 1 && pad != 2)) return -1;
    long P = pad * N, off = (P - N) / 2;
    long kmax = orc_kmax(lambda, dx, P, z, bandlimit);
    int64_t mev = orc_mlim(lambda, dx, P, z, bandlimit);
    double du = 1.0 / ((double)P * dx);
    double kp = orc_kprime(lambda, n_index);
    double s = 1.0 / ((double)P * (double)P);
    cplx *a = (cplx *)malloc((size_t)N * P * sizeof(cplx));
    cplx *out = (cplx *)calloc((size_t)nrows * P, sizeof(cplx));
    if (!a || !out) { free(a); free(out); return -2; }
    /* forward: row FFT of the N DOE rows of E_pad */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        cplx *row = a + i * P;
        memset(row, 0, (size_t)P * sizeof(cplx));
        for (long j = 0; j < N; ++j) {
            double phi = kp * (double)h[i * N + j];
            cplx t = cos(phi) + I * sin(phi);
            row[off + j] = e_in ? e_in[i * N + j] * t : t;
        }
        orc_fft1d(row, P, -1);
    }
    /* forward: per column, FFT, x H, IFFT; keep the requested output rows */
#pragma omp parallel
    {
        cplx *col = (cplx *)malloc((size_t)P * sizeof(cplx));
#pragma omp for schedule(static)
        for (long k = 0; k < P; ++k) {
            memset(col, 0, (size_t)P * sizeof(cplx));
            for (long i = 0; i < N; ++i) col[off + i] = a[i * P + k];
            orc_fft1d(col, P, -1);
            long kt = orc_signed_index(k, P);
            for (long l = 0; l < P; ++l)
                col[l] *= orc_transfer_value(kt, orc_signed_index(l, P), kmax, mev, du, lambda, z);
            orc_fft1d(col, P, +1);
            for (long r = 0; r < nrows; ++r) out[r * P + k] = col[rows[r]];
        }
        free(col);
    }
    free(a);
    /* E_out on the rows (row IFFT, 1/P^2), g_out = G E_out, then the row FFT of g_out */
#pragma omp parallel for schedule(static)
    for (long r = 0; r < nrows; ++r) {
        cplx *row = out + r * P;
        orc_fft1d(row, P, +1);
        for (long x = 0; x < P; ++x) row[x] *= s * (double)g_rows[r * P + x];
        orc_fft1d(row, P, -1);
    }
    /* adjoint: per column, FFT over the (sparse) rows, x conj(H), IFFT; keep the DOE rows */
    cplx *b = (cplx *)calloc((size_t)nd * P, sizeof(cplx));
    if (!b) { free(out); return -2; }
#pragma omp parallel
    {
        cplx *col = (cplx *)malloc((size_t)P * sizeof(cplx));
#pragma omp for schedule(static)
        for (long k = 0; k < P; ++k) {
            memset(col, 0, (size_t)P * sizeof(cplx));
            for (long r = 0; r < nrows; ++r) col[rows[r]] = out[r * P + k];
            orc_fft1d(col, P, -1);
            long kt = orc_signed_index(k, P);
            for (long l = 0; l < P; ++l)
                col[l] *= conj(orc_transfer_value(kt, orc_signed_index(l, P), kmax, mev, du, lambda, z));
            orc_fft1d(col, P, +1);
            for (long d = 0; d < nd; ++d) b[d * P + k] = col[off + drows[d]];
        }
        free(col);
    }
    free(out);
    /* row IFFT of the kept DOE rows, 1/P^2, crop to the DOE window, dL/dh */
#pragma omp parallel for schedule(static)
    for (long d = 0; d < nd; ++d) {
        cplx *row = b + d * P;
        long i = drows[d];
        orc_fft1d(row, P, +1);
        for (long x = 0; x < N; ++x) {
            cplx g = row[off + x] * s;
            double phi = kp * (double)h[i * N + x];
            cplx e = cos(phi) + I * sin(phi);
            if (e_in) e *= e_in[i * N + x];
            grad_rows[d * N + x] = -2.0 * kp * cimag(conj(g) * e);
        }
    }
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Gradient (Eq. 4).  For each wavelength j:
 *   E_out = A_j E_pad with A_j = (1/P^2) F^H diag(H_j) F (F = unnormalised 2-D DFT);
 *   g_out = dL/d conj(E_out) = 2 (I - T) E_out      (mode 0: L = sum (I - T)^2)
 *                            = G E_out               (mode 1: G = dL/dI given)
 *   g_pad = A_j^H g_out = IFFT2( conj(H_j) FFT2(g_out) )   (numpy normalisation)
 *   g_doe = g_pad cropped to the DOE window
 *   dL/dh += -2 k'_j Im( conj(g_doe) E_doe ),  k'_j = 2 pi (n_j - 1) / lambda_j
 * t_or_g is [L][P][P]; grad is [N][N] (overwritten); loss (mode 0) is sum over j.
 * ---------------------------------------------------------------------------------- */
int orc_grad(long N, long pad, double dx, double z, long L, const double *lambda,
             const double *n_index, int bandlimit, const float *h, const cplx *e_in,
             const float *t_or_g, int mode, double *grad, double *loss) {
    if (N < 2 || (N & 1) || (pad != 1 && pad != 2)) return -1;
    long P = pad * N, off = (P - N) / 2;
    cplx *e_doe = (cplx *)malloc((size_t)N * N * sizeof(cplx));
    cplx *a = (cplx *)malloc((size_t)P * P * sizeof(cplx));
    if (!e_doe || !a) { free(e_doe); free(a); return -2; }
    memset(grad, 0, (size_t)N * N * sizeof(double));
    double total = 0.0;
    for (long j = 0; j < L; ++j) {
        double kp = orc_kprime(lambda[j], n_index[j]);
        orc_doe_field(e_doe, N, h, e_in, kp);
        orc_pad(a, P, e_doe, N);
        orc_asm_inplace(a, P, dx, z, lambda[j], bandlimit, 0);
        const float *tj = t_or_g + (size_t)j * P * P;
        double lj = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : lj)
        for (long i = 0; i < P * P; ++i) {
            double in = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
            if (mode == 0) {
                double d = in - (double)tj[i];
                lj += d * d;
                a[i] *= 2.0 * d;
            } else {
                a[i] *= (double)tj[i];
            }
        }
        total += lj;
        orc_asm_inplace(a, P, dx, z, lambda[j], bandlimit, 1);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < N; ++i)
            for (long x = 0; x < N; ++x) {
                cplx g = a[(i + off) * P + (x + off)];
                grad[i * N + x] += -2.0 * kp * cimag(conj(g) * e_doe[i * N + x]);
            }
    }
    if (loss) *loss = total;
    free(e_doe);
    free(a);
    return 0;
}

/* Loss alone (mode 0) with FP64 heights, for finite differences on small grids. */
int orc_loss_l2(long N, long pad, double dx, double z, long L, const double *lambda,
                const double *n_index, int bandlimit, const double *h, const cplx *e_in,
                const float *target, double *loss) {
    if (N < 2 || (N & 1) || (pad != 1 && pad != 2)) return -1;
    long P = pad * N;
    cplx *e_doe = (cplx *)malloc((size_t)N * N * sizeof(cplx));
    cplx *a = (cplx *)malloc((size_t)P * P * sizeof(cplx));
    if (!e_doe || !a) { free(e_doe); free(a); return -2; }
    double total = 0.0;
    for (long j = 0; j < L; ++j) {
        double kp = orc_kprime(lambda[j], n_index[j]);
        for (long i = 0; i < N * N; ++i) {
            double phi = kp * h[i];
            cplx t = cos(phi) + I * sin(phi);
            e_doe[i] = e_in ? e_in[i] * t : t;
        }
        orc_pad(a, P, e_doe, N);
        orc_asm_inplace(a, P, dx, z, lambda[j], bandlimit, 0);
        const float *tj = target + (size_t)j * P * P;
        double lj = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : lj)
        for (long i = 0; i < P * P; ++i) {
            double in = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
            double d = in - (double)tj[i];
            lj += d * d;
        }
        total += lj;
    }
    *loss = total;
    free(e_doe);
    free(a);
    return 0;
}

/* Exact-difference finite differences of the L2 loss (mode 0) at selected DOE pixels.
 * FP32 cannot resolve L(h + eps e_p) - L(h), so this evaluates it algebraically in FP64:
 * moving pixel p by +-eps changes E_out by d = E_doe,p (e^{+-i k' eps} - 1) K(. - p) with
 * K = A_j applied to a unit impulse at the padded origin (a circular shift moves it to p),
 * so dI = 2 Re(conj(E) d) + |d|^2 and dL = sum 2 (I - T) dI + dI^2 exactly.
 * fd[q] = (dL(+eps) - dL(-eps)) / (2 eps), summed over wavelengths. */
int orc_fd_exact(long N, long pad, double dx, double z, long L, const double *lambda,
                 const double *n_index, int bandlimit, const float *h, const cplx *e_in,
                 const float *target, long npix, const long *pix_y, const long *pix_x, double eps,
                 double *fd) {
    if (N < 2 || (N & 1) || (pad != 1 && pad != 2)) return -1;
    long P = pad * N, off = (P - N) / 2;
    cplx *e_doe = (cplx *)malloc((size_t)N * N * sizeof(cplx));
    cplx *e = (cplx *)malloc((size_t)P * P * sizeof(cplx));
    cplx *K = (cplx *)malloc((size_t)P * P * sizeof(cplx));
    if (!e_doe || !e || !K) { free(e_doe); free(e); free(K); return -2; }
    for (long q = 0; q < npix; ++q) fd[q] = 0.0;
    for (long j = 0; j < L; ++j) {
        double kp = orc_kprime(lambda[j], n_index[j]);
        orc_doe_field(e_doe, N, h, e_in, kp);
        orc_pad(e, P, e_doe, N);
        orc_asm_inplace(e, P, dx, z, lambda[j], bandlimit, 0);
        memset(K, 0, (size_t)P * P * sizeof(cplx));
        K[0] = 1.0;
        orc_asm_inplace(K, P, dx, z, lambda[j], bandlimit, 0);
        const float *tj = target + (size_t)j * P * P;
        for (long q = 0; q < npix; ++q) {
            long py = pix_y[q] + off, px = pix_x[q] + off;
            cplx ep = e_doe[pix_y[q] * N + pix_x[q]];
            double dl[2];
            for (int sgn = 0; sgn < 2; ++sgn) {
                double s = sgn == 0 ? eps : -eps;
                cplx c = ep * ((cos(kp * s) - 1.0) + I * sin(kp * s));
                double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
                for (long y = 0; y < P; ++y) {
                    long ky = (y - py + P) % P;
                    for (long x = 0; x < P; ++x) {
                        long kx = (x - px + P) % P;
                        cplx d = c * K[ky * P + kx];
                        cplx ev = e[y * P + x];
                        double di = 2.0 * creal(conj(ev) * d) + creal(d) * creal(d) + cimag(d) * cimag(d);
                        double in = creal(ev) * creal(ev) + cimag(ev) * cimag(ev);
                        double r = in - (double)tj[y * P + x];
                        acc += 2.0 * r * di + di * di;
                    }
                }
                dl[sgn] = acc;
            }
            fd[q] += (dl[0] - dl[1]) / (2.0 * eps);
        }
    }
    free(e_doe);
    free(e);
    free(K);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Image formation by PSF convolution (the imaging application's convolution model,
 * Sec. 5.4 around Eq. 9).  Channel c uses PSF c:
 *   k_c[u][v] = psf_c[P/2 - H/2 + u][P/2 - W/2 + v],  u < H, v < W  (crop at the axis)
 *   k_c /= sum(k_c)
 *   out_c[y][x] = sum_{u,v} img_c[y + H/2 - u][x + W/2 - v] k_c[u][v]   (zero outside)
 * computed here with 2H x 2W FFTs (linear convolution, no wrap).
 * ---------------------------------------------------------------------------------- */
int orc_render(long C, long H, long W, const float *psf, long Py, long Px, const float *img,
               double *out) {
    if (!is_pow2(H) || !is_pow2(W) || H > Py || W > Px) return -1;
    long FH = 2 * H, FW = 2 * W;
    cplx *A = (cplx *)malloc((size_t)FH * FW * sizeof(cplx));
    cplx *B = (cplx *)malloc((size_t)FH * FW * sizeof(cplx));
    if (!A || !B) { free(A); free(B); return -2; }
    for (long c = 0; c < C; ++c) {
        const float *pc = psf + (size_t)c * Py * Px;
        const float *ic = img + (size_t)c * H * W;
        memset(A, 0, (size_t)FH * FW * sizeof(cplx));
        memset(B, 0, (size_t)FH * FW * sizeof(cplx));
        double ksum = 0.0;
        for (long u = 0; u < H; ++u)
            for (long v = 0; v < W; ++v) {
                double kv = (double)pc[(Py / 2 - H / 2 + u) * Px + (Px / 2 - W / 2 + v)];
                B[u * FW + v] = kv;
                ksum += kv;
                A[u * FW + v] = (double)ic[u * W + v];
            }
        orc_fft2d(A, FH, FW, -1);
        orc_fft2d(B, FH, FW, -1);
        for (long i = 0; i < FH * FW; ++i) A[i] *= B[i];
        orc_fft2d(A, FH, FW, +1);
        double s = 1.0 / ((double)FH * (double)FW * ksum);
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x)
                out[(size_t)c * H * W + y * W + x] = creal(A[(y + H / 2) * FW + (x + W / 2)]) * s;
    }
    free(A);
    free(B);
    return 0;
}

/* Wiener deconvolution (Eq. 9): xhat = IFFT( conj(K) / (|K|^2 + gamma) * Y ), with K the
 * FFT of the normalised PSF crop placed with its centre at the origin of an H x W grid
 * (circular model).  Used only as an oracle for the Wiener row. */
int orc_wiener(long C, long H, long W, const float *psf, long Py, long Px, const float *y,
               double gamma, double *out) {
    if (!is_pow2(H) || !is_pow2(W) || H > Py || W > Px) return -1;
    cplx *K = (cplx *)malloc((size_t)H * W * sizeof(cplx));
    cplx *Y = (cplx *)malloc((size_t)H * W * sizeof(cplx));
    if (!K || !Y) { free(K); free(Y); return -2; }
    for (long c = 0; c < C; ++c) {
        const float *pc = psf + (size_t)c * Py * Px;
        memset(K, 0, (size_t)H * W * sizeof(cplx));
        double ksum = 0.0;
        for (long u = 0; u < H; ++u)
            for (long v = 0; v < W; ++v) ksum += (double)pc[(Py / 2 - H / 2 + u) * Px + (Px / 2 - W / 2 + v)];
        for (long u = 0; u < H; ++u)
            for (long v = 0; v < W; ++v) {
                long yy = (u - H / 2 + H) % H, xx = (v - W / 2 + W) % W;
                K[yy * W + xx] = (double)pc[(Py / 2 - H / 2 + u) * Px + (Px / 2 - W / 2 + v)] / ksum;
            }
        for (long i = 0; i < H * W; ++i) Y[i] = (double)y[(size_t)c * H * W + i];
        orc_fft2d(K, H, W, -1);
        orc_fft2d(Y, H, W, -1);
        for (long i = 0; i < H * W; ++i) {
            double k2 = creal(K[i]) * creal(K[i]) + cimag(K[i]) * cimag(K[i]);
            Y[i] = conj(K[i]) / (k2 + gamma) * Y[i];
        }
        orc_fft2d(Y, H, W, +1);
        for (long i = 0; i < H * W; ++i) out[(size_t)c * H * W + i] = creal(Y[i]) / ((double)H * W);
    }
    free(K);
    free(Y);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Rayleigh-Sommerfeld (first kind) direct sum, used to pin the oracle's physics:
 *   E(x, y, z) = sum_{x', y'} E_doe(x', y') * z/(2 pi r^2) * (1/r - i k) * e^{+i k r} * dx^2,
 *   r = sqrt((x - x')^2 + (y - y')^2 + z^2), k = 2 pi / lambda.
 * The DOE (N x N) and the output (P x P) share the pitch dx and the same sample grid as
 * the padded ASM: output sample (y, x) is at (y - off) dx, (x - off) dx from DOE sample 0.
 * ---------------------------------------------------------------------------------- */
int orc_rs_direct(long N, long P, double dx, double z, double lambda, const cplx *e_doe,
                  cplx *e_out) {
    long off = (P - N) / 2;
    double k = 2.0 * ORC_PI / lambda;
#pragma omp parallel for schedule(dynamic)
    for (long y = 0; y < P; ++y)
        for (long x = 0; x < P; ++x) {
            cplx acc = 0;
            for (long i = 0; i < N; ++i)
                for (long j = 0; j < N; ++j) {
                    double ddy = (double)(y - off - i) * dx, ddx = (double)(x - off - j) * dx;
                    double r2 = ddx * ddx + ddy * ddy + z * z;
                    double r = sqrt(r2);
                    cplx kern = z / (2.0 * ORC_PI * r2) * (1.0 / r - I * k) * (cos(k * r) + I * sin(k * r));
                    acc += e_doe[i * N + j] * kern;
                }
            e_out[y * P + x] = acc * dx * dx;
        }
    return 0;
}
