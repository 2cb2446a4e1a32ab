/*
 * doe.h -- C ABI of libdoe: scalar-diffraction simulation of a diffractive optical element
 * (DOE) on one NVIDIA B300 (sm_103a), after Wei et al., "Large-Area Fabrication-Aware
 * Computational Diffractive Optics", ACM TOG 44(6), 2025, Sec. 3.1.
 *
 * The path: height map h -> phase Phi = 2 pi (n - 1) h / lambda (Eq. 1) -> transmittance
 * E_doe = E_in exp(+i Phi) (Eq. 2) -> zero padding -> FFT -> product with the band-limited
 * angular-spectrum transfer function H_lambda -> inverse FFT (Eq. 3) -> intensity
 * I = |E_dest|^2 (the PSF) per wavelength; the gradient of sum_lambda L(I_lambda) with
 * respect to h (Eq. 4) by a hand-written adjoint; and the convolution of an image with the
 * PSFs (the image-formation model behind the imaging application's Eq. 9).
 *
 * Conventions shared by every entry point
 *  - Arrays are row-major [row = y][col = x].  "complex" arrays are interleaved (re, im)
 *    float pairs (8 bytes per sample, the layout of CUDA float2 / torch.complex64).
 *  - Every data pointer is DEVICE memory owned by the caller, except the geometry's
 *    lambda / n_index arrays, which are HOST memory read during the call.
 *  - stream is a cudaStream_t passed as void*; NULL means the legacy default stream.  All
 *    work is enqueued on it asynchronously; no call synchronises the device.  Device-side
 *    faults therefore surface at the caller's next synchronisation.
 *  - The library allocates no device memory on these paths: the caller passes a workspace
 *    (`ws`, `ws_bytes`, 256-byte aligned) sized with the matching *_workspace_bytes call.
 *    Read-only FFT twiddle tables live in static device memory (about 1.1 MB per device,
 *    held until the process exits) and are uploaded on the first call on each device, or by
 *    doe_init(); make that first call before capturing a stream into a CUDA graph.
 *  - Return value: DOE_OK (0) or a negative DOE_E* code; nothing is launched when a call
 *    fails validation.  No C++ exception crosses this interface.
 *  - Grid: N x N DOE samples (N even, 16 <= N), padded to P = pad * N per axis with the DOE
 *    at offset (P - N) / 2; output sample (y, x) lies at the same physical position as padded
 *    input sample (y, x) (the optical axis is at (P/2, P/2)).  P is either a power of two
 *    <= 65536 (above 16384 each row / column transform is split across a thread-block
 *    cluster of P / 8192 CTAs), or an even P whose prime factors are 2, 3, 5 or primes up to
 *    127 (Table 2's 3600, 28800 and 40000 grids; the 67 of its large-area grid): a mixed-radix
 *    FFT in shared memory (no band compaction), one CTA per transform up to P = 8192, above
 *    that a cluster of Q in {2, 3, 4, 5, 8} CTAs of P / Q <= 8192 points each (P <= 65536).
 *  - Rectangular grids (Table 2's large-area grid is not square): nx x ny DOE samples padded
 *    to Px = pad nx by Py = pad ny, arrays [Py][Px] / [ny][nx].  Each axis keeps its own
 *    frequency step (1 / (Px dx), 1 / (Py dx)) and band limit (the square rule per axis); a
 *    sample propagates iff lambda^2 (fx^2 + fy^2) < 1, in integers kt^2 B^2 + lt^2 A^2 <
 *    ceil((Px Py dx / (g lambda))^2) with g = gcd(Px, Py), A = Px / g, B = Py / g.  Supported
 *    on the mixed-radix passes when each side is at most 8192 with the factors above (powers of
 *    two included; one CTA per transform) or splits as Q x M with Q in {8, 5, 4, 3, 2, 16} and
 *    M <= 8192 with those factors (a cluster of Q CTAs per transform, sides up to 131072, such
 *    as Table 2's 128640 x 85760 = 16 x 8040 by 16 x 5360), with the separable band, no
 *    upsampling and no parametric incident field (an e_in array is supported).  Other
 *    rectangles return DOE_EUNSUPPORTED.
 */
#ifndef DOE_H
#define DOE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DOE_OK 0
#define DOE_EINVAL (-1)       /* an argument is out of range or a required pointer is NULL */
#define DOE_EUNSUPPORTED (-2) /* a size or shape this build does not implement */
#define DOE_ENOWS (-3)        /* workspace missing, too small or not 256-byte aligned */
#define DOE_ECUDA (-4)        /* a CUDA runtime call or kernel launch failed */
#define DOE_ETIMEDOUT (-5)    /* a bounded host-side wait expired (serving layer) */
#define DOE_ESCRATCH (-6)     /* the problem needs more scratch than doe_psf_noalloc's static buffer */

/* ---- geometry flags ---- */
#define DOE_BANDLIMIT 0x1u /* apply the band limit of the transfer function (default on) */
/* With DOE_BANDLIMIT: a circular band, fx^2 + fy^2 < f_lim^2, instead of the separable square
 * |fx|, |fy| < f_lim.  The paper cites the band-limited angular spectrum method (Sec. 3.1, next
 * to Eq. 3) without fixing the window's shape; the disc is the rotation-invariant reading.  In
 * integers: (kt, lt) is kept iff kt^2 + lt^2 < ceil((f_lim / du)^2) (the disc lies inside the
 * square of kmax). */
#define DOE_BANDLIMIT_CIRCULAR 0x2u
/* Super-resolved design input: the heights h are a layout of (ny / f) x (nx / f) cells at
 * pitch f dx, nearest-upsampled by f = 2^u (u = 0..3) onto the dx simulation grid inside the
 * first pass (h_sim[i][x] = h[i / f][x / f]); gradients are returned on the layout (the sum
 * over each f x f block, the adjoint of the upsampling).  nx / f >= 4. */
#define DOE_UPSAMPLE_SHIFT 4
#define DOE_UPSAMPLE(u) (((uint32_t)(u) & 3u) << DOE_UPSAMPLE_SHIFT)
/* With DOE_UPSAMPLE(u), u >= 1: Lanczos-3 interpolation instead of nearest (the smooth kernel
 * the paper compares against, Sec. 3.2):
 *   h_sim[i][x] = sum_{m,n} w(i, m) w(x, n) h[m][n],
 *   w(x, n) = K(u_x - n) / sum_n' K(u_x - n'),  u_x = (x + 1/2) / f - 1/2 (cell centres),
 *   K(t) = sinc(t) sinc(t / 3) for |t| < 3, else 0,  cells clamped to the layout at its edges;
 * gradients are returned on the layout through the transpose.  The interpolation is a pre-pass
 * into the workspace (N^2 floats per Lanczos request plus one shared (N/f) x N buffer of the
 * separable passes, counted by doe_workspace_bytes*). */
#define DOE_UPSAMPLE_LANCZOS3 0x40u

/* ---- operations, for doe_workspace_bytes ---- */
#define DOE_OP_PROPAGATE 1
#define DOE_OP_PSF 2
#define DOE_OP_GRAD 3

/* ---- gradient modes ---- */
#define DOE_GRAD_L2_TARGET 0 /* L = sum_lambda sum_xy (I - T)^2 with target T */
#define DOE_GRAD_VJP 1       /* vector-Jacobian product with a given dL/dI */

/* Geometry of one DOE evaluation (Sec. 3.1 notation). */
typedef struct doe_geom {
    int32_t nx, ny;        /* DOE samples per axis; even, >= 16; ny != nx as in the rectangular-grid note above */
    int32_t pad;           /* 1 or 2: padded grid P = pad * n per axis (the paper's grids are 2x) */
    double dx;             /* sampling pitch [m], square pixels, > 0 */
    double z;              /* propagation distance [m], > 0 */
    int32_t n_lambda;      /* number of wavelengths, 1..64 */
    const double* lambda;  /* HOST [n_lambda] wavelengths [m], > 0 */
    const double* n_index; /* HOST [n_lambda] refractive index n_lambda of the DOE material, >= 1 */
    uint32_t flags;        /* DOE_BANDLIMIT | DOE_UPSAMPLE(u) [| DOE_UPSAMPLE_LANCZOS3] */
    /* Parametric incident field E_in (Eq. 2: a plane or spherical wave; Sec. 2.3 scales over
     * incidence angles), per wavelength, at sample (i, j), x = (j - nx/2) dx, y = (i - ny/2) dx
     * (the optical axis at padded index P/2):
     *   E_in = exp(+i 2 pi (x sin theta_x + y sin theta_y) / lambda)
     *        * [src_d == 0 ? 1 : (|d| / r) exp(+i sgn(d) 2 pi (r - |d|) / lambda)],
     *   r = sqrt(x^2 + y^2 + d^2), d = src_d.
     * All zero (the default): a unit plane wave at normal incidence.  Multiplies the e_in array
     * when both are given; evaluated inside the DOE-row passes (no E_in array in memory). */
    double theta_x, theta_y; /* incidence angles [rad], |theta| < pi/2 */
    double src_d;            /* [m]: > 0 point source |d| before the DOE, < 0 focus |d| behind it */
} doe_geom;

/* Per-device set-up (uploads the twiddle tables).  Optional: the first call of any entry
 * point on a device does it.  Uses the current CUDA device.  Returns DOE_OK or DOE_ECUDA. */
int doe_init(void);

/* Bytes of workspace the given operation needs for geometry g (0 on invalid geometry).
 * op is DOE_OP_PROPAGATE, DOE_OP_PSF or DOE_OP_GRAD. */
size_t doe_workspace_bytes(const doe_geom* g, int op);

/* Destination field E_dest (Eq. 3) for every wavelength.
 *   h      device float [ny/f][nx/f]      heights in metres (Eq. 1); f = 1 unless DOE_UPSAMPLE
 *   e_in   device complex [ny][nx] or NULL incident field E_in (Eq. 2); NULL = unit plane wave
 *   e_out  device complex [n_lambda][P][P] written: E_dest on the padded grid
 * Errors: DOE_EINVAL (bad geometry / NULL h or e_out), DOE_EUNSUPPORTED (a side P outside the
 * grid notes above), DOE_ENOWS (workspace), DOE_ECUDA.  On a rectangular grid every [P][P] of
 * this header reads [Py][Px]. */
int doe_propagate(const doe_geom* g, const float* h, const float* e_in, float* e_out, void* ws,
                  size_t ws_bytes, void* stream);

/* PSF I = |E_dest|^2 (Sec. 3.1, after Eq. 4) for every wavelength.
 *   psf    device float [n_lambda][P][P] written; raw intensity of a unit-amplitude field,
 *          not normalised.
 * Other arguments and errors as doe_propagate. */
int doe_psf(const doe_geom* g, const float* h, const float* e_in, float* psf, void* ws,
            size_t ws_bytes, void* stream);

/* PSFs of several independent DOEs in one set of launches (the serving path batches
 * requests this way).  All geometries must share nx, ny and pad (hence P); dx, z, the
 * wavelengths and the heights may differ.  h[r], e_in[r] (NULL entries allowed) and psf[r]
 * are device pointers held in HOST arrays of length n_req; psf[r] receives
 * [geoms[r].n_lambda][P][P].  The total number of wavelengths must be <= 64.  Workspace:
 * doe_workspace_bytes_many(..., DOE_OP_PSF).  Errors as doe_psf. */
int doe_psf_many(int n_req, const doe_geom* geoms, const float* const* h, const float* const* e_in,
                 float* const* psf, void* ws, size_t ws_bytes, void* stream);
size_t doe_workspace_bytes_many(int n_req, const doe_geom* geoms, int op);

/* Gradient of Eq. 4's objective with respect to the heights, by the adjoint of the chain:
 *   g_out = 2 (I - T) E_dest (DOE_GRAD_L2_TARGET) or (dL/dI) E_dest (DOE_GRAD_VJP);
 *   g_pad = IFFT2( conj(H) FFT2(g_out) ); g_doe = g_pad on the DOE window;
 *   dL/dh = sum_lambda -2 k'_lambda Im(conj(g_doe) E_doe), k' = 2 pi (n - 1) / lambda.
 *   t_or_dldi  device float [n_lambda][P][P]: the target T or dL/dI
 *   grad_h     device float [ny/f][nx/f], overwritten (per metre of height, on the layout)
 *   loss_dev   device double[1] or NULL: receives sum (I - T)^2 in DOE_GRAD_L2_TARGET mode
 *              (summed in FP64 from FP32 per-row partials), 0 in DOE_GRAD_VJP mode
 *   recompute  1: the forward field is recomputed inside the call (no stored field);
 *              0: ws still holds the fields left by a doe_psf call with the same
 *              geometry, heights and e_in on the same workspace (a DOE_OP_GRAD-sized ws);
 *              the forward passes are then skipped.
 * Errors as doe_propagate; DOE_EINVAL for a bad mode. */
int doe_grad(const doe_geom* g, const float* h, const float* e_in, const float* t_or_dldi, int mode,
             float* grad_h, double* loss_dev, int recompute, void* ws, size_t ws_bytes, void* stream);

/* Image formation by PSF convolution, channel c with PSF c:
 *   k_c = psf_c cropped to H x W around the optical axis (rows Py/2 - H/2 .., cols Px/2 - W/2 ..),
 *         normalised to sum 1;
 *   out_c[y][x] = sum_{u,v} img_c[y + H/2 - u][x + W/2 - v] k_c[u][v], zero outside the image
 *   (linear convolution, "same" window), computed with 2H x 2W transforms.
 *   psf  device float [C][Py][Px];  img, out  device float [C][H][W]
 * H and W are powers of two with 16 <= H <= Py, 16 <= W <= Px, 2H <= 8192 and 2W <= 16384;
 * Py is even and Px a multiple of 4.
 * Workspace: doe_render_workspace_bytes(C, H, W).  Errors: DOE_EINVAL, DOE_EUNSUPPORTED,
 * DOE_ENOWS, DOE_ECUDA. */
int doe_render(int C, int H, int W, const float* psf, int Py, int Px, const float* img, float* out,
               void* ws, size_t ws_bytes, void* stream);
size_t doe_render_workspace_bytes(int C, int H, int W);

/* Wiener deconvolution with the simulated PSF (Eq. 9, the imaging application's
 * reconstruction): per channel c,
 *   out_c = real( IFFT2( conj(K_c) / (|K_c|^2 + gamma) * FFT2(y_c) ) ),
 * with K_c = FFT2 of the PSF crop of size H x W centred at (Py/2, Px/2), normalised to sum 1
 * and placed with its centre at the origin of the H x W grid (circular model, no padding);
 * FFT2 unnormalised, IFFT2 with 1 / (H W).
 *   psf  device float [C][Py][Px];  y (blurred images), out  device float [C][H][W]
 * H and W are powers of two with 32 <= H <= min(Py, 8192), 32 <= W <= min(Px, 16384); Py
 * even, Px a multiple of 4; gamma >= 0.  Workspace: doe_wiener_workspace_bytes(C, H, W).
 * Errors: DOE_EINVAL, DOE_EUNSUPPORTED, DOE_ENOWS, DOE_ECUDA. */
int doe_wiener(int C, int H, int W, const float* psf, int Py, int Px, const float* y, double gamma,
               float* out, void* ws, size_t ws_bytes, void* stream);
size_t doe_wiener_workspace_bytes(int C, int H, int W);

/* One step of the design optimiser: Adam (Kingma & Ba 2015; the optimiser of the paper's
 * designs, Sec. 3.2 and 5) on the heights with the gradient of doe_grad, then projection onto
 * the fabricable range [h_min, h_max]:
 *   m = beta1 m + (1 - beta1) g;  v = beta2 v + (1 - beta2) g^2;
 *   h = clamp(h - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps), h_min, h_max)
 *   h, m, v  device float [n], updated in place (m = v = 0 before step t = 1)
 *   grad     device float [n]
 * t >= 1 is the step number; 0 <= beta1, beta2 < 1, eps > 0, lr >= 0, h_min <= h_max.  The
 * caller schedules lr (the paper decays it with a cosine schedule).  Errors: DOE_EINVAL,
 * DOE_ECUDA. */
int doe_adam_step(float* h, const float* grad, float* m, float* v, long long n, double lr, double beta1,
                  double beta2, double eps, int t, double h_min, double h_max, void* stream);

/* Radially symmetric height map (Sec. 5.4, broadband imaging: radial symmetry enforced through a
 * 16th-order polynomial), read as an even polynomial in the normalised radius:
 *   h[i][j] = sum_{k < n_c} c[k] s^k,  s = ((i - n/2)^2 + (j - n/2)^2) / (n/2)^2 = (rho / R)^2,
 * R = n dx / 2 the half-aperture, the axis at sample (n/2, n/2).
 *   n      even, 16 .. 65536 (the side of the height array given to doe_grad: N, or
 *          N / f with DOE_UPSAMPLE)
 *   c      device float [n_c], 1 <= n_c <= 9 (degree 2 (n_c - 1) <= 16), metres
 *   h      device float [n][n], overwritten
 * Horner in double-float, rounded once to float.  Stream-ordered.  Errors: DOE_EINVAL,
 * DOE_ECUDA. */
int doe_radial_heights(int n, const float* c, int n_c, float* h, void* stream);

/* Bytes of workspace doe_radial_grad needs (0 when n_c is out of range). */
size_t doe_radial_workspace_bytes(int n_c);

/* Transpose of doe_radial_heights: c_grad[k] = sum_{i,j} grad_h[i][j] s^k, the coefficient
 * gradient from doe_grad's height gradient.  grad_h device float [n][n]; c_grad device float
 * [n_c], overwritten; ws device, 8-byte aligned, >= doe_radial_workspace_bytes(n_c).  Double-
 * float terms, FP64 partial sums combined in a fixed order (deterministic).  Errors:
 * DOE_EINVAL, DOE_ENOWS, DOE_ECUDA. */
int doe_radial_grad(int n, int n_c, const float* grad_h, float* c_grad, void* ws, size_t ws_bytes, void* stream);

/* Integer band logic of the transfer function, computed on the host exactly as the kernels
 * use it (for bit-exact checks).  For wavelength j: kmax[j] = the largest signed frequency
 * index kept per axis (ceil(f_lim / du) - 1 capped at P/2, with
 * f_lim = 1 / (lambda sqrt((2 du z)^2 + 1)), du = 1 / (P dx), Matsushima & Shimobaba 2009
 * as cited next to Eq. 3), and m_ev[j] = ceil(1 / (lambda du)^2), or with
 * DOE_BANDLIMIT_CIRCULAR min(that, ceil((f_lim / du)^2)): a sample (kt, lt) with
 * |kt|, |lt| <= kmax is kept iff kt^2 + lt^2 < m_ev.  Host arrays of n_lambda entries. */
int doe_band_limits(const doe_geom* g, int32_t* kmax, int64_t* m_ev);
/* Rectangular grids: kmax_x from Px, kmax_y from Py, and m_ev the bound of kt^2 B^2 + lt^2 A^2
 * of the rectangular-grid note (on square grids kmax_y = kmax_x and m_ev as above). */
int doe_band_limits_xy(const doe_geom* g, int32_t* kmax_x, int32_t* kmax_y, int64_t* m_ev);

/* Debug: writes the band mask the kernels apply for wavelength j (1 = H != 0) as device
 * uint8 [P][P] in FFT order, read back from the transfer table the kernels use. */
int doe_debug_band_mask(const doe_geom* g, int j, uint8_t* mask, void* ws, size_t ws_bytes,
                        void* stream);

/* doe_psf without a workspace, for callers that cannot allocate device memory (for example a
 * plugin inside an application that owns the device-memory budget and passes in only the
 * input and output buffers, or a loop that must never call cudaMalloc).  No counterpart in
 * the paper.  The scratch is a static device array of DOE_NOALLOC_SCRATCH_BYTES inside the
 * library, held by every GPU that loads the library until the process exits; the call
 * allocates nothing.  h, e_in, psf and the errors are as for doe_psf, plus DOE_ESCRATCH when
 * doe_workspace_bytes(g, DOE_OP_PSF) exceeds DOE_NOALLOC_SCRATCH_BYTES.  The first call on a
 * device, and the first after that device's context was re-created (cudaDeviceReset), looks
 * up the array's device address (make it before any stream capture).  All calls
 * share the one array: calls whose work overlaps on the GPU (different streams, or other
 * host threads) race on it and must be serialised by the caller. */
#define DOE_NOALLOC_SCRATCH_BYTES (32u << 20)
int doe_psf_noalloc(const doe_geom* g, const float* h, const float* e_in, float* psf, void* stream);

/* Tracing (optional).  doe_trace_enable(n) makes the library bracket each of the next n pass
 * launches with a pair of CUDA events recorded on the launching stream (n = 0 turns tracing
 * off); the events are host-side objects, no device memory is allocated.  doe_trace_read()
 * waits for the recorded events, writes up to max (pass id, device milliseconds) records in
 * launch order into the host arrays pass_ids / ms, clears them and returns how many it wrote
 * (or a negative DOE_E* code).  doe_pass_name() names a pass id.  doe_launch_count() returns
 * the number of kernels this library has launched in the process so far. */
int doe_trace_enable(int max_records);
int doe_trace_read(int max, int* pass_ids, float* ms);
const char* doe_pass_name(int id);
long long doe_launch_count(void);

/* Fault word of the kernels on the current device.  Kernels never trap: a bounded wait on an
 * asynchronous copy that runs out (DOE_FAULT_WAIT_TIMEOUT), or, in a library built with
 * DOE_DEBUG, an index found outside its buffer (DOE_FAULT_BOUNDS, the access is skipped),
 * sets a bit and the kernel runs to its end, so its results are then undefined.
 * doe_fault_status() synchronises the device, writes the OR of every kernel's bits since the
 * last call into *word (host memory) and clears them; DOE_ECUDA if the device cannot be read.
 * doe_debug_build() is 1 in a DOE_DEBUG build, else 0.  Not part of the paper: diagnostics. */
#define DOE_FAULT_WAIT_TIMEOUT 0x1u
#define DOE_FAULT_BOUNDS 0x2u
int doe_fault_status(uint32_t* word);
int doe_debug_build(void);

/* Check of the fault path of the bounded waits: launches one CTA on `stream` that announces 16
 * bytes of asynchronous copies on an mbarrier and issues none, so its wait gives up after
 * `polls` polls (1 <= polls <= 2^20; DOE_EINVAL otherwise) and sets DOE_FAULT_WAIT_TIMEOUT,
 * which the next doe_fault_status() reports.  Nothing faults and the context stays usable.
 * Not part of the paper: diagnostics. */
int doe_check_wait_timeout(uint32_t polls, void* stream);

/* Human-readable text for a status code. */
const char* doe_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* DOE_H */
