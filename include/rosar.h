/*
 * rosar.h -- C ABI of librosar, the GB300 (sm_103a) imaging path for rotating
 * synthetic aperture radar by sparse-aperture azimuth filtering
 * (arXiv 2309.08038, "Efficient Rotating Synthetic Aperture Radar Imaging via
 * Robust Sparse Array Synthesis").
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Array arguments are DEVICE pointers owned by the caller (cudaMalloc'd or
 *    torch CUDA tensors, contiguous, at least 8-byte aligned).  Structs passed
 *    by pointer (rosar_radar, rosar_scan) are HOST pointers read during the call.
 *  - Complex data is interleaved (re, im) float32: rosar_c32, the layout of
 *    torch.complex64 and cuFloatComplex.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued asynchronously; no entry point synchronises the device.
 *  - Argument errors are detected on the host, before any launch, and return
 *    ROSAR_ERR_INVALID_ARG / ROSAR_ERR_UNSUPPORTED.  A failed launch returns
 *    ROSAR_ERR_CUDA.  rosar_last_error() then holds a one-line explanation
 *    (per host thread).  Nothing here aborts, exits or traps, and no entry point
 *    allocates device memory: scratch space is passed in by the caller.
 *  - Sizes are int; every product of sizes must stay below 2^31 elements.
 *
 * Notation: n_az = pulses (phase centres) per rotation, the paper's N (Sec. II-A,
 * Eq. (1)); L = ADC samples per pulse = FFT length = range bins (the paper's M and
 * L, Sec. III-D); K = sparse taps; M_ap = dense aperture length in pulses.
 */
#ifndef ROSAR_H
#define ROSAR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ROSAR_API __attribute__((visibility("default")))
#else
#define ROSAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rosar_c32 {
    float re, im;
} rosar_c32;

typedef enum rosar_status {
    ROSAR_OK = 0,
    ROSAR_ERR_INVALID_ARG = 1,  /* null pointer, non-positive or inconsistent size */
    ROSAR_ERR_UNSUPPORTED = 2,  /* valid request outside this build's limits (e.g. L not 2^p in [8, 4096]) */
    ROSAR_ERR_CUDA = 3,         /* a CUDA call or kernel launch failed; see rosar_last_error() */
    ROSAR_ERR_TIMEOUT = 4       /* a bounded device-side wait gave up (batched form) */
} rosar_status;

/* FMCW radar on a rotating arm (Sec. II-A/B; Table "Parameters of the ROSAR System"). */
typedef struct rosar_radar {
    double fc_hz;           /* carrier frequency at the start of the ramp, fc (Eq. (6)) */
    double slope_hz_per_s;  /* chirp slope, the paper's K (Eq. (6)) */
    double t_sample_s;      /* ADC sampling interval t_s (Eq. (10)) */
    double t_start_s;       /* ramp start to first ADC sample, T_Start (Eq. (10)) */
    double r0_m;            /* rotation radius r (Sec. II-A) */
    double c_mps;           /* propagation speed; 0 selects 299792458 m/s */
} rosar_radar;

/* Human-readable name of a status code (static storage, never NULL). */
ROSAR_API const char *rosar_status_string(rosar_status status);

/* Detail of the most recent failure on the calling host thread ("" if none). */
ROSAR_API const char *rosar_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
ROSAR_API int rosar_version(void);

/*
 * Range compression of every pulse (Sec. III-D, Eq. (38)):
 *   S[l][n] = c_l * sum_{m<L} win[m] * raw[n][m] * exp(-j*2*pi*l*m/L),
 *   c_l = exp(+j*pi*l*(L-1)/L) if centred, else 1.
 * The centred form takes the DFT about the centre of the ADC window, so a
 * point target's peak carries the phase 2*k_mid*R_n with
 * k_mid = 2*pi*(fc + K*(T_Start + t_s*(L-1)/2))/c; centred = 0 is Eq. (38) verbatim.
 *   raw  [n_az][L] complex, pulse-major (fast time contiguous)         (in)
 *   win  [L] float window (e.g. symmetric Hann); NULL = rectangular    (in)
 *   S    [L][n_az] complex, range-major (azimuth contiguous)           (out)
 * Limits: n_az >= 1; L a power of two in [8, 4096].  raw and S must not overlap.
 */
ROSAR_API rosar_status rosar_range_compress(const rosar_c32 *raw, const float *win, int n_az, int L,
                                  int centred, rosar_c32 *S, void *stream);

/* rosar_range_compress of each scan of a stack in one launch:
 *   raw [n_scans][n_az][L] (in), S [n_scans][L][n_az] (out); 1 <= n_scans <= 65535. */
ROSAR_API rosar_status rosar_range_compress_scans(const rosar_c32 *raw, const float *win, int n_scans, int n_az,
                                                  int L, int centred, rosar_c32 *S, void *stream);

/*
 * Sparse-aperture azimuth matched filter, the FFT+SAS image of Sec. III-D,
 * Eq. (43) and Algorithm 2, with every tap of row r reading range bin r:
 *   out[r][theta] = sum_{k<K} w[r][k] * S[r][(theta + o[r][k]) mod n_az]
 * (w is the conjugate of the paper's weight, which Eq. (43) applies as w^H y).
 * Taps are accumulated in float32 in increasing k.
 *   S    [n_rng][n_az] complex, range-major                             (in)
 *   w    [n_rng][K] complex weights, one vector per range row            (in)
 *   o    int32 pulse offsets: [K] shared by all rows if o_row_stride == 0,
 *        else row r uses o[r*o_row_stride + k] (o_row_stride >= K).  Any
 *        int32 value is valid; the modulo is non-negative.                (in)
 *   out  [n_rng][n_az] complex image on the polar grid                  (out)
 * Limits: n_rng, n_az, K >= 1.  out must not overlap S, w or o.
 */
ROSAR_API rosar_status rosar_sparse_azimuth(const rosar_c32 *S, const rosar_c32 *w, const int32_t *o,
                                  int o_row_stride, int n_rng, int n_az, int K,
                                  rosar_c32 *out, void *stream);

/*
 * Range-compressed back-projection, the "FFT+BPA" comparison path (Sec. III-D after
 * Eq. (43), with w_BP = alpha_n exp(-j2kR_n); Eq. (14) with fast time summed by the FFT):
 *   out[r][theta] = sum_{d=-M_ap/2}^{M_ap-M_ap/2-1} alpha_n * exp(-j*2*k_mid*R_n) * S(R_n/dR, n),
 *   n = (theta + d) mod n_az,
 * for the pixel at distance R_r = r0 + r*dR from the rotation centre and angle
 * 2*pi*theta/n_az, dR = c/(2*K*t_s*L).  R_n is the distance from phase centre n
 * at radius r0 + pulse_dr[n] and angle 2*pi*n/n_az + pulse_dphi[n] (Eqs. (2), (37));
 * alpha_n = max(0, cos of the off-bore-sight angle) (Eqs. (3), (8), (15)), 1 when
 * R_n = 0.  S(x, n) is linear interpolation between bins floor(x) and floor(x)+1
 * (interp = 1) or the nearest bin floor(x + 0.5) (interp = 0, the paper's l*_n of
 * Eq. (40)); bins outside 0..L-1 read zero.  S must be the centred range compression.
 *   S           [L][n_az] complex                                         (in)
 *   radar       host pointer                                              (in)
 *   pulse_dphi  [n_az] float angle errors in radians, or NULL (all zero)  (in)
 *   pulse_dr    [n_az] float radius errors in metres, or NULL (all zero)  (in)
 *   out         [n_rng][n_az] complex, rows 0..n_rng-1                    (out)
 * Limits: 1 <= n_rng <= L; 1 <= M_ap <= n_az; L >= 2.
 */
ROSAR_API rosar_status rosar_bpa(const rosar_c32 *S, const rosar_radar *radar, const float *pulse_dphi,
                       const float *pulse_dr, int L, int n_rng, int n_az, int M_ap, int interp,
                       rosar_c32 *out, void *stream);

/*
 * Whole FFT+SAS image of one scan (Sec. III-D; Algorithm 2 with the range FFT):
 * rosar_range_compress(raw, win, centred = 1) into `workspace`, then
 * rosar_sparse_azimuth over all L range rows into `out`.
 *   raw        [n_az][L] complex                                          (in)
 *   win        [L] float or NULL                                          (in)
 *   w, o, o_row_stride: as rosar_sparse_azimuth with n_rng = L           (in)
 *   workspace  [L][n_az] complex scratch; holds S on return             (scratch)
 *   out        [L][n_az] complex image                                   (out)
 */
ROSAR_API rosar_status rosar_image(const rosar_c32 *raw, const float *win, const rosar_c32 *w,
                         const int32_t *o, int o_row_stride, int n_az, int L, int K,
                         rosar_c32 *workspace, rosar_c32 *out, void *stream);

/*
 * Range-migration-aware sparse azimuth filter: Eq. (43) with each tap reading the pulse's
 * own peak bin (Sec. III-D: the paper picks l*_n of Eq. (40) per pulse), here as a row offset
 * per (row, tap) computed from the weight design's geometry:
 *   out[r][theta] = sum_k w[r][k] * S[r + dl[r][k]][(theta + o_k) mod n_az],
 * rows outside 0 .. n_bins-1 reading zero.  dl = 0 everywhere is rosar_sparse_azimuth.
 *   S   [n_bins][n_az] complex (in); w [n_rng][K] (in); o as rosar_sparse_azimuth (in);
 *   dl  [n_rng][K] int32 row offsets, any value (in); out [n_rng][n_az] (out)
 */
ROSAR_API rosar_status rosar_sparse_azimuth_migrating(const rosar_c32 *S, int n_bins, const rosar_c32 *w,
                                                      const int32_t *o, int o_row_stride, const int32_t *dl,
                                                      int n_rng, int n_az, int K, rosar_c32 *out, void *stream);

/* rosar_image with range-migration-aware taps (rows of S: n_bins = n_rng = L). */
ROSAR_API rosar_status rosar_image_migrating(const rosar_c32 *raw, const float *win, const rosar_c32 *w,
                                             const int32_t *o, int o_row_stride, const int32_t *dl, int n_az, int L,
                                             int K, rosar_c32 *workspace, rosar_c32 *out, void *stream);

/*
 * rosar_image_fft with the raw cube and the image in HOST memory: on `stream` it copies
 * raw_host into raw_dev (cudaMemcpyAsync), runs rosar_image_fft into out_dev and copies
 * the image back into out_host.  The call returns once the work is enqueued; out_host holds
 * the image after the stream has been synchronised.  Host buffers should be page-locked
 * (cudaHostAlloc or registered) so the copies run asynchronously and overlap work on other
 * streams; pageable buffers work but make the copies synchronous.  A caller pipelines scans
 * by giving each call in flight its own stream and device buffers.  The paper has no
 * counterpart (it is the I/O of one imaging step).
 *   raw_host  [n_az][L] complex, host (in)     raw_dev   [n_az][L] device staging (scratch)
 *   win, H    as rosar_image_fft (device, in)  workspace [L][n_az] device (scratch)
 *   out_dev   [L][n_az] device (out: the image, as rosar_image_fft)
 *   out_host  [L][n_az] complex, host (out)
 * Errors: argument errors before anything is enqueued; a failed copy or launch returns
 * ROSAR_ERR_CUDA (work enqueued before it may still run).
 */
ROSAR_API rosar_status rosar_image_fft_host(const rosar_c32 *raw_host, const float *win, const rosar_c32 *H,
                                            int n_az, int L, rosar_c32 *raw_dev, rosar_c32 *workspace,
                                            rosar_c32 *out_dev, rosar_c32 *out_host, void *stream);

/* ------------------------------------------------------------------------
 * Time-domain comparison paths: the paper's "BPA" (Sec. II-C, Eq. (14)) and
 * "SAS" (Sec. III-A, Algorithm 2 with W_SA).  Both read the raw IF cube and
 * sum over taps k and fast-time samples m:
 *   out[r][theta] = sum_k c[r][k] * sum_m win[m] * exp(-j*2*pi*tau_k*K*t_s*(m - m_ref))
 *                                   * raw[(theta + o_k) mod n_az][m],
 * tau_k = 2*rho_k/c with rho_k the nominal slant range (Eq. (2)) from the phase
 * centre at radius r0 and angle 2*pi*(theta + o_k)/n_az to the pixel at
 * distance R_r = r0 + r*dR and angle 2*pi*theta/n_az, dR = c/(2*K*t_s*L).
 * Cost O(K*L) per pixel (the FFT+ forms cost O(K)); the per-(r, k) slant range
 * and two-way phase in FP64, the sums on the tensor cores with each operand
 * split into bf16 hi + lo parts (three products per term, FP32 accumulation:
 * within a few 1e-5 of FP32), taps summed in ascending offset order.  win may
 * be NULL (all ones, the paper's unwindowed sums).  Requires L a multiple of 16
 * and raw 16-byte aligned.  out must not overlap raw.
 * ------------------------------------------------------------------------ */

/*
 * Time-domain BPA (Eq. (14)): taps o_k = d = -M_ap/2 .. M_ap-M_ap/2-1 (all pulses
 * of the aperture), c = alpha_d * exp(-j*2*k*rho_d), alpha_d = max(0, cos of the
 * off-bore-sight angle) (Eqs. (3), (8), (15)), 1 when rho_d = 0; m_ref = 0,
 * k = 2*pi*(fc + K*T_start)/c.  (Evaluated referenced to the window centre with
 * k_mid, which is the same product.)  Nominal geometry only.
 *   raw   [n_az][L] complex, pulse-major                                   (in)
 *   win   [L] float or NULL                                                (in)
 *   radar host pointer                                                     (in)
 *   out   [n_rng][n_az] complex                                           (out)
 * Limits: n_rng >= 1; 1 <= M_ap <= n_az; 16 <= L <= 65536, L % 16 == 0.
 */
ROSAR_API rosar_status rosar_bpa_time(const rosar_c32 *raw, const float *win, const rosar_radar *radar, int n_az,
                                      int L, int n_rng, int M_ap, rosar_c32 *out, void *stream);

/*
 * Time-domain SAS (Algorithm 2): taps o_k and coefficients c = w[r][k] from the
 * caller (layout and offset rules as in rosar_sparse_azimuth: o shared [K] if
 * o_row_stride == 0, else per row; any int32 value, taken modulo n_az).  m_ref =
 * (L-1)/2 if centred (pairs with weights built with the wavenumber at the
 * window centre, as rosar_image's weights are), else 0 (W_SA verbatim, pairs
 * with weights built with k).
 *   raw [n_az][L] complex (in); win [L] float or NULL (in); w [n_rng][K] (in);
 *   out [n_rng][n_az] complex (out).
 * Limits: n_rng, K >= 1; 16 <= L <= 65536, L % 16 == 0; centred in {0, 1}.
 */
ROSAR_API rosar_status rosar_sas_time(const rosar_c32 *raw, const float *win, const rosar_c32 *w, const int32_t *o,
                                      int o_row_stride, const rosar_radar *radar, int n_az, int L, int n_rng, int K,
                                      int centred, rosar_c32 *out, void *stream);

/*
 * The time-domain forms with their B operand precomputed once per weight design (a "plan"):
 * B[tap][sample][row] = c * win[m] * exp(-j*pi*phi*(m - m_ref)), the coefficient, window and fast-time
 * phasor of Eq. (14) / Algorithm 2's W_SA, split into bf16 hi and lo parts.  It depends on the radar
 * geometry, the window and the weights, not on the raw cube, so a caller imaging many scans with one design
 * computes it once; each planned call then only streams the raw cube through the tensor cores.  Same sums
 * as rosar_bpa_time / rosar_sas_time (shared offsets), each sample's phasor taken directly instead of by
 * recurrence (float32 rounding differs).  The plan holds the taps in ascending offset order (with their
 * offsets), tiled as the tensor cores read them; the planned call sums the taps in that order, and taps whose
 * offsets lie within 120 pulses of each other share one staged window of raw pulses.
 *   rosar_time_domain_plan_bytes: size of a plan, 16384 * ceil(n_rng / 64) * K * (L / 16) + 8 * K bytes
 *     (rounded up to 16; K = M_ap for BPA).
 *   rosar_sas_time_plan / rosar_bpa_time_plan: write the plan (device, 16-byte aligned, >= the size above);
 *     arguments as rosar_sas_time (shared offsets o [K], any int32 values) / rosar_bpa_time.
 *   rosar_sas_time_planned / rosar_bpa_time_planned: the image from raw [n_az][L] (device, 16-byte aligned)
 *     with the plan (read only; n_az, L, n_rng and K as given to the plan call).  Limits as the unplanned
 *     calls, and ceil(n_rng / 64) <= 65535, K <= 65535.  The call cannot check a plan's contents or size: a
 *     plan not written by the matching plan call with these sizes gives an undefined image and may read past
 *     the plan's end (the caller owns the plan and keeps it alive until the call's stream has passed it).
 */
ROSAR_API size_t rosar_time_domain_plan_bytes(int n_rng, int L, int K);
ROSAR_API rosar_status rosar_sas_time_plan(const float *win, const rosar_c32 *w, const int32_t *o,
                                           const rosar_radar *radar, int n_az, int L, int n_rng, int K, int centred,
                                           void *plan, size_t plan_bytes, void *stream);
ROSAR_API rosar_status rosar_sas_time_planned(const rosar_c32 *raw, const void *plan, int n_az, int L, int n_rng,
                                              int K, rosar_c32 *out, void *stream);
ROSAR_API rosar_status rosar_bpa_time_plan(const float *win, const rosar_radar *radar, int n_az, int L, int n_rng,
                                           int M_ap, void *plan, size_t plan_bytes, void *stream);
ROSAR_API rosar_status rosar_bpa_time_planned(const rosar_c32 *raw, const void *plan, int n_az, int L, int n_rng,
                                              int M_ap, rosar_c32 *out, void *stream);

/* ------------------------------------------------------------------------
 * Frequency-domain form of the sparse azimuth filter.  Eq. (43) with a fixed
 * row is a circular convolution of S[r][.] with g_r, g_r[(-o_k) mod n_az] += w[r][k];
 * it equals IFFT(H_r * FFT(S[r][.])) with H_r = FFT(g_r)/n_az.  H depends only on
 * the weight design, so it is computed once (rosar_azimuth_plan) and reused for
 * every scan.  Results equal rosar_sparse_azimuth up to float32 rounding
 * (a different summation order); cost is O(log n_az) per pixel instead of O(K).
 * ------------------------------------------------------------------------ */

/* 1 if n_az = 2^a 3^b 5^c with 2 <= n_az <= 16384 (the sizes the FFT form handles), else 0. */
ROSAR_API int rosar_azimuth_fft_supported(int n_az);

/*
 *   w, o, o_row_stride, n_rng, n_az, K: as rosar_sparse_azimuth                (in)
 *   H    [n_rng][n_az] complex transfer functions FFT(g_r)/n_az, each row stored in
 *        the library's internal (digit-reversed) frequency order: an opaque table
 *        for rosar_sparse_azimuth_fft / rosar_image_fft.  H[r][0] is the DC term.  (out)
 * ROSAR_ERR_UNSUPPORTED if rosar_azimuth_fft_supported(n_az) is 0.
 */
ROSAR_API rosar_status rosar_azimuth_plan(const rosar_c32 *w, const int32_t *o, int o_row_stride, int n_rng,
                                          int n_az, int K, rosar_c32 *H, void *stream);

/*
 * out[r][.] = IFFT(H[r][.] * FFT(S[r][.])) for every row: rosar_sparse_azimuth with the
 * weights and offsets that produced H.
 *   S [n_rng][n_az] (in); H [n_rng][n_az] from rosar_azimuth_plan (in); out [n_rng][n_az] (out)
 */
ROSAR_API rosar_status rosar_sparse_azimuth_fft(const rosar_c32 *S, const rosar_c32 *H, int n_rng, int n_az,
                                                rosar_c32 *out, void *stream);

/* rosar_image with the frequency-domain azimuth filter: range compression into
 * `workspace`, then rosar_sparse_azimuth_fft over the L rows with H [L][n_az]. */
ROSAR_API rosar_status rosar_image_fft(const rosar_c32 *raw, const float *win, const rosar_c32 *H, int n_az, int L,
                                       rosar_c32 *workspace, rosar_c32 *out, void *stream);

/*
 * rosar_image_fft for a sequence of n_scans scans that share win and H (Eq. (38) then
 * Eq. (43) per scan, Sec. III-D): out[s] equals rosar_image_fft(raw[s]) bit for bit.
 * Where a pipelined plan exists for (L, n_az) (rosar_image_fft_scans_pipelined), the
 * launches overlap consecutive scans: one launch runs the azimuth rows of scan s-1 together
 * with the range compression of scan s, the two scans alternating between the halves of
 * the workspace; otherwise the scans run one after the other through rosar_image_fft.
 *   raw       [n_scans][n_az][L] complex, pulse-major (in)
 *   win, H    as rosar_image_fft (in)
 *   workspace [2][L][n_az] complex (scratch)
 *   out       [n_scans][L][n_az] complex (out)
 * Limits as rosar_image_fft; n_scans >= 1.  No argument may overlap another (except
 * win/H, which are read only).  Errors as rosar_image_fft.
 */
ROSAR_API rosar_status rosar_image_fft_scans(const rosar_c32 *raw, const float *win, const rosar_c32 *H, int n_scans,
                                             int n_az, int L, rosar_c32 *workspace, rosar_c32 *out, void *stream);

/* 1 if rosar_image_fft_scans overlaps consecutive scans for this (L, n_az), else 0. */
ROSAR_API int rosar_image_fft_scans_pipelined(int L, int n_az);

/*
 * The range-migration-aware filter of rosar_sparse_azimuth_migrating (Sec. III-D: each pulse's
 * peak bin l*_n of Eq. (40) inside Eq. (43)) in the azimuth-frequency domain.  Grouping row
 * r's taps by their row offset d = dl[r][k],
 *   out[r][.] = sum_d IFFT(H_d[r] * FFT(S[r+d][.])),   H_d[r] = FFT(g_{r,d}) / n_az,
 *   g_{r,d}[(-o_k) mod n_az] += w[r][k] over the taps with dl[r][k] = d,
 * rows r+d outside 0 .. n_bins-1 contributing nothing: the same sums as the gather form up
 * to float32 rounding, at the cost of the fixed-row FFT filter plus one product per plane.
 *
 * rosar_azimuth_plan_migrating: the n_d planes d = d_lo .. d_lo+n_d-1 of the weight design.
 *   w, o, o_row_stride, n_rng, n_az, K: as rosar_azimuth_plan                  (in)
 *   dl   [n_rng][K] int32 row offsets; taps whose dl lies outside [d_lo, d_lo+n_d) are in
 *        no plane, so the caller passes the full range of dl                    (in)
 *   H    [n_d][n_rng][n_az] complex, an opaque table as rosar_azimuth_plan's    (out)
 * Limits: 1 <= n_d <= 16; ROSAR_ERR_UNSUPPORTED if rosar_azimuth_fft_supported(n_az) is 0.
 */
ROSAR_API rosar_status rosar_azimuth_plan_migrating(const rosar_c32 *w, const int32_t *o, int o_row_stride,
                                                    const int32_t *dl, int d_lo, int n_d, int n_rng, int n_az, int K,
                                                    rosar_c32 *H, void *stream);

/*
 *   S         [n_bins][n_az] complex range-compressed rows (in)
 *   H         [n_d][n_rng][n_az] from rosar_azimuth_plan_migrating with the same d_lo, n_d (in)
 *   spectrum  [n_bins][n_az] complex: the rows' forward transforms              (scratch)
 *   out       [n_rng][n_az] complex image                                       (out)
 * Two launches: the forward transform of every row of S, then per output row the planes'
 * products and the inverse.  out and spectrum must not overlap S, H or each other.
 */
ROSAR_API rosar_status rosar_sparse_azimuth_migrating_fft(const rosar_c32 *S, int n_bins, const rosar_c32 *H, int d_lo,
                                                          int n_d, int n_rng, int n_az, rosar_c32 *spectrum,
                                                          rosar_c32 *out, void *stream);

/* rosar_image_migrating with the frequency-domain filter: range compression into workspace[0],
 * then rosar_sparse_azimuth_migrating_fft over the L rows with spectrum = workspace[1].
 *   workspace [2][L][n_az] complex (scratch); other arguments as above with n_bins = n_rng = L. */
ROSAR_API rosar_status rosar_image_migrating_fft(const rosar_c32 *raw, const float *win, const rosar_c32 *H, int d_lo,
                                                 int n_d, int n_az, int L, rosar_c32 *workspace, rosar_c32 *out,
                                                 void *stream);

/* ------------------------------------------------------------------------
 * Differentiable form: a stack of n_scans scans [n_scans][n_rng][n_az] that share
 * one weight set, a per-pulse phase correction eps [n_scans][n_az] applied to the
 * range-compressed data, and the adjoints that give the gradient of a real image
 * loss with respect to the weights, the phase corrections, S and the raw cube.
 *   forward:  S_t = S * exp(j*eps[n])  (rosar_phase_apply), then
 *             out[s][r][t] = sum_k w[r][k] * S_t[s][r][(t + o_k) mod n_az]  (rosar_sparse_azimuth_scans)
 * Gradients follow the conjugate-Wirtinger convention of torch: for a real loss and a
 * holomorphic linear map y = A x, grad_x = A^H grad_y; for the real eps, the ordinary
 * derivative.  Every reduction runs in a fixed order (bit-reproducible).
 * ------------------------------------------------------------------------ */

/* S_t[s][r][n] = S[s][r][n] * exp(j*eps[s][n]); S_t may equal S (in place). */
ROSAR_API rosar_status rosar_phase_apply(const rosar_c32 *S, const float *eps, int n_scans, int n_rng, int n_az,
                                         rosar_c32 *S_t, void *stream);

/* rosar_sparse_azimuth over each scan of the stack with the shared w [n_rng][K] and o. */
ROSAR_API rosar_status rosar_sparse_azimuth_scans(const rosar_c32 *S, const rosar_c32 *w, const int32_t *o,
                                                  int o_row_stride, int n_scans, int n_rng, int n_az, int K,
                                                  rosar_c32 *out, void *stream);

/*
 * Adjoint of Eq. (43) for the gradient g = d loss / d conj(out) [n_scans][n_rng][n_az]:
 *   grad_S_t[s][r][n] = sum_k conj(w[r][k]) * g[s][r][(n - o_k) mod n_az]        (NULL to skip)
 *   grad_w[r][k]      = sum_s sum_t g[s][r][t] * conj(S_t[s][r][(t + o_k) mod n_az])  (NULL to skip;
 *                       needs S_t, the forward's phase-corrected input)
 * grad_S_t is the transposed gather (conjugated weights, negated offsets); grad_w is a
 * per-(row, tap) reduction over scans and azimuth.
 */
ROSAR_API rosar_status rosar_sparse_azimuth_adjoint(const rosar_c32 *g, const rosar_c32 *S_t, const rosar_c32 *w,
                                                    const int32_t *o, int o_row_stride, int n_scans, int n_rng,
                                                    int n_az, int K, rosar_c32 *grad_S_t, rosar_c32 *grad_w,
                                                    void *stream);

/*
 * Frequency-domain form of the differentiable filter (Eq. (43) as a circular
 * convolution, as rosar_sparse_azimuth_fft), for a stack of scans sharing one plan:
 *   out[s][r][.] = IFFT(H[r] * FFT(S[s][r][.]))          (adjoint = 0: rosar_sparse_azimuth_scans)
 *   out[s][r][.] = IFFT(conj(H[r]) * FFT(S[s][r][.]))    (adjoint = 1: grad_S_t of rosar_sparse_azimuth_adjoint)
 *   S, out [n_scans][n_rng][n_az] (in, out); H [n_rng][n_az] from rosar_azimuth_plan (in).
 * Limits: n_az = 2^a 3^b 5^c <= 16384; out must not overlap S or H.
 */
ROSAR_API rosar_status rosar_sparse_azimuth_fft_scans(const rosar_c32 *S, const rosar_c32 *H, int n_scans, int n_rng,
                                                      int n_az, int adjoint, rosar_c32 *out, void *stream);

/*
 * grad_w of rosar_sparse_azimuth_adjoint through the cross-spectrum: per row r,
 *   corr_r[tau] = sum_s sum_t g[s][r][t] conj(S_t[s][r][(t + tau) mod n_az]) = DFT(sum_s G_s conj(S_s))[tau] / n_az,
 * with G_s, S_s the rows' transforms, then grad_w[r][k] = corr_r[o_k mod n_az].
 *   g, S_t [n_scans][n_rng][n_az] (in); o as rosar_sparse_azimuth (in); grad_w [n_rng][K] (out).
 * Limits: n_az = 2^a 3^b 5^c with three rows of n_az in 200 KB of shared memory (n_az <= 8400 or so).
 */
ROSAR_API rosar_status rosar_azimuth_weight_grad_fft(const rosar_c32 *g, const rosar_c32 *S_t, const int32_t *o,
                                                     int o_row_stride, int n_scans, int n_rng, int n_az, int K,
                                                     rosar_c32 *grad_w, void *stream);

/*
 * grad_eps[s][n] = sum_r Im(conj(S_t[s][r][n]) * grad_S_t[s][r][n])   (NULL to skip)
 * grad_S[s][r][n] = grad_S_t[s][r][n] * exp(-j*eps[s][n])             (NULL to skip; needs eps)
 */
ROSAR_API rosar_status rosar_phase_grad(const rosar_c32 *S_t, const rosar_c32 *grad_S_t, const float *eps,
                                        int n_scans, int n_rng, int n_az, float *grad_eps, rosar_c32 *grad_S,
                                        void *stream);

/*
 * The same step without the corrected copy S_t in memory: the phase factors P = exp(j*eps) are computed once
 * per (scan, pulse) and every kernel that reads S_t forms S * P as it loads S (same products, same results as
 * rosar_phase_apply followed by the calls above).
 *   rosar_phasors:        P[i] = exp(j*eps[i]) for i < n (eps float, P complex; n = n_scans * n_az).
 *   rosar_sparse_azimuth_fft_scans_ex: rosar_sparse_azimuth_fft_scans of S * P (P NULL: of S), and (spectrum
 *                         not NULL) the rows' forward transforms written to spectrum [n_scans][n_rng][n_az] in an
 *                         internal order (fixed per n_az), before the product with H or conj(H).
 *   rosar_azimuth_weight_grad_fft_phase: rosar_azimuth_weight_grad_fft with S_t = S * P.
 *   rosar_azimuth_weight_grad_spectra: the same gradient from stored transforms: G = the spectrum of the
 *                         adjoint call (g), X = the spectrum of the forward call (S * P); the cross-spectrum
 *                         sum_s G_s conj(X_s) (scan order) into workspace [n_rng][n_az] (scratch), then per row
 *                         one inverse transform: no forward transform repeated.
 *   rosar_phase_grad_phasor: rosar_phase_grad with S_t = S * P and grad_S = grad_S_t * conj(P).
 *   S [n_scans][n_rng][n_az], P [n_scans][n_az] (in); other arguments and limits as the calls above.
 */
ROSAR_API rosar_status rosar_phasors(const float *eps, long long n, rosar_c32 *P, void *stream);
ROSAR_API rosar_status rosar_sparse_azimuth_fft_scans_ex(const rosar_c32 *S, const rosar_c32 *P, const rosar_c32 *H,
                                                         int n_scans, int n_rng, int n_az, int adjoint, rosar_c32 *out,
                                                         rosar_c32 *spectrum, void *stream);
ROSAR_API rosar_status rosar_azimuth_weight_grad_fft_phase(const rosar_c32 *g, const rosar_c32 *S, const rosar_c32 *P,
                                                           const int32_t *o, int o_row_stride, int n_scans, int n_rng,
                                                           int n_az, int K, rosar_c32 *grad_w, void *stream);
ROSAR_API rosar_status rosar_azimuth_weight_grad_spectra(const rosar_c32 *G, const rosar_c32 *X, const int32_t *o,
                                                         int o_row_stride, int n_scans, int n_rng, int n_az, int K,
                                                         rosar_c32 *workspace, rosar_c32 *grad_w, void *stream);
ROSAR_API rosar_status rosar_phase_grad_phasor(const rosar_c32 *S, const rosar_c32 *P, const rosar_c32 *grad_S_t,
                                               int n_scans, int n_rng, int n_az, float *grad_eps, rosar_c32 *grad_S,
                                               void *stream);

/*
 * Image loss of the differentiable form: the squared L2 distance between an image stack and a reference
 * stack (e.g. back-projection images of the same scans), and its gradient in the same convention:
 *   loss    = sum_{i<n} |out[i] - ref[i]|^2                       (rosar_image_l2_loss)
 *   grad[i] = 2 * g * (out[i] - ref[i])                            (rosar_image_l2_loss_grad)
 * g is the upstream gradient of the loss (a device float).  The sum is deterministic: fixed contiguous chunks
 * (their number fixed by the library) summed in a fixed order, chunk sums added in double precision in
 * chunk order.  One read of both stacks per call.
 *   out, ref  [n] complex (in);  workspace rosar_image_l2_loss_workspace_bytes() bytes of device scratch;
 *   loss      device float (out);  grad [n] complex (out; may be out or ref itself, no partial overlap).
 * Errors: null pointers, n < 1, misaligned pointers -> ROSAR_ERR_INVALID_ARG before any launch.
 */
ROSAR_API size_t rosar_image_l2_loss_workspace_bytes(void);
ROSAR_API rosar_status rosar_image_l2_loss(const rosar_c32 *out, const rosar_c32 *ref, long long n, void *workspace,
                                           float *loss, void *stream);
ROSAR_API rosar_status rosar_image_l2_loss_grad(const rosar_c32 *out, const rosar_c32 *ref, long long n,
                                                const float *g, rosar_c32 *grad, void *stream);

/*
 * Adjoint of rosar_range_compress (Eq. (38) transposed):
 *   grad_raw[n][m] = win[m] * sum_l conj(c_l) * exp(+j*2*pi*l*m/L) * g[l][n]
 *   g [L][n_az] range-major (in); grad_raw [n_az][L] pulse-major (out).
 */
ROSAR_API rosar_status rosar_range_compress_adjoint(const rosar_c32 *g, const float *win, int n_az, int L,
                                                    int centred, rosar_c32 *grad_raw, void *stream);

/* rosar_range_compress_adjoint of each scan of a stack in one launch:
 *   g [n_scans][L][n_az] (in), grad_raw [n_scans][n_az][L] (out); 1 <= n_scans <= 65535. */
ROSAR_API rosar_status rosar_range_compress_adjoint_scans(const rosar_c32 *g, const float *win, int n_scans, int n_az,
                                                          int L, int centred, rosar_c32 *grad_raw, void *stream);

/* ------------------------------------------------------------------------
 * Batched form: many scans of uneven n_az, L and K imaged by ONE persistent
 * kernel launch, captured once in a CUDA graph.
 *
 * The persistent CTAs pull tiles from an atomic ticket counter: range tiles
 * (P pulses of one scan through the range FFT, as rosar_range_compress) and
 * azimuth tiles (one row segment of one scan through the gather-MAC filter, as
 * rosar_sparse_azimuth).  An azimuth tile waits, on the device, until every range
 * tile of its scan has completed.  Every range tile of a scan holds a smaller
 * ticket than any of its azimuth tiles, so the tiles a wait depends on are
 * already owned by running CTAs and the wait ends; it is nevertheless bounded
 * (spin_limit polls), after which the kernel records ROSAR_ERR_TIMEOUT and
 * every CTA returns.  Results equal rosar_image (or rosar_image_fft, for a scan
 * given its plan H) scan by scan, bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct rosar_scan {
    const rosar_c32 *raw;   /* [n_az][L] complex input                                  (in) */
    const float *win;       /* [L] window or NULL                                       (in) */
    const rosar_c32 *w;     /* [L][K] weights                                           (in) */
    const int32_t *o;       /* [K] shared offsets (o_row_stride 0) or rows of o_row_stride (in) */
    int o_row_stride;
    int n_az;               /* >= 1 */
    int L;                  /* power of two in [16, 2048] */
    int K;                  /* >= 1 */
    rosar_c32 *S;           /* [L][n_az] workspace: range-compressed data          (scratch) */
    rosar_c32 *out;         /* [L][n_az] image                                          (out) */
    const rosar_c32 *H;     /* [L][n_az] plan from rosar_azimuth_plan for this scan's w, o: its
                               azimuth filter runs as whole-row FFT tiles (as rosar_image_fft);
                               NULL: gather tiles (as rosar_image).  n_az must then satisfy
                               rosar_azimuth_fft_supported.                             (in) */
} rosar_scan;

typedef struct rosar_batch_tuning {
    int az_tile;            /* azimuth outputs per tile: 256, 512, 1024 or 2048; 0 selects 1024 */
    int ctas_per_sm;        /* persistent CTAs per SM; 0 or more than fit selects the occupancy limit */
    int interleave;         /* 0: every range tile first, then every azimuth tile; 1: scan by scan;
                               d in [2, 8]: range tiles run d-1 scans ahead of azimuth tiles */
    int spin_limit;         /* polls (~0.1 us apart) before a dependency wait gives up; 0 selects 2^24 */
    int debug_unmet_scan;   /* test hook, -1 = off: scan whose azimuth tiles wait for one range tile
                               more than exists, so that their wait must time out */
    int mix;                /* interleave >= 2: the range tiles of scan s+d-1 and the azimuth tiles of scan s
                               alternate in `mix` chunks each (1..32; 0 selects 1: one block each) */
    int flags;              /* ROSAR_BATCH_* bits, 0 = none */
} rosar_batch_tuning;

/* Whole-row FFT tiles drop each S row from L2 once they have read it, so range-compressed data that is
 * still cached is never written back to memory: the scans' S buffers (scratch) hold undefined values after
 * the launch. */
#define ROSAR_BATCH_DISCARD_S 2

typedef struct rosar_batch rosar_batch;   /* opaque host handle */

/* Device workspace the batch needs for its descriptors and counters. */
ROSAR_API size_t rosar_batch_workspace_bytes(int n_scans);

/* Validates the scans (host array, read during the call), writes the descriptors into
 * `workspace` (device, >= rosar_batch_workspace_bytes(n_scans), synchronous copy) and
 * captures [counter reset, persistent kernel] into a CUDA graph.  `tuning` may be NULL
 * (defaults).  The scans' buffers are bound at creation: later launches re-read them. */
ROSAR_API rosar_status rosar_batch_create(const rosar_scan *scans, int n_scans, const rosar_batch_tuning *tuning,
                                          void *workspace, size_t workspace_bytes, rosar_batch **batch);

/* Enqueues the graph (one cudaGraphLaunch) on `stream`. */
ROSAR_API rosar_status rosar_batch_launch(rosar_batch *batch, void *stream);

/* Waits for `stream`, then reports ROSAR_OK or ROSAR_ERR_TIMEOUT (a dependency wait gave up). */
ROSAR_API rosar_status rosar_batch_status(rosar_batch *batch, void *stream);

/* Number of tiles (range, azimuth), persistent CTAs and shared bytes per CTA; any pointer may be NULL. */
ROSAR_API rosar_status rosar_batch_info(const rosar_batch *batch, int *range_tiles, int *azimuth_tiles,
                                        int *ctas, int *smem_bytes);

/* Releases the graph and the host handle (not the caller's workspace). */
ROSAR_API rosar_status rosar_batch_destroy(rosar_batch *batch);

/*
 * rosar_image without a caller-provided workspace, for callers that cannot
 * allocate device memory: a plugin whose host passes in device buffers but no
 * allocator, or a real-time loop that may not call cudaMalloc after start-up
 * (it can stall the whole device).  The paper has no counterpart; this is a
 * deployment convenience with the same result as rosar_image.
 *   raw, win, w, o, o_row_stride, n_az, L, K, out: as rosar_image.
 * The range-compressed intermediate lives in a fixed array inside the library
 * (ROSAR_NOALLOC_MAX_ELEMS complex elements = 16 MiB, held on every GPU that
 * loads the library until the process exits); L*n_az beyond that returns
 * ROSAR_ERR_UNSUPPORTED.  The first call on each device looks up the array's
 * device address, so make it before any stream capture.  Every call shares the
 * array: calls that overlap on the GPU race and must be serialised.  Nothing
 * is allocated, by this library or any library it calls.
 */
#define ROSAR_NOALLOC_MAX_ELEMS (1 << 21)
ROSAR_API rosar_status rosar_image_noalloc(const rosar_c32 *raw, const float *win, const rosar_c32 *w,
                                           const int32_t *o, int o_row_stride, int n_az, int L, int K,
                                           rosar_c32 *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ROSAR_H */
