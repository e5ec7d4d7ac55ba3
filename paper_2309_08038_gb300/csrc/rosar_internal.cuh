// Internal helpers shared by the librosar translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rosar.h"

namespace rosar {

// Records a one-line error message for rosar_last_error() and returns `st`.
rosar_status set_error(rosar_status st, const char *fmt, ...);

// Clears the message (called at entry of every API function).
void clear_error();

// Maps the launch status of the calling thread to ROSAR_OK / ROSAR_ERR_CUDA.
rosar_status check_launch(const char *what);

static inline bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the current device.
// `limits` is a per-kernel array of kMaxDevices ints holding the limit set so far per device.
constexpr int kMaxDevices = 64;
rosar_status ensure_smem(const void *func, size_t bytes, int *limits, const char *what);

// ------------------------------------------------------------ complex ops --

// Complex add and subtract, and a real multiple of a complex added to another, each as ONE packed FP32x2
// instruction (sm_100 and later): per lane the same IEEE round-to-nearest result as the scalar expression,
// in half the issue slots of two scalar instructions.  The transforms are issue-bound, and most of a
// butterfly's arithmetic is these three forms.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// a + s*b for real s (one rounding per lane, as fmaf(s, b.x, a.x), fmaf(s, b.y, a.y))
__device__ __forceinline__ float2 caxpy(float s, float2 b, float2 a) { return __ffma2_rn(make_float2(s, s), b, a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// acc += a * b, in the order re: a.x*b.x - a.y*b.y, im: a.x*b.y + a.y*b.x
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may start
// before its predecessor in the stream has finished; griddep_wait() blocks until that predecessor has
// completed and its memory is visible, griddep_launch_dependents() lets the successor start early.
// Both are no-ops when no such launch relation exists.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Non-negative modulo for any int32 value and n >= 1.
__device__ __forceinline__ int pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------- launchers --
// Each .cu file exposes a host-side launcher; the API layer validates first.

rosar_status launch_range_compress(const float2 *raw, const float *win, int n_az, int L, int centred,
                                   float2 *S, cudaStream_t s, int n_scans = 1);

rosar_status launch_sparse_azimuth(const float2 *S, const float2 *w, const int32_t *o, int o_row_stride,
                                   int n_rng, int n_az, int K, float2 *out, cudaStream_t s);

// Range-migration-aware taps: tap k of row r reads row r + dl[r][k] of S (n_bins rows).
rosar_status launch_sparse_azimuth_migrating(const float2 *S, int n_bins, const float2 *w, const int32_t *o,
                                             int o_row_stride, const int32_t *dl, int n_rng, int n_az, int K,
                                             float2 *out, cudaStream_t s);

// Stacked scans [n_scans][n_rng][n_az] sharing w and o; adjoint = conjugated weights, negated offsets.
rosar_status launch_sparse_azimuth_scans(const float2 *S, const float2 *w, const int32_t *o, int o_row_stride,
                                         int n_scans, int n_rng, int n_az, int K, bool adjoint, float2 *out,
                                         cudaStream_t s);

// Differentiable form (diff.cu, range_compress.cu).
rosar_status launch_phase_apply(const float2 *S, const float *eps, int n_scans, int n_rng, int n_az, float2 *S_t,
                                cudaStream_t s);
rosar_status launch_azimuth_weight_grad(const float2 *g, const float2 *S_t, const int32_t *o, int o_row_stride,
                                        int n_scans, int n_rng, int n_az, int K, float2 *grad_w, cudaStream_t s);
rosar_status launch_phase_grad(const float2 *S_t, const float2 *G, const float *eps, int n_scans, int n_rng, int n_az,
                               float *grad_eps, float2 *grad_S, cudaStream_t s);
// The same with S uncorrected and the phase factors P = e^{j eps} [n_scans][n_az] given: S_t = S P is formed at load.
rosar_status launch_phase_grad_phasor(const float2 *S, const float2 *P, const float2 *G, int n_scans, int n_rng,
                                      int n_az, float *grad_eps, float2 *grad_S, cudaStream_t s);
rosar_status launch_phasors(const float *eps, long long n, float2 *P, cudaStream_t s);
rosar_status launch_range_compress_adjoint(const float2 *g, const float *win, int n_az, int L, int centred,
                                           float2 *grad_raw, cudaStream_t s, int n_scans = 1);

// Azimuth filter in the frequency domain (azimuth_fft.cu).
int azimuth_fft_supported(int n_az);

// Image loss of the differentiable form (image_loss.cu): partial sums per call = image_loss_partials().
int image_loss_partials();
rosar_status launch_image_l2_loss(const float2 *out, const float2 *ref, long long n, double *partial, float *loss,
                                  cudaStream_t s);
rosar_status launch_image_l2_loss_grad(const float2 *out, const float2 *ref, long long n, const float *g,
                                       float2 *grad, cudaStream_t s);

// Pipelined multi-scan imaging (image_pipeline.cu): 1 if a stage kernel exists for (L, n_az).
int image_pipeline_supported(int L, int n_az);
rosar_status launch_image_pipeline(const float2 *raw, const float *win, const float2 *H, int n_scans, int n_az, int L,
                                   float2 *workspace, float2 *out, cudaStream_t s);
// overlap_predecessor: launch with programmatic stream serialization (only when the preceding kernel in
// the stream writes S and nothing else the kernel reads before its grid-dependency wait, i.e. H).
// h_rows: row b of S uses row (b mod h_rows) of H (0 = n_rng: one plan row per S row); conj_h: filter with conj(H),
// the adjoint of the filter.
// phase (optional): [n_rng / h_rows][n_az] factors applied to the rows of S as they are loaded; spec (optional):
// [n_rng][n_az] receives the rows' forward transforms (digit-reversed, before the product with H).
rosar_status launch_azimuth_fft(const float2 *S, const float2 *H, int n_rng, int n_az, float2 *out, cudaStream_t s,
                                bool overlap_predecessor = false, int h_rows = 0, bool conj_h = false,
                                const float2 *phase = nullptr, float2 *spec = nullptr);
// grad_w from the rows' stored transforms G (image gradient) and X (corrected S), [n_scans][n_rng][n_az] each;
// P [n_rng][n_az] scratch for the cross-spectrum.
rosar_status launch_azimuth_weight_grad_spectra(const float2 *G, const float2 *X, const int32_t *o, int o_row_stride,
                                                int n_scans, int n_rng, int n_az, int K, float2 *P, float2 *grad_w,
                                                cudaStream_t s);
// grad_w[r][k] = sum_s sum_t g[s][r][t] conj(S_t[s][r][(t + o_k) mod n_az]) from the per-row cross-spectrum.
// phase (optional): S_t = S_t[s] * phase[s] per column (the phase-corrected rows computed at load).
rosar_status launch_azimuth_weight_grad_fft(const float2 *g, const float2 *S_t, const int32_t *o, int o_row_stride,
                                            int n_scans, int n_rng, int n_az, int K, float2 *grad_w, cudaStream_t s,
                                            const float2 *phase = nullptr);
// dl != nullptr: the n_d planes of the range-migration-aware plan, plane i from the taps with dl = d_lo + i,
// H [n_d][n_rng][n_az].
rosar_status launch_azimuth_plan(const float2 *w, const int32_t *o, int o_row_stride, int n_rng, int n_az, int K,
                                 float2 *H, cudaStream_t s, const int32_t *dl = nullptr, int d_lo = 0, int n_d = 1);
// Range-migration-aware filter in the frequency domain (azimuth_mig_fft.cu): X [n_bins][n_az] scratch.
rosar_status launch_sparse_azimuth_migrating_fft(const float2 *S, int n_bins, const float2 *H, int d_lo, int n_d,
                                                 int n_rng, int n_az, float2 *X, float2 *out, cudaStream_t s);

struct BpaParams {
    float inv_dR;        // 1/dR, bins per metre
    float two_f_over_c;  // 2*f_mid/c, cycles of two-way phase per metre
    double two_f_over_c_d;
    double dR;
    double r0;
};

// Time-domain BPA / SAS (time_domain.cu).  phi_scale = 2/(dR*L): half-turns of fast-time phase per
// sample per metre of slant range; two_f_over_c = 2*f_mid/c; m_ref = fast-time phase reference sample.
struct TdParams {
    double dR;
    double r0;
    double two_f_over_c;
    double phi_scale;
    float m_ref;
    int n_az;
    int L;
    int n_rng;
};
int time_domain_sample_multiple();
rosar_status launch_time_domain(const float2 *raw, const float *win, const float2 *w, const int32_t *o,
                                int o_row_stride, const TdParams &p, int K, bool bpa, float2 *out, cudaStream_t s);
// The precomputed B operand of the tensor-core form (shared offsets; taps sorted by offset, the sorted offsets kept
// in the plan): plan bytes, the plan kernels, the planned call.
size_t time_domain_plan_bytes(int n_rng, int L, int K);
rosar_status launch_time_domain_plan(const float *win, const float2 *w, const int32_t *o, const TdParams &p, int K,
                                     bool bpa, void *plan, cudaStream_t s);
rosar_status launch_time_domain_planned(const float2 *raw, const TdParams &p, int K, bool bpa, const void *plan,
                                        float2 *out, cudaStream_t s);

rosar_status launch_bpa(const float2 *S, const BpaParams &p, const float *dphi, const float *dr, int L, int n_rng,
                        int n_az, int M_ap, int interp, float2 *out, cudaStream_t s);

}  // namespace rosar
