// C ABI of librosar: argument validation, error reporting and dispatch to the kernels.
// Every check here runs on the host before any launch; nothing synchronises the device.

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "rosar_internal.cuh"

namespace rosar {

static thread_local char g_msg[512];

rosar_status set_error(rosar_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_msg[0] = '\0'; }

rosar_status check_launch(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
    return ROSAR_OK;
}

rosar_status ensure_smem(const void *func, size_t bytes, int *limits, const char *what) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "%s: cudaGetDevice: %s", what, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(ROSAR_ERR_UNSUPPORTED, "%s: device ordinal %d", what, dev);
    if ((size_t)__atomic_load_n(limits + dev, __ATOMIC_ACQUIRE) >= bytes) return ROSAR_OK;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess)
        return set_error(ROSAR_ERR_CUDA, "%s: cudaFuncSetAttribute(%zu B): %s", what, bytes, cudaGetErrorString(e));
    int cur = __atomic_load_n(limits + dev, __ATOMIC_ACQUIRE);
    while (cur < (int)bytes && !__atomic_compare_exchange_n(limits + dev, &cur, (int)bytes, false, __ATOMIC_ACQ_REL,
                                                            __ATOMIC_ACQUIRE)) {
    }
    return ROSAR_OK;
}

namespace {

bool misaligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) != 0; }

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

constexpr long long kMaxElems = (1LL << 31) - 1;

rosar_status check_range_args(const void *raw, const float *win, int n_az, int L, const void *S) {
    if (!raw || !S) return set_error(ROSAR_ERR_INVALID_ARG, "range_compress: null raw or S");
    if (n_az < 1) return set_error(ROSAR_ERR_INVALID_ARG, "range_compress: n_az=%d < 1", n_az);
    if (!is_pow2(L) || L < 8 || L > 4096)
        return set_error(ROSAR_ERR_UNSUPPORTED, "range_compress: L=%d is not a power of two in [8, 4096]", L);
    if ((long long)n_az * L > kMaxElems) return set_error(ROSAR_ERR_UNSUPPORTED, "range_compress: n_az*L too large");
    if (misaligned(raw, 8) || misaligned(S, 8) || (win && misaligned(win, 4)))
        return set_error(ROSAR_ERR_INVALID_ARG, "range_compress: misaligned pointer");
    const size_t bytes = sizeof(rosar_c32) * (size_t)n_az * L;
    if (overlaps(raw, bytes, S, bytes)) return set_error(ROSAR_ERR_INVALID_ARG, "range_compress: raw and S overlap");
    return ROSAR_OK;
}

rosar_status check_azimuth_args(const void *S, const void *w, const int32_t *o, int o_row_stride, int n_rng, int n_az,
                                int K, const void *out) {
    if (!S || !w || !o || !out) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth: null pointer argument");
    if (n_rng < 1 || n_az < 1 || K < 1)
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth: sizes must be >= 1 (n_rng=%d n_az=%d K=%d)", n_rng,
                         n_az, K);
    if (o_row_stride != 0 && o_row_stride < K)
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth: o_row_stride=%d < K=%d", o_row_stride, K);
    if ((long long)n_rng * n_az > kMaxElems || (long long)n_rng * K > kMaxElems ||
        (long long)n_rng * o_row_stride > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth: array too large");
    if (misaligned(S, 8) || misaligned(w, 8) || misaligned(o, 4) || misaligned(out, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth: misaligned pointer");
    const size_t img = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    const size_t ob = sizeof(int32_t) * (o_row_stride ? (size_t)(n_rng - 1) * o_row_stride + K : (size_t)K);
    if (overlaps(out, img, S, img) || overlaps(out, img, w, sizeof(rosar_c32) * (size_t)n_rng * K) ||
        overlaps(out, img, o, ob))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth: out overlaps an input");
    return ROSAR_OK;
}

}  // namespace
}  // namespace rosar

using namespace rosar;

extern "C" {

const char *rosar_status_string(rosar_status status) {
    switch (status) {
        case ROSAR_OK: return "ROSAR_OK";
        case ROSAR_ERR_INVALID_ARG: return "ROSAR_ERR_INVALID_ARG";
        case ROSAR_ERR_UNSUPPORTED: return "ROSAR_ERR_UNSUPPORTED";
        case ROSAR_ERR_CUDA: return "ROSAR_ERR_CUDA";
        case ROSAR_ERR_TIMEOUT: return "ROSAR_ERR_TIMEOUT";
        default: return "ROSAR_ERR_UNKNOWN";
    }
}

const char *rosar_last_error(void) { return g_msg; }

int rosar_version(void) { return 100; }

rosar_status rosar_range_compress(const rosar_c32 *raw, const float *win, int n_az, int L, int centred, rosar_c32 *S,
                                  void *stream) {
    clear_error();
    rosar_status st = check_range_args(raw, win, n_az, L, S);
    if (st != ROSAR_OK) return st;
    return launch_range_compress(reinterpret_cast<const float2 *>(raw), win, n_az, L, centred,
                                 reinterpret_cast<float2 *>(S), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_range_compress_scans(const rosar_c32 *raw, const float *win, int n_scans, int n_az, int L,
                                        int centred, rosar_c32 *S, void *stream) {
    clear_error();
    if (n_scans < 1 || n_scans > 65535)
        return set_error(ROSAR_ERR_INVALID_ARG, "range_compress_scans: n_scans=%d not in [1, 65535]", n_scans);
    rosar_status st = check_range_args(raw, win, n_az, L, S);
    if (st != ROSAR_OK) return st;
    const size_t all = sizeof(rosar_c32) * (size_t)n_az * L * n_scans;
    if (overlaps(raw, all, S, all)) return set_error(ROSAR_ERR_INVALID_ARG, "range_compress_scans: raw and S overlap");
    return launch_range_compress(reinterpret_cast<const float2 *>(raw), win, n_az, L, centred,
                                 reinterpret_cast<float2 *>(S), static_cast<cudaStream_t>(stream), n_scans);
}

rosar_status rosar_sparse_azimuth(const rosar_c32 *S, const rosar_c32 *w, const int32_t *o, int o_row_stride,
                                  int n_rng, int n_az, int K, rosar_c32 *out, void *stream) {
    clear_error();
    rosar_status st = check_azimuth_args(S, w, o, o_row_stride, n_rng, n_az, K, out);
    if (st != ROSAR_OK) return st;
    return launch_sparse_azimuth(reinterpret_cast<const float2 *>(S), reinterpret_cast<const float2 *>(w), o,
                                 o_row_stride, n_rng, n_az, K, reinterpret_cast<float2 *>(out),
                                 static_cast<cudaStream_t>(stream));
}

rosar_status rosar_bpa(const rosar_c32 *S, const rosar_radar *radar, const float *pulse_dphi, const float *pulse_dr,
                       int L, int n_rng, int n_az, int M_ap, int interp, rosar_c32 *out, void *stream) {
    clear_error();
    if (!S || !radar || !out) return set_error(ROSAR_ERR_INVALID_ARG, "bpa: null S, radar or out");
    if (L < 2 || n_rng < 1 || n_rng > L || n_az < 1 || M_ap < 1 || M_ap > n_az)
        return set_error(ROSAR_ERR_INVALID_ARG, "bpa: need 1<=n_rng<=L, L>=2, 1<=M_ap<=n_az (L=%d n_rng=%d n_az=%d M_ap=%d)",
                         L, n_rng, n_az, M_ap);
    if ((long long)L * n_az > kMaxElems) return set_error(ROSAR_ERR_UNSUPPORTED, "bpa: L*n_az too large");
    if (interp != 0 && interp != 1) return set_error(ROSAR_ERR_INVALID_ARG, "bpa: interp must be 0 or 1");
    if (misaligned(S, 8) || misaligned(out, 8) || (pulse_dphi && misaligned(pulse_dphi, 4)) ||
        (pulse_dr && misaligned(pulse_dr, 4)))
        return set_error(ROSAR_ERR_INVALID_ARG, "bpa: misaligned pointer");
    const double c = radar->c_mps > 0 ? radar->c_mps : 299792458.0;
    if (!(radar->slope_hz_per_s > 0) || !(radar->t_sample_s > 0) || !(radar->r0_m >= 0) || !(radar->fc_hz > 0))
        return set_error(ROSAR_ERR_INVALID_ARG, "bpa: radar parameters must be positive");
    const size_t img = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    if (overlaps(out, img, S, sizeof(rosar_c32) * (size_t)L * n_az))
        return set_error(ROSAR_ERR_INVALID_ARG, "bpa: out overlaps S");
    BpaParams p;
    p.dR = c / (2.0 * radar->slope_hz_per_s * radar->t_sample_s * L);
    const double f_mid = radar->fc_hz + radar->slope_hz_per_s * (radar->t_start_s + radar->t_sample_s * (L - 1) / 2.0);
    p.two_f_over_c_d = 2.0 * f_mid / c;
    p.two_f_over_c = (float)p.two_f_over_c_d;
    p.inv_dR = (float)(1.0 / p.dR);
    p.r0 = radar->r0_m;
    return launch_bpa(reinterpret_cast<const float2 *>(S), p, pulse_dphi, pulse_dr, L, n_rng, n_az, M_ap, interp,
                      reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream));
}

namespace {

rosar_status time_domain_params(const char *what, const rosar_c32 *raw, const rosar_radar *radar, int n_az, int L,
                                int n_rng, int K, bool centred, const rosar_c32 *out, TdParams *p) {
    if (!raw || !radar || !out) return set_error(ROSAR_ERR_INVALID_ARG, "%s: null raw, radar or out", what);
    if (n_az < 1 || n_rng < 1 || K < 1 || L < 16 || L > 65536)
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: need n_az, n_rng, K >= 1 and 16 <= L <= 65536 (n_az=%d L=%d "
                         "n_rng=%d K=%d)", what, n_az, L, n_rng, K);
    if (L % time_domain_sample_multiple() != 0)
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: L=%d is not a multiple of %d", what, L,
                         time_domain_sample_multiple());
    if ((long long)n_az * L > kMaxElems || (long long)n_rng * n_az > kMaxElems || (long long)n_rng * K > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: sizes too large", what);
    if (misaligned(raw, 16) || misaligned(out, 8)) return set_error(ROSAR_ERR_INVALID_ARG, "%s: misaligned pointer", what);
    const double c = radar->c_mps > 0 ? radar->c_mps : 299792458.0;
    if (!(radar->slope_hz_per_s > 0) || !(radar->t_sample_s > 0) || !(radar->r0_m >= 0) || !(radar->fc_hz > 0))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: radar parameters must be positive", what);
    if (overlaps(out, sizeof(rosar_c32) * (size_t)n_rng * n_az, raw, sizeof(rosar_c32) * (size_t)n_az * L))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: out overlaps raw", what);
    p->dR = c / (2.0 * radar->slope_hz_per_s * radar->t_sample_s * L);
    const double f_mid = radar->fc_hz + radar->slope_hz_per_s * (radar->t_start_s + radar->t_sample_s * (L - 1) / 2.0);
    p->two_f_over_c = 2.0 * f_mid / c;
    p->phi_scale = 2.0 / (p->dR * L);
    p->r0 = radar->r0_m;
    p->m_ref = centred ? 0.5f * (float)(L - 1) : 0.f;
    p->n_az = n_az;
    p->L = L;
    p->n_rng = n_rng;
    return ROSAR_OK;
}

}  // namespace

rosar_status rosar_bpa_time(const rosar_c32 *raw, const float *win, const rosar_radar *radar, int n_az, int L,
                            int n_rng, int M_ap, rosar_c32 *out, void *stream) {
    clear_error();
    TdParams p;
    rosar_status st = time_domain_params("bpa_time", raw, radar, n_az, L, n_rng, M_ap, true, out, &p);
    if (st != ROSAR_OK) return st;
    if (M_ap > n_az) return set_error(ROSAR_ERR_INVALID_ARG, "bpa_time: M_ap=%d exceeds n_az=%d", M_ap, n_az);
    if (win && misaligned(win, 4)) return set_error(ROSAR_ERR_INVALID_ARG, "bpa_time: misaligned win");
    return launch_time_domain(reinterpret_cast<const float2 *>(raw), win, nullptr, nullptr, 0, p, M_ap, true,
                              reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_sas_time(const rosar_c32 *raw, const float *win, const rosar_c32 *w, const int32_t *o,
                            int o_row_stride, const rosar_radar *radar, int n_az, int L, int n_rng, int K, int centred,
                            rosar_c32 *out, void *stream) {
    clear_error();
    if (centred != 0 && centred != 1) return set_error(ROSAR_ERR_INVALID_ARG, "sas_time: centred must be 0 or 1");
    TdParams p;
    rosar_status st = time_domain_params("sas_time", raw, radar, n_az, L, n_rng, K, centred == 1, out, &p);
    if (st != ROSAR_OK) return st;
    if (!w || !o) return set_error(ROSAR_ERR_INVALID_ARG, "sas_time: null w or o");
    if (o_row_stride != 0 && o_row_stride < K)
        return set_error(ROSAR_ERR_INVALID_ARG, "sas_time: o_row_stride=%d must be 0 or >= K=%d", o_row_stride, K);
    if ((long long)n_rng * o_row_stride > kMaxElems) return set_error(ROSAR_ERR_UNSUPPORTED, "sas_time: o too large");
    if (misaligned(w, 8) || misaligned(o, 4) || (win && misaligned(win, 4)))
        return set_error(ROSAR_ERR_INVALID_ARG, "sas_time: misaligned pointer");
    const size_t img = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    const size_t ob = sizeof(int32_t) * (o_row_stride ? (size_t)(n_rng - 1) * o_row_stride + K : (size_t)K);
    if (overlaps(out, img, w, sizeof(rosar_c32) * (size_t)n_rng * K) || overlaps(out, img, o, ob))
        return set_error(ROSAR_ERR_INVALID_ARG, "sas_time: out overlaps w or o");
    return launch_time_domain(reinterpret_cast<const float2 *>(raw), win, reinterpret_cast<const float2 *>(w), o,
                              o_row_stride, p, K, false, reinterpret_cast<float2 *>(out),
                              static_cast<cudaStream_t>(stream));
}

size_t rosar_time_domain_plan_bytes(int n_rng, int L, int K) {
    if (n_rng < 1 || L < 1 || K < 1) return 0;
    return time_domain_plan_bytes(n_rng, L, K);
}

namespace {
// Geometry of a plan call (the plan kernel reads no raw cube): the checks of time_domain_params without raw/out.
rosar_status plan_params(const char *what, const rosar_radar *radar, int n_az, int L, int n_rng, int K, bool centred,
                         const void *plan, size_t plan_bytes, TdParams *p) {
    if (!radar || !plan) return set_error(ROSAR_ERR_INVALID_ARG, "%s: null radar or plan", what);
    if (n_az < 1 || n_rng < 1 || K < 1 || L < 16 || L > 65536)
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: need n_az, n_rng, K >= 1 and 16 <= L <= 65536", what);
    if (L % time_domain_sample_multiple() != 0)
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: L=%d is not a multiple of %d", what, L, time_domain_sample_multiple());
    if ((long long)n_rng * K > kMaxElems || (long long)n_rng * n_az > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: sizes too large", what);
    if (plan_bytes < time_domain_plan_bytes(n_rng, L, K))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: plan of %zu bytes < %zu needed", what, plan_bytes,
                         time_domain_plan_bytes(n_rng, L, K));
    if (misaligned(plan, 16)) return set_error(ROSAR_ERR_INVALID_ARG, "%s: plan must be 16-byte aligned", what);
    const double c = radar->c_mps > 0 ? radar->c_mps : 299792458.0;
    if (!(radar->slope_hz_per_s > 0) || !(radar->t_sample_s > 0) || !(radar->r0_m >= 0) || !(radar->fc_hz > 0))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: radar parameters must be positive", what);
    p->dR = c / (2.0 * radar->slope_hz_per_s * radar->t_sample_s * L);
    const double f_mid = radar->fc_hz + radar->slope_hz_per_s * (radar->t_start_s + radar->t_sample_s * (L - 1) / 2.0);
    p->two_f_over_c = 2.0 * f_mid / c;
    p->phi_scale = 2.0 / (p->dR * L);
    p->r0 = radar->r0_m;
    p->m_ref = centred ? 0.5f * (float)(L - 1) : 0.f;
    p->n_az = n_az;
    p->L = L;
    p->n_rng = n_rng;
    return ROSAR_OK;
}

rosar_status planned_params(const char *what, const rosar_c32 *raw, const void *plan, int n_az, int L, int n_rng, int K,
                            const rosar_c32 *out, TdParams *p) {
    if (!raw || !plan || !out) return set_error(ROSAR_ERR_INVALID_ARG, "%s: null raw, plan or out", what);
    if (n_az < 1 || n_rng < 1 || K < 1 || L < 16 || L > 65536)
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: need n_az, n_rng, K >= 1 and 16 <= L <= 65536", what);
    if (L % time_domain_sample_multiple() != 0)
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: L=%d is not a multiple of %d", what, L, time_domain_sample_multiple());
    if ((long long)n_az * L > kMaxElems || (long long)n_rng * n_az > kMaxElems || (long long)n_rng * K > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: sizes too large", what);
    if (misaligned(raw, 16) || misaligned(out, 8) || misaligned(plan, 16))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: misaligned pointer", what);
    const size_t ob = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    if (overlaps(out, ob, raw, sizeof(rosar_c32) * (size_t)n_az * L) ||
        overlaps(out, ob, plan, time_domain_plan_bytes(n_rng, L, K)))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: out overlaps raw or the plan", what);
    *p = TdParams{};
    p->n_az = n_az;
    p->L = L;
    p->n_rng = n_rng;
    return ROSAR_OK;
}
}  // namespace

rosar_status rosar_sas_time_plan(const float *win, const rosar_c32 *w, const int32_t *o, const rosar_radar *radar,
                                 int n_az, int L, int n_rng, int K, int centred, void *plan, size_t plan_bytes,
                                 void *stream) {
    clear_error();
    if (centred != 0 && centred != 1) return set_error(ROSAR_ERR_INVALID_ARG, "sas_time_plan: centred must be 0 or 1");
    if (!w || !o) return set_error(ROSAR_ERR_INVALID_ARG, "sas_time_plan: null w or o");
    TdParams p;
    rosar_status st = plan_params("sas_time_plan", radar, n_az, L, n_rng, K, centred == 1, plan, plan_bytes, &p);
    if (st != ROSAR_OK) return st;
    if (misaligned(w, 8) || misaligned(o, 4) || (win && misaligned(win, 4)))
        return set_error(ROSAR_ERR_INVALID_ARG, "sas_time_plan: misaligned pointer");
    return launch_time_domain_plan(win, reinterpret_cast<const float2 *>(w), o, p, K, false, plan,
                                   static_cast<cudaStream_t>(stream));
}

rosar_status rosar_sas_time_planned(const rosar_c32 *raw, const void *plan, int n_az, int L, int n_rng, int K,
                                    rosar_c32 *out, void *stream) {
    clear_error();
    TdParams p;
    rosar_status st = planned_params("sas_time_planned", raw, plan, n_az, L, n_rng, K, out, &p);
    if (st != ROSAR_OK) return st;
    return launch_time_domain_planned(reinterpret_cast<const float2 *>(raw), p, K, false, plan,
                                      reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_bpa_time_plan(const float *win, const rosar_radar *radar, int n_az, int L, int n_rng, int M_ap,
                                 void *plan, size_t plan_bytes, void *stream) {
    clear_error();
    TdParams p;
    rosar_status st = plan_params("bpa_time_plan", radar, n_az, L, n_rng, M_ap, true, plan, plan_bytes, &p);
    if (st != ROSAR_OK) return st;
    if (M_ap > n_az) return set_error(ROSAR_ERR_INVALID_ARG, "bpa_time_plan: M_ap=%d exceeds n_az=%d", M_ap, n_az);
    if (win && misaligned(win, 4)) return set_error(ROSAR_ERR_INVALID_ARG, "bpa_time_plan: misaligned win");
    return launch_time_domain_plan(win, nullptr, nullptr, p, M_ap, true, plan, static_cast<cudaStream_t>(stream));
}

rosar_status rosar_bpa_time_planned(const rosar_c32 *raw, const void *plan, int n_az, int L, int n_rng, int M_ap,
                                    rosar_c32 *out, void *stream) {
    clear_error();
    TdParams p;
    rosar_status st = planned_params("bpa_time_planned", raw, plan, n_az, L, n_rng, M_ap, out, &p);
    if (st != ROSAR_OK) return st;
    if (M_ap > n_az) return set_error(ROSAR_ERR_INVALID_ARG, "bpa_time_planned: M_ap=%d exceeds n_az=%d", M_ap, n_az);
    return launch_time_domain_planned(reinterpret_cast<const float2 *>(raw), p, M_ap, true, plan,
                                      reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_image(const rosar_c32 *raw, const float *win, const rosar_c32 *w, const int32_t *o,
                         int o_row_stride, int n_az, int L, int K, rosar_c32 *workspace, rosar_c32 *out, void *stream) {
    clear_error();
    rosar_status st = check_range_args(raw, win, n_az, L, workspace);
    if (st != ROSAR_OK) return st;
    st = check_azimuth_args(workspace, w, o, o_row_stride, L, n_az, K, out);
    if (st != ROSAR_OK) return st;
    const size_t bytes = sizeof(rosar_c32) * (size_t)n_az * L;
    if (overlaps(raw, bytes, out, bytes)) return set_error(ROSAR_ERR_INVALID_ARG, "image: raw and out overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = launch_range_compress(reinterpret_cast<const float2 *>(raw), win, n_az, L, 1,
                               reinterpret_cast<float2 *>(workspace), s);
    if (st != ROSAR_OK) return st;
    return launch_sparse_azimuth(reinterpret_cast<const float2 *>(workspace), reinterpret_cast<const float2 *>(w), o,
                                 o_row_stride, L, n_az, K, reinterpret_cast<float2 *>(out), s);
}

int rosar_azimuth_fft_supported(int n_az) { return azimuth_fft_supported(n_az); }

rosar_status rosar_azimuth_plan(const rosar_c32 *w, const int32_t *o, int o_row_stride, int n_rng, int n_az, int K,
                                rosar_c32 *H, void *stream) {
    clear_error();
    if (!w || !o || !H) return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan: null pointer argument");
    if (n_rng < 1 || n_az < 1 || K < 1 || (o_row_stride != 0 && o_row_stride < K))
        return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan: n_rng=%d n_az=%d K=%d o_row_stride=%d", n_rng, n_az, K,
                         o_row_stride);
    if ((long long)n_rng * n_az > kMaxElems) return set_error(ROSAR_ERR_UNSUPPORTED, "azimuth_plan: H too large");
    if (misaligned(w, 8) || misaligned(o, 4) || misaligned(H, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan: misaligned pointer");
    const size_t hb = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    if (overlaps(H, hb, w, sizeof(rosar_c32) * (size_t)n_rng * K)) return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan: H overlaps w");
    return launch_azimuth_plan(reinterpret_cast<const float2 *>(w), o, o_row_stride, n_rng, n_az, K,
                               reinterpret_cast<float2 *>(H), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_azimuth_plan_migrating(const rosar_c32 *w, const int32_t *o, int o_row_stride, const int32_t *dl,
                                          int d_lo, int n_d, int n_rng, int n_az, int K, rosar_c32 *H, void *stream) {
    clear_error();
    if (!w || !o || !dl || !H) return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan_migrating: null pointer argument");
    if (n_rng < 1 || n_az < 1 || K < 1 || (o_row_stride != 0 && o_row_stride < K) || n_d < 1 || n_d > 16)
        return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan_migrating: n_rng=%d n_az=%d K=%d o_row_stride=%d n_d=%d",
                         n_rng, n_az, K, o_row_stride, n_d);
    if ((long long)n_d * n_rng * n_az > kMaxElems || (long long)n_rng * K > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "azimuth_plan_migrating: H too large");
    if (misaligned(w, 8) || misaligned(o, 4) || misaligned(dl, 4) || misaligned(H, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan_migrating: misaligned pointer");
    const size_t hb = sizeof(rosar_c32) * (size_t)n_d * n_rng * n_az;
    if (overlaps(H, hb, w, sizeof(rosar_c32) * (size_t)n_rng * K) || overlaps(H, hb, dl, sizeof(int32_t) * (size_t)n_rng * K))
        return set_error(ROSAR_ERR_INVALID_ARG, "azimuth_plan_migrating: H overlaps an input");
    return launch_azimuth_plan(reinterpret_cast<const float2 *>(w), o, o_row_stride, n_rng, n_az, K,
                               reinterpret_cast<float2 *>(H), static_cast<cudaStream_t>(stream), dl, d_lo, n_d);
}

namespace {
rosar_status check_migrating_fft(const void *S, int n_bins, const void *H, int n_d, int n_rng, int n_az,
                                 const void *spectrum, const void *out, const char *what) {
    if (!S || !H || !spectrum || !out) return set_error(ROSAR_ERR_INVALID_ARG, "%s: null pointer argument", what);
    if (n_bins < 1 || n_rng < 1 || n_az < 1 || n_d < 1 || n_d > 16)
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: n_bins=%d n_rng=%d n_az=%d n_d=%d", what, n_bins, n_rng, n_az, n_d);
    if ((long long)n_bins * n_az > kMaxElems || (long long)n_d * n_rng * n_az > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: array too large", what);
    if (misaligned(S, 8) || misaligned(H, 8) || misaligned(spectrum, 8) || misaligned(out, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: misaligned pointer", what);
    const size_t sb = sizeof(rosar_c32) * (size_t)n_bins * n_az, ob = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    const size_t hb = sizeof(rosar_c32) * (size_t)n_d * n_rng * n_az;
    if (overlaps(out, ob, S, sb) || overlaps(out, ob, H, hb) || overlaps(out, ob, spectrum, sb) ||
        overlaps(spectrum, sb, S, sb) || overlaps(spectrum, sb, H, hb))
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: out or spectrum overlaps another argument", what);
    if (!azimuth_fft_supported(n_az))
        return set_error(ROSAR_ERR_UNSUPPORTED, "%s: n_az=%d is not 2^a 3^b 5^c <= 16384", what, n_az);
    return ROSAR_OK;
}
}  // namespace

rosar_status rosar_sparse_azimuth_migrating_fft(const rosar_c32 *S, int n_bins, const rosar_c32 *H, int d_lo, int n_d,
                                                int n_rng, int n_az, rosar_c32 *spectrum, rosar_c32 *out,
                                                void *stream) {
    clear_error();
    rosar_status st = check_migrating_fft(S, n_bins, H, n_d, n_rng, n_az, spectrum, out, "sparse_azimuth_migrating_fft");
    if (st != ROSAR_OK) return st;
    return launch_sparse_azimuth_migrating_fft(reinterpret_cast<const float2 *>(S), n_bins,
                                               reinterpret_cast<const float2 *>(H), d_lo, n_d, n_rng, n_az,
                                               reinterpret_cast<float2 *>(spectrum), reinterpret_cast<float2 *>(out),
                                               static_cast<cudaStream_t>(stream));
}

rosar_status rosar_image_migrating_fft(const rosar_c32 *raw, const float *win, const rosar_c32 *H, int d_lo, int n_d,
                                       int n_az, int L, rosar_c32 *workspace, rosar_c32 *out, void *stream) {
    clear_error();
    rosar_status st = check_range_args(raw, win, n_az, L, workspace);
    if (st != ROSAR_OK) return st;
    rosar_c32 *S = workspace, *X = workspace + (size_t)n_az * L;
    st = check_migrating_fft(S, L, H, n_d, L, n_az, X, out, "image_migrating_fft");
    if (st != ROSAR_OK) return st;
    const size_t bytes = sizeof(rosar_c32) * (size_t)n_az * L;
    if (overlaps(raw, bytes, out, bytes) || overlaps(raw, bytes, workspace, 2 * bytes))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_migrating_fft: raw overlaps out or the workspace");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = launch_range_compress(reinterpret_cast<const float2 *>(raw), win, n_az, L, 1, reinterpret_cast<float2 *>(S), s);
    if (st != ROSAR_OK) return st;
    return launch_sparse_azimuth_migrating_fft(reinterpret_cast<const float2 *>(S), L, reinterpret_cast<const float2 *>(H),
                                               d_lo, n_d, L, n_az, reinterpret_cast<float2 *>(X),
                                               reinterpret_cast<float2 *>(out), s);
}

rosar_status rosar_sparse_azimuth_fft(const rosar_c32 *S, const rosar_c32 *H, int n_rng, int n_az, rosar_c32 *out,
                                      void *stream) {
    clear_error();
    if (!S || !H || !out) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft: null pointer argument");
    if (n_rng < 1 || n_az < 1) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft: n_rng=%d n_az=%d", n_rng, n_az);
    if ((long long)n_rng * n_az > kMaxElems) return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth_fft: too large");
    if (misaligned(S, 8) || misaligned(H, 8) || misaligned(out, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft: misaligned pointer");
    const size_t img = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    if (overlaps(out, img, S, img) || overlaps(out, img, H, img))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft: out overlaps an input");
    return launch_azimuth_fft(reinterpret_cast<const float2 *>(S), reinterpret_cast<const float2 *>(H), n_rng, n_az,
                              reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_image_fft(const rosar_c32 *raw, const float *win, const rosar_c32 *H, int n_az, int L,
                             rosar_c32 *workspace, rosar_c32 *out, void *stream) {
    clear_error();
    rosar_status st = check_range_args(raw, win, n_az, L, workspace);
    if (st != ROSAR_OK) return st;
    if (!H || !out) return set_error(ROSAR_ERR_INVALID_ARG, "image_fft: null H or out");
    if (misaligned(H, 8) || misaligned(out, 8)) return set_error(ROSAR_ERR_INVALID_ARG, "image_fft: misaligned pointer");
    const size_t bytes = sizeof(rosar_c32) * (size_t)n_az * L;
    if (overlaps(out, bytes, workspace, bytes) || overlaps(out, bytes, raw, bytes) || overlaps(out, bytes, H, bytes))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_fft: out overlaps an input");
    if (!azimuth_fft_supported(n_az))
        return set_error(ROSAR_ERR_UNSUPPORTED, "image_fft: n_az=%d is not 2^a 3^b 5^c <= 16384", n_az);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = launch_range_compress(reinterpret_cast<const float2 *>(raw), win, n_az, L, 1,
                               reinterpret_cast<float2 *>(workspace), s);
    if (st != ROSAR_OK) return st;
    // the azimuth kernel may overlap the range kernel's tail: before its grid-dependency wait it reads only
    // H and its own shared memory, and H is not written by the range kernel
    return launch_azimuth_fft(reinterpret_cast<const float2 *>(workspace), reinterpret_cast<const float2 *>(H), L,
                              n_az, reinterpret_cast<float2 *>(out), s, true);
}

int rosar_image_fft_scans_pipelined(int L, int n_az) {
    return (is_pow2(L) && L >= 8 && L <= 4096 && n_az >= 1) ? image_pipeline_supported(L, n_az) : 0;
}

rosar_status rosar_image_fft_scans(const rosar_c32 *raw, const float *win, const rosar_c32 *H, int n_scans, int n_az,
                                   int L, rosar_c32 *workspace, rosar_c32 *out, void *stream) {
    clear_error();
    if (n_scans < 1) return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_scans: n_scans=%d < 1", n_scans);
    rosar_status st = check_range_args(raw, win, n_az, L, workspace);
    if (st != ROSAR_OK) return st;
    if (!H || !out) return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_scans: null H or out");
    if (misaligned(H, 8) || misaligned(out, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_scans: misaligned pointer");
    const size_t cube = sizeof(rosar_c32) * (size_t)n_az * L;
    const size_t all = cube * (size_t)n_scans;
    if (overlaps(raw, all, workspace, 2 * cube) || overlaps(out, all, raw, all) || overlaps(out, all, workspace, 2 * cube) ||
        overlaps(out, all, H, cube) || overlaps(workspace, 2 * cube, H, cube))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_scans: buffers overlap");
    if (!azimuth_fft_supported(n_az))
        return set_error(ROSAR_ERR_UNSUPPORTED, "image_fft_scans: n_az=%d is not 2^a 3^b 5^c <= 16384", n_az);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (image_pipeline_supported(L, n_az))
        return launch_image_pipeline(reinterpret_cast<const float2 *>(raw), win, reinterpret_cast<const float2 *>(H),
                                     n_scans, n_az, L, reinterpret_cast<float2 *>(workspace),
                                     reinterpret_cast<float2 *>(out), s);
    const size_t elems = (size_t)n_az * L;
    for (int i = 0; i < n_scans; ++i) {
        st = launch_range_compress(reinterpret_cast<const float2 *>(raw + i * elems), win, n_az, L, 1,
                                   reinterpret_cast<float2 *>(workspace), s);
        if (st != ROSAR_OK) return st;
        st = launch_azimuth_fft(reinterpret_cast<const float2 *>(workspace), reinterpret_cast<const float2 *>(H), L,
                                n_az, reinterpret_cast<float2 *>(out + i * elems), s, true);
        if (st != ROSAR_OK) return st;
    }
    return ROSAR_OK;
}

rosar_status rosar_image_fft_host(const rosar_c32 *raw_host, const float *win, const rosar_c32 *H, int n_az, int L,
                                  rosar_c32 *raw_dev, rosar_c32 *workspace, rosar_c32 *out_dev, rosar_c32 *out_host,
                                  void *stream) {
    clear_error();
    if (!raw_host || !out_host) return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_host: null host buffer");
    rosar_status st = check_range_args(raw_dev, win, n_az, L, workspace);
    if (st != ROSAR_OK) return st;
    if (!H || !out_dev) return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_host: null H or out_dev");
    if (misaligned(H, 8) || misaligned(out_dev, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_host: misaligned pointer");
    const size_t bytes = sizeof(rosar_c32) * (size_t)n_az * L;
    if (overlaps(out_dev, bytes, workspace, bytes) || overlaps(out_dev, bytes, raw_dev, bytes) ||
        overlaps(out_dev, bytes, H, bytes) || overlaps(raw_dev, bytes, workspace, bytes))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_host: device buffers overlap");
    if (overlaps(raw_host, bytes, out_host, bytes))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_fft_host: host buffers overlap");
    if (!azimuth_fft_supported(n_az))
        return set_error(ROSAR_ERR_UNSUPPORTED, "image_fft_host: n_az=%d is not 2^a 3^b 5^c <= 16384", n_az);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(raw_dev, raw_host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "image_fft_host: H2D copy: %s", cudaGetErrorString(e));
    st = launch_range_compress(reinterpret_cast<const float2 *>(raw_dev), win, n_az, L, 1,
                               reinterpret_cast<float2 *>(workspace), s);
    if (st != ROSAR_OK) return st;
    st = launch_azimuth_fft(reinterpret_cast<const float2 *>(workspace), reinterpret_cast<const float2 *>(H), L, n_az,
                            reinterpret_cast<float2 *>(out_dev), s, true);
    if (st != ROSAR_OK) return st;
    e = cudaMemcpyAsync(out_host, out_dev, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "image_fft_host: D2H copy: %s", cudaGetErrorString(e));
    return ROSAR_OK;
}

// ------------------------------------------------------------ differentiable form --

namespace {

rosar_status check_stack(const char *what, int n_scans, int n_rng, int n_az) {
    if (n_scans < 1 || n_rng < 1 || n_az < 1)
        return set_error(ROSAR_ERR_INVALID_ARG, "%s: n_scans=%d n_rng=%d n_az=%d must be >= 1", what, n_scans, n_rng,
                         n_az);
    if ((long long)n_scans * n_rng * n_az > kMaxElems) return set_error(ROSAR_ERR_UNSUPPORTED, "%s: stack too large", what);
    return ROSAR_OK;
}

}  // namespace

rosar_status rosar_phase_apply(const rosar_c32 *S, const float *eps, int n_scans, int n_rng, int n_az, rosar_c32 *S_t,
                               void *stream) {
    clear_error();
    if (!S || !eps || !S_t) return set_error(ROSAR_ERR_INVALID_ARG, "phase_apply: null pointer argument");
    rosar_status st = check_stack("phase_apply", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (misaligned(S, 8) || misaligned(S_t, 8) || misaligned(eps, 4))
        return set_error(ROSAR_ERR_INVALID_ARG, "phase_apply: misaligned pointer");
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az;
    if (S != S_t && overlaps(S, b, S_t, b)) return set_error(ROSAR_ERR_INVALID_ARG, "phase_apply: S and S_t partly overlap");
    return launch_phase_apply(reinterpret_cast<const float2 *>(S), eps, n_scans, n_rng, n_az,
                              reinterpret_cast<float2 *>(S_t), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_sparse_azimuth_scans(const rosar_c32 *S, const rosar_c32 *w, const int32_t *o, int o_row_stride,
                                        int n_scans, int n_rng, int n_az, int K, rosar_c32 *out, void *stream) {
    clear_error();
    rosar_status st = check_stack("sparse_azimuth_scans", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    st = check_azimuth_args(S, w, o, o_row_stride, n_rng, n_az, K, out);
    if (st != ROSAR_OK) return st;
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az;
    if (overlaps(out, b, S, b)) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_scans: out overlaps S");
    return launch_sparse_azimuth_scans(reinterpret_cast<const float2 *>(S), reinterpret_cast<const float2 *>(w), o,
                                       o_row_stride, n_scans, n_rng, n_az, K, false, reinterpret_cast<float2 *>(out),
                                       static_cast<cudaStream_t>(stream));
}

rosar_status rosar_sparse_azimuth_adjoint(const rosar_c32 *g, const rosar_c32 *S_t, const rosar_c32 *w,
                                          const int32_t *o, int o_row_stride, int n_scans, int n_rng, int n_az, int K,
                                          rosar_c32 *grad_S_t, rosar_c32 *grad_w, void *stream) {
    clear_error();
    rosar_status st = check_stack("sparse_azimuth_adjoint", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (!g || !w || !o || (!grad_S_t && !grad_w) || (grad_w && !S_t))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_adjoint: null pointer argument");
    if (K < 1 || (o_row_stride != 0 && o_row_stride < K))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_adjoint: K=%d o_row_stride=%d", K, o_row_stride);
    if (misaligned(g, 8) || misaligned(w, 8) || misaligned(o, 4) || (S_t && misaligned(S_t, 8)) ||
        (grad_S_t && misaligned(grad_S_t, 8)) || (grad_w && misaligned(grad_w, 8)))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_adjoint: misaligned pointer");
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az;
    if (grad_S_t && (overlaps(grad_S_t, b, g, b) || (S_t && overlaps(grad_S_t, b, S_t, b))))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_adjoint: grad_S_t overlaps an input");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grad_S_t) {
        st = launch_sparse_azimuth_scans(reinterpret_cast<const float2 *>(g), reinterpret_cast<const float2 *>(w), o,
                                         o_row_stride, n_scans, n_rng, n_az, K, true,
                                         reinterpret_cast<float2 *>(grad_S_t), s);
        if (st != ROSAR_OK) return st;
    }
    if (grad_w)
        st = launch_azimuth_weight_grad(reinterpret_cast<const float2 *>(g), reinterpret_cast<const float2 *>(S_t), o,
                                        o_row_stride, n_scans, n_rng, n_az, K, reinterpret_cast<float2 *>(grad_w), s);
    return st;
}

rosar_status rosar_sparse_azimuth_fft_scans(const rosar_c32 *S, const rosar_c32 *H, int n_scans, int n_rng, int n_az,
                                            int adjoint, rosar_c32 *out, void *stream) {
    clear_error();
    rosar_status st = check_stack("sparse_azimuth_fft_scans", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (!S || !H || !out) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans: null pointer argument");
    if (adjoint != 0 && adjoint != 1)
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans: adjoint must be 0 or 1");
    if (misaligned(S, 8) || misaligned(H, 8) || misaligned(out, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans: misaligned pointer");
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az;
    if (overlaps(out, b, S, b) || overlaps(out, b, H, sizeof(rosar_c32) * (size_t)n_rng * n_az))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans: out overlaps an input");
    if (!azimuth_fft_supported(n_az))
        return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth_fft_scans: n_az=%d is not 2^a 3^b 5^c <= 16384", n_az);
    return launch_azimuth_fft(reinterpret_cast<const float2 *>(S), reinterpret_cast<const float2 *>(H), n_scans * n_rng,
                              n_az, reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream), false, n_rng,
                              adjoint == 1);
}

rosar_status rosar_azimuth_weight_grad_fft(const rosar_c32 *g, const rosar_c32 *S_t, const int32_t *o, int o_row_stride,
                                           int n_scans, int n_rng, int n_az, int K, rosar_c32 *grad_w, void *stream) {
    clear_error();
    rosar_status st = check_stack("weight_grad_fft", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (!g || !S_t || !o || !grad_w) return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft: null pointer argument");
    if (K < 1 || (o_row_stride != 0 && o_row_stride < K))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft: K=%d o_row_stride=%d", K, o_row_stride);
    if ((long long)n_rng * K > kMaxElems || (long long)n_rng * o_row_stride > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "weight_grad_fft: sizes too large");
    if (misaligned(g, 8) || misaligned(S_t, 8) || misaligned(o, 4) || misaligned(grad_w, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft: misaligned pointer");
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az, gw = sizeof(rosar_c32) * (size_t)n_rng * K;
    if (overlaps(grad_w, gw, g, b) || overlaps(grad_w, gw, S_t, b))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft: grad_w overlaps an input");
    return launch_azimuth_weight_grad_fft(reinterpret_cast<const float2 *>(g), reinterpret_cast<const float2 *>(S_t), o,
                                          o_row_stride, n_scans, n_rng, n_az, K, reinterpret_cast<float2 *>(grad_w),
                                          static_cast<cudaStream_t>(stream));
}

rosar_status rosar_phase_grad(const rosar_c32 *S_t, const rosar_c32 *grad_S_t, const float *eps, int n_scans,
                              int n_rng, int n_az, float *grad_eps, rosar_c32 *grad_S, void *stream) {
    clear_error();
    if (!S_t || !grad_S_t || (!grad_eps && !grad_S) || (grad_S && !eps))
        return set_error(ROSAR_ERR_INVALID_ARG, "phase_grad: null pointer argument");
    rosar_status st = check_stack("phase_grad", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (misaligned(S_t, 8) || misaligned(grad_S_t, 8) || (eps && misaligned(eps, 4)) ||
        (grad_eps && misaligned(grad_eps, 4)) || (grad_S && misaligned(grad_S, 8)))
        return set_error(ROSAR_ERR_INVALID_ARG, "phase_grad: misaligned pointer");
    return launch_phase_grad(reinterpret_cast<const float2 *>(S_t), reinterpret_cast<const float2 *>(grad_S_t), eps,
                             n_scans, n_rng, n_az, grad_eps, reinterpret_cast<float2 *>(grad_S),
                             static_cast<cudaStream_t>(stream));
}

rosar_status rosar_phasors(const float *eps, long long n, rosar_c32 *P, void *stream) {
    clear_error();
    if (!eps || !P) return set_error(ROSAR_ERR_INVALID_ARG, "phasors: null pointer argument");
    if (n < 1) return set_error(ROSAR_ERR_INVALID_ARG, "phasors: n=%lld < 1", n);
    if (misaligned(eps, 4) || misaligned(P, 8)) return set_error(ROSAR_ERR_INVALID_ARG, "phasors: misaligned pointer");
    if (overlaps(P, sizeof(rosar_c32) * (size_t)n, eps, sizeof(float) * (size_t)n))
        return set_error(ROSAR_ERR_INVALID_ARG, "phasors: P overlaps eps");
    return launch_phasors(eps, n, reinterpret_cast<float2 *>(P), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_sparse_azimuth_fft_scans_ex(const rosar_c32 *S, const rosar_c32 *P, const rosar_c32 *H, int n_scans,
                                              int n_rng, int n_az, int adjoint, rosar_c32 *out, rosar_c32 *spectrum,
                                              void *stream) {
    clear_error();
    rosar_status st = check_stack("sparse_azimuth_fft_scans_ex", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (!S || !H || !out) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans_ex: null pointer argument");
    if (adjoint != 0 && adjoint != 1)
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans_ex: adjoint must be 0 or 1");
    if (misaligned(S, 8) || misaligned(H, 8) || misaligned(out, 8) || (P && misaligned(P, 8)) ||
        (spectrum && misaligned(spectrum, 8)))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans_ex: misaligned pointer");
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az;
    const size_t hb = sizeof(rosar_c32) * (size_t)n_rng * n_az, pb = sizeof(rosar_c32) * (size_t)n_scans * n_az;
    if (overlaps(out, b, S, b) || overlaps(out, b, H, hb) || (P && overlaps(out, b, P, pb)))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans_ex: out overlaps an input");
    if (spectrum && (overlaps(spectrum, b, S, b) || overlaps(spectrum, b, H, hb) || overlaps(spectrum, b, out, b) ||
                     (P && overlaps(spectrum, b, P, pb))))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_fft_scans_ex: spectrum overlaps another argument");
    if (!azimuth_fft_supported(n_az))
        return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth_fft_scans_ex: n_az=%d is not 2^a 3^b 5^c <= 16384", n_az);
    return launch_azimuth_fft(reinterpret_cast<const float2 *>(S), reinterpret_cast<const float2 *>(H), n_scans * n_rng,
                              n_az, reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream), false, n_rng,
                              adjoint == 1, reinterpret_cast<const float2 *>(P), reinterpret_cast<float2 *>(spectrum));
}

rosar_status rosar_azimuth_weight_grad_spectra(const rosar_c32 *G, const rosar_c32 *X, const int32_t *o,
                                               int o_row_stride, int n_scans, int n_rng, int n_az, int K,
                                               rosar_c32 *workspace, rosar_c32 *grad_w, void *stream) {
    clear_error();
    rosar_status st = check_stack("weight_grad_spectra", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (!G || !X || !o || !workspace || !grad_w)
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_spectra: null pointer argument");
    if (misaligned(workspace, 8)) return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_spectra: misaligned workspace");
    {
        const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az, wb = sizeof(rosar_c32) * (size_t)n_rng * n_az;
        if (overlaps(workspace, wb, G, b) || overlaps(workspace, wb, X, b) ||
            overlaps(workspace, wb, grad_w, sizeof(rosar_c32) * (size_t)n_rng * K))
            return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_spectra: workspace overlaps another argument");
    }
    if (K < 1 || (o_row_stride != 0 && o_row_stride < K))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_spectra: K=%d o_row_stride=%d", K, o_row_stride);
    if ((long long)n_rng * K > kMaxElems || (long long)n_rng * o_row_stride > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "weight_grad_spectra: sizes too large");
    if (misaligned(G, 8) || misaligned(X, 8) || misaligned(o, 4) || misaligned(grad_w, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_spectra: misaligned pointer");
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az, gw = sizeof(rosar_c32) * (size_t)n_rng * K;
    if (overlaps(grad_w, gw, G, b) || overlaps(grad_w, gw, X, b))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_spectra: grad_w overlaps an input");
    return launch_azimuth_weight_grad_spectra(reinterpret_cast<const float2 *>(G), reinterpret_cast<const float2 *>(X), o,
                                              o_row_stride, n_scans, n_rng, n_az, K,
                                              reinterpret_cast<float2 *>(workspace), reinterpret_cast<float2 *>(grad_w),
                                              static_cast<cudaStream_t>(stream));
}

rosar_status rosar_azimuth_weight_grad_fft_phase(const rosar_c32 *g, const rosar_c32 *S, const rosar_c32 *P,
                                                 const int32_t *o, int o_row_stride, int n_scans, int n_rng, int n_az,
                                                 int K, rosar_c32 *grad_w, void *stream) {
    clear_error();
    if (!P) return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft_phase: null P");
    if (misaligned(P, 8)) return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft_phase: misaligned P");
    rosar_status st = check_stack("weight_grad_fft_phase", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (!g || !S || !o || !grad_w) return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft_phase: null pointer argument");
    if (K < 1 || (o_row_stride != 0 && o_row_stride < K))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft_phase: K=%d o_row_stride=%d", K, o_row_stride);
    if ((long long)n_rng * K > kMaxElems || (long long)n_rng * o_row_stride > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "weight_grad_fft_phase: sizes too large");
    if (misaligned(g, 8) || misaligned(S, 8) || misaligned(o, 4) || misaligned(grad_w, 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft_phase: misaligned pointer");
    const size_t b = sizeof(rosar_c32) * (size_t)n_scans * n_rng * n_az, gw = sizeof(rosar_c32) * (size_t)n_rng * K;
    if (overlaps(grad_w, gw, g, b) || overlaps(grad_w, gw, S, b) ||
        overlaps(grad_w, gw, P, sizeof(rosar_c32) * (size_t)n_scans * n_az))
        return set_error(ROSAR_ERR_INVALID_ARG, "weight_grad_fft_phase: grad_w overlaps an input");
    return launch_azimuth_weight_grad_fft(reinterpret_cast<const float2 *>(g), reinterpret_cast<const float2 *>(S), o,
                                          o_row_stride, n_scans, n_rng, n_az, K, reinterpret_cast<float2 *>(grad_w),
                                          static_cast<cudaStream_t>(stream), reinterpret_cast<const float2 *>(P));
}

rosar_status rosar_phase_grad_phasor(const rosar_c32 *S, const rosar_c32 *P, const rosar_c32 *grad_S_t, int n_scans,
                                     int n_rng, int n_az, float *grad_eps, rosar_c32 *grad_S, void *stream) {
    clear_error();
    if (!S || !P || !grad_S_t || (!grad_eps && !grad_S))
        return set_error(ROSAR_ERR_INVALID_ARG, "phase_grad_phasor: null pointer argument");
    rosar_status st = check_stack("phase_grad_phasor", n_scans, n_rng, n_az);
    if (st != ROSAR_OK) return st;
    if (misaligned(S, 8) || misaligned(P, 8) || misaligned(grad_S_t, 8) || (grad_eps && misaligned(grad_eps, 4)) ||
        (grad_S && misaligned(grad_S, 8)))
        return set_error(ROSAR_ERR_INVALID_ARG, "phase_grad_phasor: misaligned pointer");
    return launch_phase_grad_phasor(reinterpret_cast<const float2 *>(S), reinterpret_cast<const float2 *>(P),
                                    reinterpret_cast<const float2 *>(grad_S_t), n_scans, n_rng, n_az, grad_eps,
                                    reinterpret_cast<float2 *>(grad_S), static_cast<cudaStream_t>(stream));
}

size_t rosar_image_l2_loss_workspace_bytes(void) { return sizeof(double) * (size_t)image_loss_partials(); }

rosar_status rosar_image_l2_loss(const rosar_c32 *out, const rosar_c32 *ref, long long n, void *workspace,
                                 float *loss, void *stream) {
    clear_error();
    if (!out || !ref || !workspace || !loss) return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss: null pointer argument");
    if (n < 1) return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss: n=%lld < 1", n);
    if (misaligned(out, 8) || misaligned(ref, 8) || misaligned(workspace, 8) || misaligned(loss, 4))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss: misaligned pointer");
    return launch_image_l2_loss(reinterpret_cast<const float2 *>(out), reinterpret_cast<const float2 *>(ref), n,
                                static_cast<double *>(workspace), loss, static_cast<cudaStream_t>(stream));
}

rosar_status rosar_image_l2_loss_grad(const rosar_c32 *out, const rosar_c32 *ref, long long n, const float *g,
                                      rosar_c32 *grad, void *stream) {
    clear_error();
    if (!out || !ref || !g || !grad) return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss_grad: null pointer argument");
    if (n < 1) return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss_grad: n=%lld < 1", n);
    if (misaligned(out, 8) || misaligned(ref, 8) || misaligned(grad, 8) || misaligned(g, 4))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss_grad: misaligned pointer");
    const size_t bytes = sizeof(rosar_c32) * (size_t)n;
    if (overlaps(grad, bytes, out, bytes) && grad != out)
        return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss_grad: grad partially overlaps out");
    if (overlaps(grad, bytes, ref, bytes) && grad != ref)
        return set_error(ROSAR_ERR_INVALID_ARG, "image_l2_loss_grad: grad partially overlaps ref");
    return launch_image_l2_loss_grad(reinterpret_cast<const float2 *>(out), reinterpret_cast<const float2 *>(ref), n,
                                     g, reinterpret_cast<float2 *>(grad), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_range_compress_adjoint(const rosar_c32 *g, const float *win, int n_az, int L, int centred,
                                          rosar_c32 *grad_raw, void *stream) {
    clear_error();
    rosar_status st = check_range_args(g, win, n_az, L, grad_raw);
    if (st != ROSAR_OK) return st;
    return launch_range_compress_adjoint(reinterpret_cast<const float2 *>(g), win, n_az, L, centred,
                                         reinterpret_cast<float2 *>(grad_raw), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_range_compress_adjoint_scans(const rosar_c32 *g, const float *win, int n_scans, int n_az, int L,
                                                int centred, rosar_c32 *grad_raw, void *stream) {
    clear_error();
    if (n_scans < 1 || n_scans > 65535)
        return set_error(ROSAR_ERR_INVALID_ARG, "range_compress_adjoint_scans: n_scans=%d not in [1, 65535]", n_scans);
    rosar_status st = check_range_args(g, win, n_az, L, grad_raw);
    if (st != ROSAR_OK) return st;
    const size_t all = sizeof(rosar_c32) * (size_t)n_az * L * n_scans;
    if (overlaps(g, all, grad_raw, all))
        return set_error(ROSAR_ERR_INVALID_ARG, "range_compress_adjoint_scans: g and grad_raw overlap");
    return launch_range_compress_adjoint(reinterpret_cast<const float2 *>(g), win, n_az, L, centred,
                                         reinterpret_cast<float2 *>(grad_raw), static_cast<cudaStream_t>(stream),
                                         n_scans);
}

// ------------------------------------------------------- range-migration-aware taps --

rosar_status rosar_sparse_azimuth_migrating(const rosar_c32 *S, int n_bins, const rosar_c32 *w, const int32_t *o,
                                            int o_row_stride, const int32_t *dl, int n_rng, int n_az, int K,
                                            rosar_c32 *out, void *stream) {
    clear_error();
    if (!dl) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_migrating: null dl");
    if (n_bins < 1) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_migrating: n_bins=%d < 1", n_bins);
    rosar_status st = check_azimuth_args(S, w, o, o_row_stride, n_rng, n_az, K, out);
    if (st != ROSAR_OK) return st;
    if ((long long)n_bins * n_az > kMaxElems || (long long)n_rng * K > kMaxElems)
        return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth_migrating: array too large");
    if (misaligned(dl, 4)) return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_migrating: misaligned dl");
    const size_t img = sizeof(rosar_c32) * (size_t)n_rng * n_az;
    if (overlaps(out, img, S, sizeof(rosar_c32) * (size_t)n_bins * n_az) ||
        overlaps(out, img, dl, sizeof(int32_t) * (size_t)n_rng * K))
        return set_error(ROSAR_ERR_INVALID_ARG, "sparse_azimuth_migrating: out overlaps an input");
    return launch_sparse_azimuth_migrating(reinterpret_cast<const float2 *>(S), n_bins,
                                           reinterpret_cast<const float2 *>(w), o, o_row_stride, dl, n_rng, n_az, K,
                                           reinterpret_cast<float2 *>(out), static_cast<cudaStream_t>(stream));
}

rosar_status rosar_image_migrating(const rosar_c32 *raw, const float *win, const rosar_c32 *w, const int32_t *o,
                                   int o_row_stride, const int32_t *dl, int n_az, int L, int K, rosar_c32 *workspace,
                                   rosar_c32 *out, void *stream) {
    clear_error();
    rosar_status st = check_range_args(raw, win, n_az, L, workspace);
    if (st != ROSAR_OK) return st;
    st = check_azimuth_args(workspace, w, o, o_row_stride, L, n_az, K, out);
    if (st != ROSAR_OK) return st;
    if (!dl || misaligned(dl, 4)) return set_error(ROSAR_ERR_INVALID_ARG, "image_migrating: null or misaligned dl");
    const size_t bytes = sizeof(rosar_c32) * (size_t)n_az * L;
    if (overlaps(raw, bytes, out, bytes)) return set_error(ROSAR_ERR_INVALID_ARG, "image_migrating: raw and out overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = launch_range_compress(reinterpret_cast<const float2 *>(raw), win, n_az, L, 1,
                               reinterpret_cast<float2 *>(workspace), s);
    if (st != ROSAR_OK) return st;
    return launch_sparse_azimuth_migrating(reinterpret_cast<const float2 *>(workspace), L,
                                           reinterpret_cast<const float2 *>(w), o, o_row_stride, dl, L, n_az, K,
                                           reinterpret_cast<float2 *>(out), s);
}

}  // extern "C"
