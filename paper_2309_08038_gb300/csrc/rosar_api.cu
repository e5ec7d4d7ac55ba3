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
    return launch_azimuth_fft(reinterpret_cast<const float2 *>(workspace), reinterpret_cast<const float2 *>(H), L,
                              n_az, reinterpret_cast<float2 *>(out), s);
}

}  // extern "C"
