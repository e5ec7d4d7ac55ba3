// rosar_image_noalloc: the whole-scan image for callers that cannot allocate device memory.
//
// rosar_image needs an L x n_az complex workspace for the range-compressed data.
// Some callers only own the input and output buffers: a plugin whose host hands
// it device buffers but no allocator, or a real-time radar loop that must not
// call cudaMalloc after start-up (it can block on the whole device for
// milliseconds).  This entry point keeps that intermediate in a fixed-size
// array that lives in the library's own device memory instead.
//
// The array is a file-scope __device__ object: every GPU that loads the library
// holds ROSAR_NOALLOC_MAX_ELEMS * 8 bytes (16 MiB) until the process exits.  In
// host code its name is only a host-side stand-in, so the first call on each
// device (with that device current) looks up its device address with
// cudaGetSymbolAddress and caches it; that first call should therefore come
// before any stream capture.  All calls share the one array: calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it, so serialise them.  The range compression overwrites every element it
// later reads, so nothing left by an earlier call needs clearing.

#include <mutex>

#include "rosar_internal.cuh"

namespace rosar {
namespace {

static __device__ __align__(256) float2 g_noalloc_scratch[ROSAR_NOALLOC_MAX_ELEMS];

float2 *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device (looked up once per device).
rosar_status scratch_address(float2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "image_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(ROSAR_ERR_UNSUPPORTED, "image_noalloc: device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return set_error(ROSAR_ERR_CUDA, "image_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<float2 *>(p);
    }
    *out = g_scratch_addr[dev];
    return ROSAR_OK;
}

bool unaligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) != 0; }

}  // namespace
}  // namespace rosar

using namespace rosar;

extern "C" rosar_status rosar_image_noalloc(const rosar_c32 *raw, const float *win, const rosar_c32 *w,
                                           const int32_t *o, int o_row_stride, int n_az, int L, int K,
                                           rosar_c32 *out, void *stream) {
    clear_error();
    if (!raw || !w || !o || !out) return set_error(ROSAR_ERR_INVALID_ARG, "image_noalloc: null pointer argument");
    if (n_az < 1 || K < 1) return set_error(ROSAR_ERR_INVALID_ARG, "image_noalloc: n_az=%d and K=%d must be >= 1", n_az, K);
    if (!is_pow2(L) || L < 8 || L > 4096)
        return set_error(ROSAR_ERR_UNSUPPORTED, "image_noalloc: L=%d is not a power of two in [8, 4096]", L);
    if ((long long)n_az * L > (long long)ROSAR_NOALLOC_MAX_ELEMS)
        return set_error(ROSAR_ERR_UNSUPPORTED,
                         "image_noalloc: L*n_az = %lld exceeds the built-in scratch of %d complex elements; "
                         "use rosar_image with a caller-provided workspace",
                         (long long)n_az * L, (int)ROSAR_NOALLOC_MAX_ELEMS);
    if (o_row_stride != 0 && o_row_stride < K)
        return set_error(ROSAR_ERR_INVALID_ARG, "image_noalloc: o_row_stride=%d < K=%d", o_row_stride, K);
    if (unaligned(raw, 8) || unaligned(w, 8) || unaligned(o, 4) || unaligned(out, 8) || (win && unaligned(win, 4)))
        return set_error(ROSAR_ERR_INVALID_ARG, "image_noalloc: misaligned pointer");
    const uintptr_t a = reinterpret_cast<uintptr_t>(raw), b = reinterpret_cast<uintptr_t>(out);
    const uintptr_t nb = sizeof(rosar_c32) * (uintptr_t)n_az * L;
    if (a < b + nb && b < a + nb) return set_error(ROSAR_ERR_INVALID_ARG, "image_noalloc: raw and out overlap");

    float2 *S = nullptr;
    rosar_status st = scratch_address(&S);
    if (st != ROSAR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = launch_range_compress(reinterpret_cast<const float2 *>(raw), win, n_az, L, 1, S, s);
    if (st != ROSAR_OK) return st;
    return launch_sparse_azimuth(S, reinterpret_cast<const float2 *>(w), o, o_row_stride, L, n_az, K,
                                 reinterpret_cast<float2 *>(out), s);
}
