// K2: sparse-aperture azimuth matched filter (arXiv 2309.08038, Sec. III-D, Eq. (43); Algorithm 2).
//
//   out[r][theta] = sum_{k<K} w[r][k] * S[r][(theta + o_k) mod n_az]
//
// Grid: (azimuth tiles of TW = 1024 outputs, range rows); each CTA runs one
// gather-MAC tile (azimuth_tile.cuh): the row's circular window staged in shared
// memory, 4 outputs per thread, taps broadcast from shared memory.

#include "azimuth_tile.cuh"

namespace rosar {
namespace {

constexpr int SA_J = 4;
using SaGeo = az::Geo<SA_J>;

__global__ void __launch_bounds__(az::THREADS)
sparse_azimuth_kernel(const float2 *__restrict__ S, const float2 *__restrict__ w, const int32_t *__restrict__ o,
                      int o_row_stride, int n_az, int K, float2 *__restrict__ out) {
    extern __shared__ __align__(16) char sm[];
    __shared__ int red[2 * az::THREADS / 32];
    az::azimuth_tile<SA_J, false>(S, w, o, o_row_stride, n_az, K, out, blockIdx.y, blockIdx.x * SaGeo::TW, sm, red);
}

}  // namespace

rosar_status launch_sparse_azimuth(const float2 *S, const float2 *w, const int32_t *o, int o_row_stride, int n_rng,
                                   int n_az, int K, float2 *out, cudaStream_t s) {
    static int done[kMaxDevices] = {};
    rosar_status st = ensure_smem((const void *)sparse_azimuth_kernel, SaGeo::SMEM_BYTES, done, "sparse_azimuth");
    if (st != ROSAR_OK) return st;
    if (n_rng > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth: n_rng=%d exceeds 65535", n_rng);
    dim3 grid((n_az + SaGeo::TW - 1) / SaGeo::TW, n_rng);
    sparse_azimuth_kernel<<<grid, az::THREADS, SaGeo::SMEM_BYTES, s>>>(S, w, o, o_row_stride, n_az, K, out);
    return check_launch("sparse_azimuth");
}

}  // namespace rosar
