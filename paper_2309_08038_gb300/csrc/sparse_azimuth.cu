// K2: sparse-aperture azimuth matched filter (arXiv 2309.08038, Sec. III-D, Eq. (43); Algorithm 2).
//
//   out[r][theta] = sum_{k<K} w[r][k] * S[r][(theta + o_k) mod n_az]
//
// Grid: (azimuth tiles of TW = 1024 outputs, range rows, scans); each CTA runs one
// gather-MAC tile (azimuth_tile.cuh): the row's circular window staged in shared
// memory, 4 outputs per thread, taps broadcast from shared memory.  The same
// kernel with conjugated weights and negated offsets is the adjoint in S.

#include "azimuth_tile.cuh"

namespace rosar {
namespace {

constexpr int SA_J = 4;
using SaGeo = az::Geo<SA_J>;

// blockIdx = (azimuth tile, range row, scan); scans are stacked [n_scans][n_rng][n_az] and share w, o.
template <bool ADJ>
__global__ void __launch_bounds__(az::THREADS)
sparse_azimuth_kernel(const float2 *__restrict__ S, const float2 *__restrict__ w, const int32_t *__restrict__ o,
                      int o_row_stride, int n_rng, int n_az, int K, float2 *__restrict__ out) {
    extern __shared__ __align__(16) char sm[];
    __shared__ int red[4 * az::THREADS / 32];
    const size_t scan = (size_t)blockIdx.z * n_rng * n_az;
    az::azimuth_tile<SA_J, false, ADJ>(S + scan, w, o, o_row_stride, n_az, K, out + scan, blockIdx.y,
                                       blockIdx.x * SaGeo::TW, sm, red);
}

template <bool ADJ>
rosar_status launch_gather(const float2 *S, const float2 *w, const int32_t *o, int o_row_stride, int n_scans,
                           int n_rng, int n_az, int K, float2 *out, cudaStream_t s) {
    static int done[kMaxDevices] = {};
    rosar_status st = ensure_smem((const void *)sparse_azimuth_kernel<ADJ>, SaGeo::SMEM_BYTES, done, "sparse_azimuth");
    if (st != ROSAR_OK) return st;
    if (n_rng > 65535 || n_scans > 65535)
        return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth: n_rng=%d or n_scans=%d exceeds 65535", n_rng, n_scans);
    dim3 grid((n_az + SaGeo::TW - 1) / SaGeo::TW, n_rng, n_scans);
    sparse_azimuth_kernel<ADJ><<<grid, az::THREADS, SaGeo::SMEM_BYTES, s>>>(S, w, o, o_row_stride, n_rng, n_az, K, out);
    return check_launch(ADJ ? "sparse_azimuth_adjoint" : "sparse_azimuth");
}

using MigGeo = az::GeoMig<SA_J>;

__global__ void __launch_bounds__(az::THREADS)
sparse_azimuth_mig_kernel(const float2 *__restrict__ S, int n_bins, const float2 *__restrict__ w,
                          const int32_t *__restrict__ o, int o_row_stride, const int32_t *__restrict__ dl, int n_az,
                          int K, float2 *__restrict__ out) {
    extern __shared__ __align__(16) char sm[];
    __shared__ int red[4 * az::THREADS / 32];
    az::azimuth_tile<SA_J, false, false, true>(S, w, o, o_row_stride, n_az, K, out, blockIdx.y,
                                               blockIdx.x * MigGeo::TW, sm, red, dl, n_bins);
}

}  // namespace

rosar_status launch_sparse_azimuth_migrating(const float2 *S, int n_bins, const float2 *w, const int32_t *o,
                                             int o_row_stride, const int32_t *dl, int n_rng, int n_az, int K,
                                             float2 *out, cudaStream_t s) {
    static int done[kMaxDevices] = {};
    rosar_status st = ensure_smem((const void *)sparse_azimuth_mig_kernel, MigGeo::SMEM_BYTES, done,
                                  "sparse_azimuth_migrating");
    if (st != ROSAR_OK) return st;
    if (n_rng > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth_migrating: n_rng=%d exceeds 65535", n_rng);
    dim3 grid((n_az + MigGeo::TW - 1) / MigGeo::TW, n_rng);
    sparse_azimuth_mig_kernel<<<grid, az::THREADS, MigGeo::SMEM_BYTES, s>>>(S, n_bins, w, o, o_row_stride, dl, n_az,
                                                                           K, out);
    return check_launch("sparse_azimuth_migrating");
}

rosar_status launch_sparse_azimuth(const float2 *S, const float2 *w, const int32_t *o, int o_row_stride, int n_rng,
                                   int n_az, int K, float2 *out, cudaStream_t s) {
    return launch_gather<false>(S, w, o, o_row_stride, 1, n_rng, n_az, K, out, s);
}

rosar_status launch_sparse_azimuth_scans(const float2 *S, const float2 *w, const int32_t *o, int o_row_stride,
                                         int n_scans, int n_rng, int n_az, int K, bool adjoint, float2 *out,
                                         cudaStream_t s) {
    return adjoint ? launch_gather<true>(S, w, o, o_row_stride, n_scans, n_rng, n_az, K, out, s)
                   : launch_gather<false>(S, w, o, o_row_stride, n_scans, n_rng, n_az, K, out, s);
}

}  // namespace rosar
