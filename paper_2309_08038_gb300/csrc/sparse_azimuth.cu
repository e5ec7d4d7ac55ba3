// K2: sparse-aperture azimuth matched filter (arXiv 2309.08038, Sec. III-D, Eq. (43); Algorithm 2).
//
//   out[r][theta] = sum_{k<K} w[r][k] * S[r][(theta + o_k) mod n_az]
//
// Grid: (azimuth tiles of TW = 1024 outputs, range rows).  A CTA first reduces its
// row's offsets to a canonical representative in [-n_az/2, n_az/2] and finds their
// span [lo, hi]; it then stages the circular window S[r][theta0+lo .. theta0+TW-1+hi]
// in shared memory with coalesced loads (wrap handled at staging, so the inner
// loop has no modulo).  Each thread owns J = 4 outputs strided by the block size,
// so for every tap the warp reads 32 consecutive window entries (conflict-free)
// and the tap's weight and relative offset are shared-memory broadcasts.  Taps
// are staged in chunks of KC and accumulated in float32 in increasing k.
// A row whose offsets span more than SPAN_CAP pulses falls back to direct
// (L1/L2-cached) gathers with an explicit modulo.

#include <limits.h>

#include "rosar_internal.cuh"

namespace rosar {
namespace {

constexpr int SA_THREADS = 256;
constexpr int SA_J = 4;
constexpr int SA_TW = SA_THREADS * SA_J;
constexpr int SA_SPAN_CAP = 4096;
constexpr int SA_KC = 256;
constexpr size_t SA_SMEM = sizeof(float2) * (SA_TW + SA_SPAN_CAP) + SA_KC * (sizeof(float2) + sizeof(int));

__device__ __forceinline__ int canon_offset(int o, int n) {
    int c = pmod(o, n);
    return (c > n / 2) ? c - n : c;
}

__global__ void __launch_bounds__(SA_THREADS)
sparse_azimuth_kernel(const float2 *__restrict__ S, const float2 *__restrict__ w, const int32_t *__restrict__ o,
                      int o_row_stride, int n_az, int K, float2 *__restrict__ out) {
    extern __shared__ float2 sm[];
    float2 *win = sm;                                   // [TW + SPAN_CAP]
    float2 *wk = sm + SA_TW + SA_SPAN_CAP;              // [KC]
    int *rel = reinterpret_cast<int *>(wk + SA_KC);     // [KC]
    __shared__ int red_lo[SA_THREADS / 32], red_hi[SA_THREADS / 32];

    const int r = blockIdx.y;
    const int th0 = blockIdx.x * SA_TW;
    const int tid = threadIdx.x;
    const float2 *Srow = S + (size_t)r * n_az;
    const float2 *wrow = w + (size_t)r * K;
    const int32_t *orow = o + (size_t)r * o_row_stride;

    // span of the canonical offsets
    int lo = INT_MAX, hi = INT_MIN;
    for (int k = tid; k < K; k += SA_THREADS) {
        const int c = canon_offset(__ldg(orow + k), n_az);
        lo = min(lo, c);
        hi = max(hi, c);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s));
    }
    if ((tid & 31) == 0) {
        red_lo[tid >> 5] = lo;
        red_hi[tid >> 5] = hi;
    }
    __syncthreads();
    lo = red_lo[0];
    hi = red_hi[0];
#pragma unroll
    for (int i = 1; i < SA_THREADS / 32; ++i) {
        lo = min(lo, red_lo[i]);
        hi = max(hi, red_hi[i]);
    }
    const int span = hi - lo;
    const bool staged = span <= SA_SPAN_CAP;
    const int tw = min(SA_TW, n_az - th0);

    if (staged) {
        const int wlen = tw + span;
        const int start = pmod(th0 + lo, n_az);
        for (int i = tid; i < wlen; i += SA_THREADS) {
            int idx = start + i;
            if (idx >= n_az) idx %= n_az;
            win[i] = __ldg(Srow + idx);
        }
    }

    float2 acc[SA_J];
#pragma unroll
    for (int j = 0; j < SA_J; ++j) acc[j] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < K; k0 += SA_KC) {
        const int kc = min(SA_KC, K - k0);
        __syncthreads();   // window staged / previous chunk consumed
        for (int i = tid; i < kc; i += SA_THREADS) {
            wk[i] = __ldg(wrow + k0 + i);
            const int c = canon_offset(__ldg(orow + k0 + i), n_az);
            rel[i] = staged ? c - lo : c;
        }
        __syncthreads();
        if (staged) {
#pragma unroll 4
            for (int i = 0; i < kc; ++i) {
                const float2 wv = wk[i];
                const float2 *src = win + rel[i] + tid;
#pragma unroll
                for (int j = 0; j < SA_J; ++j) cmac(acc[j], wv, src[j * SA_THREADS]);
            }
        } else {
            for (int i = 0; i < kc; ++i) {
                const float2 wv = wk[i];
                const int c = rel[i];
#pragma unroll
                for (int j = 0; j < SA_J; ++j) {
                    const int th = th0 + tid + j * SA_THREADS;
                    if (th < n_az) cmac(acc[j], wv, __ldg(Srow + pmod(th + c, n_az)));
                }
            }
        }
    }
    float2 *orow_out = out + (size_t)r * n_az;
#pragma unroll
    for (int j = 0; j < SA_J; ++j) {
        const int th = th0 + tid + j * SA_THREADS;
        if (th < n_az) orow_out[th] = acc[j];
    }
}

}  // namespace

rosar_status launch_sparse_azimuth(const float2 *S, const float2 *w, const int32_t *o, int o_row_stride, int n_rng,
                                   int n_az, int K, float2 *out, cudaStream_t s) {
    static unsigned long long done = 0;
    rosar_status st = ensure_smem((const void *)sparse_azimuth_kernel, SA_SMEM, &done, "sparse_azimuth");
    if (st != ROSAR_OK) return st;
    if (n_rng > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth: n_rng=%d exceeds 65535", n_rng);
    dim3 grid((n_az + SA_TW - 1) / SA_TW, n_rng);
    sparse_azimuth_kernel<<<grid, SA_THREADS, SA_SMEM, s>>>(S, w, o, o_row_stride, n_az, K, out);
    return check_launch("sparse_azimuth");
}

}  // namespace rosar
