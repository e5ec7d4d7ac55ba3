// Gather-MAC tile of the sparse-aperture azimuth matched filter
// (arXiv 2309.08038, Sec. III-D, Eq. (43); Algorithm 2):
//
//   out[r][theta] = sum_{k<K} w[r][k] * S[r][(theta + o_k) mod n_az],  theta0 <= theta < theta0 + 256*J
//
// The CTA (256 threads) first reduces its row's offsets to a canonical representative
// in [-n_az/2, n_az/2] and finds their span [lo, hi]; it then stages the circular
// window S[r][theta0+lo .. theta0+TW-1+hi] in shared memory with coalesced loads
// (wrap handled at staging, so the inner loop has no modulo).  Each thread owns J
// outputs strided by the block size, so for every tap the warp reads 32 consecutive
// window entries (conflict-free) while the tap's weight and relative offset are
// shared-memory broadcasts.  Taps are staged in chunks of KC and accumulated in
// float32 in increasing k.  A row whose offsets span more than SPAN_CAP pulses
// falls back to direct gathers with an explicit modulo.
#pragma once

#include <limits.h>

#include "rosar_internal.cuh"

namespace rosar {
namespace az {

constexpr int THREADS = 256;
constexpr int SPAN_CAP = 2560;
constexpr int KC = 256;

template <int J>
struct Geo {
    static constexpr int TW = THREADS * J;
    static constexpr int SMEM_BYTES = (int)(sizeof(float2) * (TW + SPAN_CAP) + KC * (sizeof(float2) + sizeof(int)));
};

__device__ __forceinline__ int canon_offset(int o, int n) {
    int c = pmod(o, n);
    return (c > n / 2) ? c - n : c;
}

// Offset of tap k as the tile uses it: o_k, or -o_k for the adjoint (transposed gather).
template <bool ADJ>
__device__ __forceinline__ int tap_offset(const int32_t *o, int n) {
    const int v = __ldg(o);
    if (!ADJ) return canon_offset(v, n);
    const long long m = (-(long long)v) % n;      // -INT_MIN does not fit an int
    return canon_offset((int)m, n);
}

// COHERENT: S was written earlier in the same kernel (read through L2, not the non-coherent path).
template <bool COHERENT>
__device__ __forceinline__ float2 load_s(const float2 *p) {
    if (COHERENT) return __ldcg(p);
    return __ldg(p);
}

// `smem` holds Geo<J>::SMEM_BYTES bytes; `red` 2*THREADS/32 ints.  Called by all 256 threads.
// ADJ: the adjoint in S, out[r][n] = sum_k conj(w[r][k]) * S[r][(n - o_k) mod n_az] (conjugated weights,
// negated offsets), which is the scatter-add of the forward filter written as a gather.
template <int J, bool COHERENT, bool ADJ = false>
__device__ __forceinline__ void azimuth_tile(const float2 *__restrict__ S, const float2 *__restrict__ w,
                                             const int32_t *__restrict__ o, int o_row_stride, int n_az, int K,
                                             float2 *__restrict__ out, int r, int th0, char *smem, int *red) {
    constexpr int TW = Geo<J>::TW;
    float2 *win = reinterpret_cast<float2 *>(smem);        // [TW + SPAN_CAP]
    float2 *wk = win + TW + SPAN_CAP;                      // [KC]
    int *rel = reinterpret_cast<int *>(wk + KC);           // [KC]
    int *red_lo = red, *red_hi = red + THREADS / 32;

    const int tid = threadIdx.x;
    const float2 *Srow = S + (size_t)r * n_az;
    const float2 *wrow = w + (size_t)r * K;
    const int32_t *orow = o + (size_t)r * o_row_stride;

    // span of the canonical offsets
    int lo = INT_MAX, hi = INT_MIN;
    for (int k = tid; k < K; k += THREADS) {
        const int c = tap_offset<ADJ>(orow + k, n_az);
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
    for (int i = 1; i < THREADS / 32; ++i) {
        lo = min(lo, red_lo[i]);
        hi = max(hi, red_hi[i]);
    }
    const int span = hi - lo;
    const bool staged = span <= SPAN_CAP;
    const int tw = min(TW, n_az - th0);

    if (staged) {
        const int wlen = tw + span;
        const int start = pmod(th0 + lo, n_az);
        for (int i = tid; i < wlen; i += THREADS) {
            int idx = start + i;
            if (idx >= n_az) idx %= n_az;
            win[i] = load_s<COHERENT>(Srow + idx);
        }
    }

    float2 acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < K; k0 += KC) {
        const int kc = min(KC, K - k0);
        __syncthreads();   // window staged / previous chunk consumed
        for (int i = tid; i < kc; i += THREADS) {
            const float2 wv = __ldg(wrow + k0 + i);
            wk[i] = ADJ ? cconj(wv) : wv;
            const int c = tap_offset<ADJ>(orow + k0 + i, n_az);
            rel[i] = staged ? c - lo : c;
        }
        __syncthreads();
        if (staged) {
#pragma unroll 4
            for (int i = 0; i < kc; ++i) {
                const float2 wv = wk[i];
                const float2 *src = win + rel[i] + tid;
#pragma unroll
                for (int j = 0; j < J; ++j) cmac(acc[j], wv, src[j * THREADS]);
            }
        } else {
            for (int i = 0; i < kc; ++i) {
                const float2 wv = wk[i];
                const int c = rel[i];
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int th = th0 + tid + j * THREADS;
                    if (th < n_az) cmac(acc[j], wv, load_s<COHERENT>(Srow + pmod(th + c, n_az)));
                }
            }
        }
    }
    float2 *orow_out = out + (size_t)r * n_az;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int th = th0 + tid + j * THREADS;
        if (th < n_az) orow_out[th] = acc[j];
    }
    __syncthreads();   // smem may be reused by the caller's next tile
}

}  // namespace az
}  // namespace rosar
