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

// Range-migration-aware tiles stage one window per row the taps reach (up to MIG_ROWS rows in a buffer of
// WIN elements) and keep each tap's row offset.
constexpr int MIG_ROWS = 4;
template <int J>
struct GeoMig {
    static constexpr int TW = THREADS * J;
    static constexpr int WIN = 2 * (TW + SPAN_CAP);
    static constexpr int SMEM_BYTES = (int)(sizeof(float2) * WIN + KC * (sizeof(float2) + 2 * sizeof(int)));
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

// `smem` holds Geo<J>::SMEM_BYTES bytes (GeoMig<J> when MIG); `red` 4*THREADS/32 ints.  Called by all
// 256 threads.
// ADJ: the adjoint in S, out[r][n] = sum_k conj(w[r][k]) * S[r][(n - o_k) mod n_az] (conjugated weights,
// negated offsets), which is the scatter-add of the forward filter written as a gather.
// MIG: range-migration-aware taps, out[r][t] = sum_k w[r][k] * S[r + dl[r][k]][(t + o_k) mod n_az] with S
// holding n_bins rows (rows outside read zero): the windows of rows r + min(dl) .. r + max(dl) are staged
// back to back and each tap's row folds into its shared-memory offset, so the inner loop is unchanged.
template <int J, bool COHERENT, bool ADJ = false, bool MIG = false>
__device__ __forceinline__ void azimuth_tile(const float2 *__restrict__ S, const float2 *__restrict__ w,
                                             const int32_t *__restrict__ o, int o_row_stride, int n_az, int K,
                                             float2 *__restrict__ out, int r, int th0, char *smem, int *red,
                                             const int32_t *__restrict__ dl = nullptr, int n_bins = 0) {
    static_assert(!(ADJ && MIG), "the migrating filter has no adjoint here");
    constexpr int TW = Geo<J>::TW;
    constexpr int WIN = MIG ? GeoMig<J>::WIN : TW + SPAN_CAP;
    float2 *win = reinterpret_cast<float2 *>(smem);        // [WIN]
    float2 *wk = win + WIN;                                // [KC]
    int *rel = reinterpret_cast<int *>(wk + KC);           // [KC]
    int *dk = rel + KC;                                    // [KC] (MIG) row offset of each staged tap
    int *red_lo = red, *red_hi = red + THREADS / 32, *red_dlo = red + 2 * THREADS / 32, *red_dhi = red + 3 * THREADS / 32;

    const int tid = threadIdx.x;
    const float2 *wrow = w + (size_t)r * K;
    const int32_t *orow = o + (size_t)r * o_row_stride;
    const int32_t *drow = MIG ? dl + (size_t)r * K : nullptr;

    // span of the canonical offsets (and of the row offsets)
    int lo = INT_MAX, hi = INT_MIN, dlo = INT_MAX, dhi = INT_MIN;
    for (int k = tid; k < K; k += THREADS) {
        const int c = tap_offset<ADJ>(orow + k, n_az);
        lo = min(lo, c);
        hi = max(hi, c);
        if (MIG) {
            const int d = __ldg(drow + k);
            dlo = min(dlo, d);
            dhi = max(dhi, d);
        }
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s));
        if (MIG) {
            dlo = min(dlo, __shfl_xor_sync(0xffffffffu, dlo, s));
            dhi = max(dhi, __shfl_xor_sync(0xffffffffu, dhi, s));
        }
    }
    if ((tid & 31) == 0) {
        red_lo[tid >> 5] = lo;
        red_hi[tid >> 5] = hi;
        if (MIG) {
            red_dlo[tid >> 5] = dlo;
            red_dhi[tid >> 5] = dhi;
        }
    }
    __syncthreads();
    lo = red_lo[0];
    hi = red_hi[0];
    if (MIG) {
        dlo = red_dlo[0];
        dhi = red_dhi[0];
    }
#pragma unroll
    for (int i = 1; i < THREADS / 32; ++i) {
        lo = min(lo, red_lo[i]);
        hi = max(hi, red_hi[i]);
        if (MIG) {
            dlo = min(dlo, red_dlo[i]);
            dhi = max(dhi, red_dhi[i]);
        }
    }
    const int span = hi - lo;
    const int tw = min(TW, n_az - th0);
    // rows are laid out at the full-tile stride TW + span, so that lanes past a ragged tile's end (whose
    // outputs are discarded) still read inside the window: max index (nrows-1)*wl + span + TW-1 < nrows*wl
    const int wl = TW + span;
    const long long nrows = MIG ? (long long)dhi - dlo + 1 : 1;
    const bool staged = MIG ? (span <= SPAN_CAP && nrows <= MIG_ROWS && nrows * wl <= WIN) : span <= SPAN_CAP;

    if (staged) {
        const int start = pmod(th0 + lo, n_az);
        for (int q = 0; q < (int)nrows; ++q) {
            const long long row = MIG ? (long long)r + dlo + q : r;
            const bool live = !MIG || (row >= 0 && row < n_bins);
            const float2 *Srow = S + (live ? (size_t)row * n_az : 0);
            for (int i = tid; i < tw + span; i += THREADS) {
                int idx = start + i;
                if (idx >= n_az) idx %= n_az;
                win[q * wl + i] = live ? load_s<COHERENT>(Srow + idx) : make_float2(0.f, 0.f);
            }
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
            const int d = MIG ? __ldg(drow + k0 + i) : 0;
            if (MIG) dk[i] = d;
            rel[i] = staged ? (MIG ? (d - dlo) * wl : 0) + c - lo : c;
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
                const long long row = MIG ? (long long)r + dk[i] : r;
                if (MIG && (row < 0 || row >= n_bins)) continue;
                const float2 *Srow = S + (size_t)row * n_az;
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
