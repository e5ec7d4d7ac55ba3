// Mixed-radix row FFT used by the frequency-domain azimuth filter (azimuth_fft.cu), the
// pipelined multi-scan stage kernel (image_pipeline.cu) and the batched persistent kernel
// (batch.cu): in-place decimation-in-frequency forward transform (digit-reversed output) and
// its transposed decimation-in-time sequence, radices 16, 8, 4, 2, 5, 3 and a prime-factor 15.
// The pass functions run on the whole CTA (blockDim.x threads, any count) and end with a barrier
// (row_filter_fused and dit_last_global, whose last pass writes global memory, do not).
#pragma once

#include <map>
#include <mutex>
#include <vector>

#include "fft_tile.cuh"

namespace rosar {
namespace rowfft {


constexpr int AF_MAX_N = 16384;
constexpr int AF_MAXPASS = 16;

struct RowPlan {
    int npass;
    int pad_shift;            // shared-memory padding: one element per 2^pad_shift (31 = none)
    int rad[AF_MAXPASS];
};

// Padding: one element per 16 for power-of-two rows (whose late passes have power-of-two strides), none
// for rows with an odd factor: their plan puts the power-of-two radix first, where accesses are
// contiguous, and padding would scramble the odd strides of the later passes.
__host__ __device__ constexpr int pad_shift_for(int n) { return (n & (n - 1)) == 0 ? 4 : 31; }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> pad_shift_for(n)) + 1; }
__host__ __device__ constexpr int coarse_len(int n) { return n / 64 + 1; }

// Forward DFT of size R on v[0..R), natural-order output.
template <int R>
__device__ __forceinline__ void small_dft(float2 *v);

template <>
__device__ __forceinline__ void small_dft<2>(float2 *v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void small_dft<3>(float2 *v) {
    constexpr float h = 0.86602540378443865f;   // sin(2*pi/3)
    const float2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    const float2 y0 = cadd(v[0], t1);
    const float2 a = caxpy(-0.5f, t1, v[0]);                     // y1 = a - i h t2, y2 = a + i h t2
    v[0] = y0;
    v[1] = make_float2(fmaf(h, t2.y, a.x), fmaf(-h, t2.x, a.y));
    v[2] = make_float2(fmaf(-h, t2.y, a.x), fmaf(h, t2.x, a.y));
}

template <>
__device__ __forceinline__ void small_dft<4>(float2 *v) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = make_float2(d02.x + d13.y, d02.y - d13.x);          // d02 - i d13
    v[3] = make_float2(d02.x - d13.y, d02.y + d13.x);          // d02 + i d13
}

template <>
__device__ __forceinline__ void small_dft<5>(float2 *v) {
    constexpr float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos(2pi/5), cos(4pi/5)
    constexpr float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin(2pi/5), sin(4pi/5)
    const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    const float2 x0 = v[0];
    const float2 a1 = caxpy(c1, t1, caxpy(c2, t2, x0));
    const float2 a2 = caxpy(c2, t1, caxpy(c1, t2, x0));
    const float2 b1 = caxpy(s1, t3, cscale(t4, s2));
    const float2 b2 = caxpy(s2, t3, cscale(t4, -s1));
    v[0] = cadd(cadd(x0, t1), t2);
    v[1] = make_float2(a1.x + b1.y, a1.y - b1.x);              // a1 - i b1
    v[4] = make_float2(a1.x - b1.y, a1.y + b1.x);              // a1 + i b1
    v[2] = make_float2(a2.x + b2.y, a2.y - b2.x);              // a2 - i b2
    v[3] = make_float2(a2.x - b2.y, a2.y + b2.x);              // a2 + i b2
}

// 15 = 3 x 5 by the prime-factor (Good-Thomas) index maps, which need no twiddles between the two sets of
// small DFTs: input n = (5 n1 + 3 n2) mod 15, output k = (10 k1 + 6 k2) mod 15 (10 = 1 mod 3 and 0 mod 5,
// 6 = 0 mod 3 and 1 mod 5), so that W_15^(nk) = W_3^(n1 k1) W_5^(n2 k2).
template <>
__device__ __forceinline__ void small_dft<15>(float2 *v) {
    float2 a[5][3];
#pragma unroll
    for (int n2 = 0; n2 < 5; ++n2)
#pragma unroll
        for (int n1 = 0; n1 < 3; ++n1) a[n2][n1] = v[(5 * n1 + 3 * n2) % 15];
#pragma unroll
    for (int n2 = 0; n2 < 5; ++n2) small_dft<3>(a[n2]);
    float2 b[3][5];
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
        for (int n2 = 0; n2 < 5; ++n2) b[k1][n2] = a[n2][k1];
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) small_dft<5>(b[k1]);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 5; ++k2) v[(10 * k1 + 6 * k2) % 15] = b[k1][k2];
}

template <int R>
__device__ __forceinline__ void pow2_dft(float2 *v) {
    fft::dft_dif<R>(v);                     // output index r sits at v[brev(r)]
    float2 t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) t[r] = v[fft::brev(r, fft::ilog2(R))];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = t[r];
}

template <>
__device__ __forceinline__ void small_dft<8>(float2 *v) { pow2_dft<8>(v); }

template <>
__device__ __forceinline__ void small_dft<16>(float2 *v) { pow2_dft<16>(v); }

__device__ __forceinline__ int rpad(int e, int sh) { return e + (e >> sh); }

// Compile-time padding for the passes: PAD = one element per 16, else none.
template <bool PAD>
__device__ __forceinline__ int cpad(int e) { return PAD ? e + (e >> 4) : e; }

// floor(i / s) for 0 <= i < 2^23 and 1 <= s <= 2^14, from inv_s = 1/s rounded to float: (i + 1/2)/s is at
// least 1/(2s) away from an integer while the float product errs by at most about i * 2^-23 / s.
__device__ __forceinline__ int quot(int i, float inv_s) { return __float2int_rz(__fmul_rn((float)i + 0.5f, inv_s)); }

__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int G>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(G) : "memory"); }

// exp(-2*pi*i*q/N), 0 <= q < N: from the full table (tc == nullptr: tf holds all N entries) or from
// the coarse (q >> 6) and fine (q & 63) tables.
__device__ __forceinline__ float2 twiddle(int q, const float2 *tc, const float2 *tf) {
    return tc ? cmul(tc[q >> 6], tf[q & 63]) : tf[q];
}

using fft::twiddle_powers;

// One in-place decimation-in-frequency stage: radix R on blocks of length M (stride s = M/R):
// v = DFT_R(x[base + r*s]); x[base + q*s] = v[q] * W_M^(j*q).
template <int R, bool PAD>
__device__ __forceinline__ void dif_pass(float2 *x, int N, int M, const float2 *tc, const float2 *tf) {
    const int s = M / R, tstep = N / M, nb = N / R, nblk = N / M;
    const bool by_blk = !PAD && nblk >= 16 && (M & 1);     // as butterfly_index: odd lane strides
    const float inv_d = 1.f / (float)(by_blk ? nblk : s);
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int q = quot(idx, inv_d);
        const int blk = by_blk ? idx - q * nblk : q, j = by_blk ? q : idx - q * s;
        const int base = blk * M + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[cpad<PAD>(base + r * s)];
        small_dft<R>(v);
        x[cpad<PAD>(base)] = v[0];
        float2 wq[R];
        twiddle_powers<R>(twiddle(j * tstep, tc, tf), wq);
#pragma unroll
        for (int q = 1; q < R; ++q) x[cpad<PAD>(base + q * s)] = cmul(v[q], wq[q]);
    }
    __syncthreads();
}

// The transposed stage (decimation in time): v[q] = x[base + q*s] * W_M^(j*q); x[base + r*s] = DFT_R(v)[r].
template <int R, bool PAD>
__device__ __forceinline__ void dit_pass(float2 *x, int N, int M, const float2 *tc, const float2 *tf) {
    const int s = M / R, tstep = N / M, nb = N / R, nblk = N / M;
    const bool by_blk = !PAD && nblk >= 16 && (M & 1);     // as butterfly_index: odd lane strides
    const float inv_d = 1.f / (float)(by_blk ? nblk : s);
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int q = quot(idx, inv_d);
        const int blk = by_blk ? idx - q * nblk : q, j = by_blk ? q : idx - q * s;
        const int base = blk * M + j;
        float2 v[R];
        float2 wq[R];
        twiddle_powers<R>(twiddle(j * tstep, tc, tf), wq);
        v[0] = x[cpad<PAD>(base)];
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmul(x[cpad<PAD>(base + q * s)], wq[q]);
        small_dft<R>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) x[cpad<PAD>(base + r * s)] = v[r];
    }
    __syncthreads();
}

#define ROSAR_STAGE_CASE(RR) \
    case RR: DIF ? dif_pass<RR, PAD>(x, N, M, tc, tf) : dit_pass<RR, PAD>(x, N, M, tc, tf); break;

template <bool DIF, bool PAD>
__device__ __forceinline__ void stage(int R, float2 *x, int N, int M, const float2 *tc, const float2 *tf) {
    switch (R) {
        ROSAR_STAGE_CASE(16)
        ROSAR_STAGE_CASE(15)
        ROSAR_STAGE_CASE(8)
        ROSAR_STAGE_CASE(5)
        ROSAR_STAGE_CASE(4)
        ROSAR_STAGE_CASE(3)
        default: DIF ? dif_pass<2, PAD>(x, N, M, tc, tf) : dit_pass<2, PAD>(x, N, M, tc, tf); break;
    }
}
#undef ROSAR_STAGE_CASE

// Compile-time plans: the same passes for a row length N and a radix sequence fixed at compile time, run by
// exactly T threads.  Strides, block counts and the quotient by the stride become constants and the
// per-pass radix dispatch disappears; results are identical to the run-time plan with the same radices.
template <int... R>
struct Radices {};

// Butterfly idx of a pass with nblk = N/M blocks of s = M/R butterflies: blocks vary fastest across threads
// when there are at least 16 blocks of odd length M (the 16 lanes of a 64-bit shared-memory phase then stride
// by M: distinct bank pairs, and the lanes share one twiddle), else positions within a block vary fastest.
template <int N, int M, int R>
__device__ __forceinline__ void butterfly_index(int idx, int &blk, int &j) {
    constexpr int s = M / R, nblk = N / M;
    if constexpr (nblk >= 16 && (M & 1)) {
        j = idx / nblk;
        blk = idx - j * nblk;
    } else {
        blk = idx / s;
        j = idx - blk * s;
    }
}

template <int N, int M, int R, bool PAD, int T>
__device__ __forceinline__ void dif_pass_c(float2 *x, const float2 *tc, const float2 *tf) {
    constexpr int s = M / R, tstep = N / M, nb = N / R;
#pragma unroll 1
    for (int idx = threadIdx.x; idx < nb; idx += T) {
        int blk, j;
        butterfly_index<N, M, R>(idx, blk, j);
        const int base = blk * M + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[cpad<PAD>(base + r * s)];
        small_dft<R>(v);
        x[cpad<PAD>(base)] = v[0];
        float2 wq[R];
        twiddle_powers<R>(twiddle(j * tstep, tc, tf), wq);
#pragma unroll
        for (int q = 1; q < R; ++q) x[cpad<PAD>(base + q * s)] = cmul(v[q], wq[q]);
    }
    __syncthreads();
}

template <int N, int M, int R, bool PAD, int T>
__device__ __forceinline__ void dit_pass_c(float2 *x, const float2 *tc, const float2 *tf) {
    constexpr int s = M / R, tstep = N / M, nb = N / R;
#pragma unroll 1
    for (int idx = threadIdx.x; idx < nb; idx += T) {
        int blk, j;
        butterfly_index<N, M, R>(idx, blk, j);
        const int base = blk * M + j;
        float2 v[R];
        float2 wq[R];
        twiddle_powers<R>(twiddle(j * tstep, tc, tf), wq);
        v[0] = x[cpad<PAD>(base)];
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmul(x[cpad<PAD>(base + q * s)], wq[q]);
        small_dft<R>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) x[cpad<PAD>(base + r * s)] = v[r];
    }
    __syncthreads();
}

// DIF passes in plan order, the block length M shrinking by each radix.
template <int N, int M, bool PAD, int T, int R, int... Rest>
__device__ __forceinline__ void dif_seq(float2 *x, const float2 *tc, const float2 *tf) {
    dif_pass_c<N, M, R, PAD, T>(x, tc, tf);
    if constexpr (sizeof...(Rest) > 0) dif_seq<N, M / R, PAD, T, Rest...>(x, tc, tf);
}

// DIT passes in reverse plan order: the last radix first (M = that radix), the first radix last (M = N).
template <int N, int M, bool PAD, int T, int R, int... Rest>
__device__ __forceinline__ void dit_seq(float2 *x, const float2 *tc, const float2 *tf) {
    if constexpr (sizeof...(Rest) > 0) dit_seq<N, M / R, PAD, T, Rest...>(x, tc, tf);
    dit_pass_c<N, M, R, PAD, T>(x, tc, tf);
}

// The whole row filter conj(DIT(conj(H . DIF(src)))) with the first and last passes on global memory and the
// last forward pass, the product with H and the first inverse pass fused into one step: per element four
// shared-memory round trips fewer than loading the row, running dif_seq, multiplying and running dit_seq, with
// the same arithmetic (the two fused passes act on blocks of one butterfly, whose twiddles are 1).

// First DIF pass (M = N, stride s = N/R) with its inputs read from global memory (ld.cg: src may have been
// written earlier by the same kernel).  WAIT_ASYNC: the thread's cp.async copies (the H row) complete before
// the closing barrier, so they are visible to the whole CTA after it.  discard: src is scratch that nothing
// reads again, so after the barrier (every element has been read) the 128-byte L2 lines lying wholly inside
// the row are dropped without being written back to memory; the lines it shares with neighbouring rows stay.
// phase (optional, [N]): element n is multiplied by phase[n] as it is loaded (the per-pulse phase correction
// of the differentiable form, S e^{j eps_n}, without a corrected copy of S in memory).
template <int N, int R, int T, bool WAIT_ASYNC>
__device__ __forceinline__ void dif_first_global(const float2 *__restrict__ src, float2 *x, const float2 *tc,
                                                 const float2 *tf, bool discard = false,
                                                 const float2 *__restrict__ phase = nullptr) {
    constexpr int s = N / R;
#pragma unroll 1
    for (int j = threadIdx.x; j < s; j += T) {
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = __ldcg(src + j + r * s);
        if (phase) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = cmul(v[r], __ldg(phase + j + r * s));
        }
        small_dft<R>(v);
        x[j] = v[0];
        float2 wq[R];
        twiddle_powers<R>(twiddle(j, tc, tf), wq);
#pragma unroll
        for (int q = 1; q < R; ++q) x[j + q * s] = cmul(v[q], wq[q]);
    }
    if (WAIT_ASYNC) cp_async_wait<0>();
    __syncthreads();
    if (discard) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(src);
        const uintptr_t first = (a + 127) & ~(uintptr_t)127, end = (a + sizeof(float2) * (size_t)N) & ~(uintptr_t)127;
        for (uintptr_t l = first + 128 * (uintptr_t)threadIdx.x; l < end; l += 128 * (uintptr_t)T)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(l) : "memory");
    }
}

// Last forward pass (blocks of R, stride 1), y = conj(H . X) (conj(H) . X conjugated when hs = -1), and the
// first pass of the inverse on the same block.  H is in the forward transform's digit-reversed order; h is
// shared memory (H_SMEM) or global.
// spec (optional): the row's forward transform (before the product with H) is also written there, radix-major:
// element r of block b (digit-reversed position b*R + r) at spec[r*(N/R) + b], so that a warp's stores of one r
// are consecutive.
template <int N, int R, int T, bool H_SMEM>
__device__ __forceinline__ void fused_mid(float2 *x, const float2 *h, float hs, float2 *__restrict__ spec = nullptr) {
    constexpr int nb = N / R;
#pragma unroll 1
    for (int b = threadIdx.x; b < nb; b += T) {
        const int base = b * R;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[base + r];
        small_dft<R>(v);
        if (spec) {
#pragma unroll
            for (int r = 0; r < R; ++r) spec[r * nb + b] = v[r];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 hv = H_SMEM ? h[base + r] : __ldg(h + base + r);
            hv.y *= hs;
            const float2 y = cmul(hv, v[r]);
            v[r] = make_float2(y.x, -y.y);
        }
        small_dft<R>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) x[base + r] = v[r];
    }
    __syncthreads();
}

// Last DIT pass (M = N) written to global memory with the final conjugation of the inverse.
template <int N, int R, int T>
__device__ __forceinline__ void dit_last_global(const float2 *x, float2 *__restrict__ dst, const float2 *tc,
                                                const float2 *tf) {
    constexpr int s = N / R;
#pragma unroll 1
    for (int j = threadIdx.x; j < s; j += T) {
        float2 v[R], wq[R];
        twiddle_powers<R>(twiddle(j, tc, tf), wq);
        v[0] = x[j];
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmul(x[j + q * s], wq[q]);
        small_dft<R>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[j + r * s] = make_float2(v[r].x, -v[r].y);
    }
}

template <int N, int M, int T, bool H_SMEM, int R, int... Rest>
__device__ __forceinline__ void filter_middle(float2 *x, const float2 *h, float hs, const float2 *tc, const float2 *tf,
                                              float2 *__restrict__ spec = nullptr) {
    if constexpr (sizeof...(Rest) == 0) {
        static_assert(M == R, "the last radix spans the last block");
        fused_mid<N, R, T, H_SMEM>(x, h, hs, spec);
    } else {
        dif_pass_c<N, M, R, false, T>(x, tc, tf);
        filter_middle<N, M / R, T, H_SMEM, Rest...>(x, h, hs, tc, tf, spec);
        dit_pass_c<N, M, R, false, T>(x, tc, tf);
    }
}

// src, dst: the row in global memory (natural order); x: N elements of shared memory (no padding); the
// caller has built the twiddle table and synchronised.  With H_SMEM, h may still be arriving by cp.async
// when this starts (waited for at the end of the first pass).  No barrier at the end.  discard: src is
// scratch, dropped from L2 once read (dif_first_global).
template <int N, int T, bool H_SMEM, int R1, int... Rs>
__device__ __forceinline__ void row_filter_fused(const float2 *__restrict__ src, const float2 *h, float hs, float2 *x,
                                                 float2 *__restrict__ dst, const float2 *tc, const float2 *tf,
                                                 bool discard = false, const float2 *__restrict__ phase = nullptr,
                                                 float2 *__restrict__ spec = nullptr) {
    static_assert(sizeof...(Rs) >= 1, "at least two passes");
    dif_first_global<N, R1, T, H_SMEM>(src, x, tc, tf, discard, phase);
    filter_middle<N, N / R1, T, H_SMEM, Rs...>(x, h, hs, tc, tf, spec);
    dit_last_global<N, R1, T>(x, dst, tc, tf);
}

// Forward DFT of the row, output in digit-reversed order.
template <bool PAD>
__device__ __forceinline__ void row_dif_t(float2 *x, int N, const RowPlan &pl, const float2 *tc, const float2 *tf) {
    int M = N;
    for (int p = 0; p < pl.npass; ++p) {
        stage<true, PAD>(pl.rad[p], x, N, M, tc, tf);
        M /= pl.rad[p];
    }
}

__device__ __forceinline__ void row_dif(float2 *x, int N, const RowPlan &pl, const float2 *tc, const float2 *tf) {
    if (pl.pad_shift == 4) row_dif_t<true>(x, N, pl, tc, tf);
    else row_dif_t<false>(x, N, pl, tc, tf);
}

// Forward DFT of a row held in digit-reversed order, output in natural order.
template <bool PAD>
__device__ __forceinline__ void row_dit_t(float2 *x, int N, const RowPlan &pl, const float2 *tc, const float2 *tf) {
    int M = 1;
    for (int p = pl.npass - 1; p >= 0; --p) {
        M *= pl.rad[p];
        stage<false, PAD>(pl.rad[p], x, N, M, tc, tf);
    }
}

__device__ __forceinline__ void row_dit(float2 *x, int N, const RowPlan &pl, const float2 *tc, const float2 *tf) {
    if (pl.pad_shift == 4) row_dit_t<true>(x, N, pl, tc, tf);
    else row_dit_t<false>(x, N, pl, tc, tf);
}

// Full table (tc == nullptr on return): tw[q] = exp(-2*pi*i*q/N), q < N.  Two-level: tw[0..64) fine, then coarse.
__device__ __forceinline__ void build_twiddles(int N, bool full, float2 *tw, const float2 **tc, const float2 **tf) {
    if (full) {
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
            float s, c;
            sincospif(2.f * (float)q / (float)N, &s, &c);
            tw[q] = make_float2(c, -s);
        }
        *tc = nullptr;
        *tf = tw;
        return;
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        float s, c;
        sincospif(2.f * (float)i / (float)N, &s, &c);
        tw[i] = make_float2(c, -s);
    }
    for (int i = threadIdx.x; i < coarse_len(N); i += blockDim.x) {
        float s, c;
        sincospif(2.f * (float)(64 * i) / (float)N, &s, &c);
        tw[64 + i] = make_float2(c, -s);
    }
    *tc = tw + 64;
    *tf = tw;
}


// One row of the azimuth filter on one CTA of T threads with a compile-time plan (N with an odd factor):
// stage the H row (cp.async; H_SMEM) and the twiddle table, wait for the predecessor grid (S is complete), run
// row_filter_fused.  sm: (H_SMEM ? 2 : 1) (N + 1) + 64 + coarse_len(N) float2 of shared memory
// (filter_row_smem); without H_SMEM the fused middle step reads H from global memory (rows too long to
// stage two of them).
template <int N, bool H_SMEM = true>
constexpr size_t filter_row_smem() {
    return sizeof(float2) * (size_t)((H_SMEM ? 2 : 1) * padded_len(N) + 64 + coarse_len(N));
}

template <int T, int N, bool H_SMEM, int... R>
__device__ __forceinline__ void filter_row_cta(const float2 *__restrict__ S_row, const float2 *__restrict__ H_row,
                                               bool conj_h, float2 *__restrict__ out_row, float2 *sm,
                                               const float2 *__restrict__ phase = nullptr,
                                               float2 *__restrict__ spec = nullptr) {
    static_assert(pad_shift_for(N) == 31, "compile-time filter plans are for rows with an odd factor");
    float2 *x = sm;
    float2 *hb = x + padded_len(N);
    float2 *tw = H_SMEM ? hb + padded_len(N) : hb;
    if (H_SMEM) {
        for (int n = threadIdx.x; n < N; n += T) cp_async8(hb + n, H_row + n);   // waited for after the first pass
        cp_async_commit();
    }
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    __syncthreads();
    griddep_wait();                          // S is complete (no-op unless launched to overlap its producer)
    row_filter_fused<N, T, H_SMEM, R...>(S_row, H_SMEM ? hb : H_row, conj_h ? -1.f : 1.f, x, out_row, tc, tf, false,
                                         phase, spec);
}

inline int threads_for(int N) { return N <= 4096 ? 256 : N <= 8192 ? 512 : 1024; }

// Radix sequence for N over radices {16, 8, 4, 2, 5, 3, 15}: fewest passes, then fewest butterflies per thread
// (the first radix found wins a tie).  15 is a prime-factor butterfly without inner twiddles, so a row with
// a factor 225 takes two passes for it instead of four: 3600 = 16.15.15, 1800 = 8.15.15, 7200 = 8.4.15.15.
inline bool make_plan(int N, RowPlan *pl) {
    static const int kRad[] = {16, 8, 4, 2, 5, 3, 15};
    if (N < 2 || N > AF_MAX_N) return false;
    static std::mutex mu;
    static std::map<int, RowPlan> cache;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(N);
        if (it != cache.end()) {
            *pl = it->second;
            return pl->npass > 0;
        }
    }
    const int T = threads_for(N);
    // dynamic programme over the divisors m of N: best[m] = (passes, iterations) to transform the remaining factor m
    std::map<int, std::pair<std::pair<int, int>, int>> best;   // m -> ((passes, iters), first radix)
    std::vector<int> divs;
    for (int d = 1; d <= N; ++d)
        if (N % d == 0) divs.push_back(d);
    best[1] = {{0, 0}, 0};
    for (int m : divs) {
        if (m == 1) continue;
        std::pair<int, int> b = {1 << 30, 1 << 30};
        int br = 0;
        for (int R : kRad) {
            if (m % R) continue;
            auto it = best.find(m / R);
            if (it == best.end() || it->second.first.first >= (1 << 30)) continue;
            const int iters = (N / R + T - 1) / T;
            std::pair<int, int> c = {it->second.first.first + 1, it->second.first.second + iters};
            if (c < b) {
                b = c;
                br = R;
            }
        }
        best[m] = {b, br};
    }
    RowPlan p{};
    p.pad_shift = pad_shift_for(N);
    int m = N, np = 0;
    bool ok = best[N].second != 0;
    while (ok && m > 1 && np < AF_MAXPASS) {
        const int R = best[m].second;
        if (R == 0) { ok = false; break; }
        p.rad[np++] = R;
        m /= R;
    }
    p.npass = (ok && m == 1) ? np : 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        cache[N] = p;
    }
    *pl = p;
    return p.npass > 0;
}


}  // namespace rowfft
}  // namespace rosar
