// Shared-memory radix-16 Stockham FFT tile used by the range-compression kernels
// (arXiv 2309.08038, Sec. III-D, Eq. (38)): window at load, centring phase
// c_l = exp(+j*pi*l*(L-1)/L) and the pulse-major -> range-major transpose at store.
#pragma once

#include "rosar_internal.cuh"

namespace rosar {
namespace fft {

// A raw sample is read once: through L2 without allocating in L1, which stays with the window and the data the
// other CTAs of the SM reuse.
__device__ __forceinline__ float2 ld_stream(const float2 *p) {
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

// exp(-2*pi*i*q/16) for compile-time q (after unrolling the switch folds away).
__device__ __forceinline__ float2 w16(int q) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
    switch (q & 15) {
        case 0: return make_float2(1.f, 0.f);
        case 1: return make_float2(c1, -s1);
        case 2: return make_float2(h, -h);
        case 3: return make_float2(s1, -c1);
        case 4: return make_float2(0.f, -1.f);
        case 5: return make_float2(-s1, -c1);
        case 6: return make_float2(-h, -h);
        case 7: return make_float2(-c1, -s1);
        case 8: return make_float2(-1.f, 0.f);
        case 9: return make_float2(-c1, s1);
        case 10: return make_float2(-h, h);
        case 11: return make_float2(-s1, c1);
        case 12: return make_float2(0.f, 1.f);
        case 13: return make_float2(s1, c1);
        case 14: return make_float2(h, h);
        default: return make_float2(c1, s1);
    }
}

__device__ __forceinline__ float2 twmul16(float2 d, int q) {
    q &= 15;
    if (q == 0) return d;
    if (q == 4) return make_float2(d.y, -d.x);
    if (q == 8) return make_float2(-d.x, -d.y);
    if (q == 12) return make_float2(-d.y, d.x);
    return cmul(d, w16(q));
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

__host__ __device__ constexpr int brev(int x, int bits) {
    int y = 0;
    for (int i = 0; i < bits; ++i) y |= ((x >> i) & 1) << (bits - 1 - i);
    return y;
}

// In-register radix-2 decimation-in-frequency DFT of size R <= 16 on v[0..R).
// Output index r ends up in v[brev(r)].
template <int R>
__device__ __forceinline__ void dft_dif(float2 *v) {
    constexpr int LG = ilog2(R);
#pragma unroll
    for (int s = 0; s < LG; ++s) {
        const int span = R >> (s + 1);
#pragma unroll
        for (int start = 0; start < R; start += 2 * span) {
#pragma unroll
            for (int i = 0; i < span; ++i) {
                const float2 a = v[start + i], b = v[start + i + span];
                v[start + i] = cadd(a, b);
                v[start + i + span] = twmul16(csub(a, b), i * (16 / (2 * span)));
            }
        }
    }
}

__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

// exp(-j*pi*q/L) for 0 <= q < 2L from a two-level table: tab[b] = exp(-j*pi*b/L) for b < 32 and
// tab[32 + a] = exp(-j*pi*32a/L); a product of two rounded factors (about 1.5 ulp).
__device__ __forceinline__ float2 half_twiddle(const float2 *tab, int q) {
    const float2 a = tab[32 + (q >> 5)], b = tab[q & 31];
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

template <int L>
__device__ __forceinline__ void build_half_twiddles(float2 *tab, int nthreads) {
    for (int i = threadIdx.x; i < 32 + (2 * L + 31) / 32; i += nthreads) {
        const int q = i < 32 ? i : 32 * (i - 32);
        float s, c;
        sincospif((float)q / (float)L, &s, &c);
        tab[i] = make_float2(c, -s);
    }
}

// wq[q] = w1^q for q = 0..R-1 by squaring and products (depth <= 4 multiplications: a few ulp of error).
// One table load per butterfly (w1, at a unit stride across threads) replaces R-1 strided loads that
// would pile onto few shared-memory banks.
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 w1, float2 (&wq)[R]) {
    wq[0] = make_float2(1.f, 0.f);
    if (R > 1) wq[1] = w1;
#pragma unroll
    for (int q = 2; q < R; ++q) wq[q] = (q & 1) ? cmul(wq[q - 1], w1) : cmul(wq[q / 2], wq[q / 2]);
}

// Geometry of a tile of P pulses of length L transformed by T*P threads.
template <int L, int P_>
struct Tile {
    static constexpr int P = P_;
    static constexpr int RM = L >= 16 ? 16 : L;       // elements per thread
    static constexpr int T = L / RM;                   // threads per pulse
    static constexpr int LG = ilog2(L);
    static constexpr int NF = L >= 16 ? LG / 4 : 0;    // full radix-16 passes
    static constexpr int RR = L >= 16 ? (L >> (4 * NF)) : 1;   // remainder radix (1 = none)
    static constexpr int LP = L + L / 16;              // padded per-pulse stride in the FFT buffer
    // row stride of the transposed tile: the last pass's stores tile[l*TP + p] hit 16 distinct 8-byte bank pairs per
    // half-warp (T threads per pulse: 16/T pulses of a half-warp differ by TP = 16/T mod 16; T >= 16: odd TP)
    static constexpr int TP = P + (T >= 16 ? 1 : 16 / T);
    static constexpr bool TP_EVEN = TP % 2 == 0;       // rows 16-byte aligned: pairs of pulses copied as float4
    static constexpr int BUF = (P * LP > L * TP) ? P * LP : L * TP;
    static constexpr int THREADS = T * P;
    static constexpr int TAB = 32 + ((2 * L + 31) / 32 + 1) / 2 * 2;   // two-level table, even (16-B alignment)
    static constexpr int SMEM_ELEMS = TAB + BUF;       // float2 elements: twiddle table + buffer
    static constexpr size_t SMEM = sizeof(float2) * (size_t)SMEM_ELEMS;
    static_assert(P % 2 == 0, "pulse tiles hold an even number of pulses");
};

// One Stockham pass of radix R (sub-transform size NS before the pass).
// FIRST: v already holds x[t + r*T] (loaded from HBM).  LAST: write the transposed tile.
template <int L, int P, int R, int NS, bool FIRST, bool LAST>
__device__ __forceinline__ void stockham_pass(float2 (&v)[Tile<L, P>::RM], int t, int p, float2 *pb, float2 *tile,
                                              const float2 *tab, bool centred) {
    using PL = Tile<L, P>;
    constexpr int RM = PL::RM, T = PL::T, NB = RM / R;
    if (!FIRST) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + b * T;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = pb[pad16(j + r * (L / R))];
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * T;
        const int k = j & (NS - 1);
        if (NS > 1) {
            float2 wq[R];
            twiddle_powers<R>(half_twiddle(tab, 2 * k * (L / (NS * R))), wq);   // W_{NS*R}^(r*k) = (W_{NS*R}^k)^r
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], wq[r]);
        }
        dft_dif<R>(v + b * R);
    }
    __syncthreads();   // every thread has read its inputs from the buffer (or the table is ready)
    if (!LAST) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + b * T;
            const int k = j & (NS - 1);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) pb[pad16(base + r * NS)] = v[b * R + brev(r, ilog2(R))];
        }
    } else {
        // last pass: NS*R == L, so j < NS and bin l = j + r*NS
        // centring c_l = (-1)^l exp(-j*pi*l/L) with exp(-j*pi*(j + r*NS)/L) = exp(-j*pi*j/L) * exp(-j*pi*NS/L)^r
        float2 sp[R];
        if (centred) twiddle_powers<R>(half_twiddle(tab, NS), sp);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + b * T;
            const float2 cj = centred ? half_twiddle(tab, j) : make_float2(1.f, 0.f);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l = j + r * NS;
                float2 y = v[b * R + brev(r, ilog2(R))];
                if (centred) {
                    const float2 c = r == 0 ? cj : cmul(cj, sp[r]);
                    y = cmul(y, (l & 1) ? make_float2(-c.x, -c.y) : c);
                }
                tile[l * PL::TP + p] = y;
            }
        }
    }
    __syncthreads();
}


// Range compression of pulses n0 .. n0+P-1 (those < n_az) into S[:, n0 .. n0+P), run by
// blockDim.x == T*P threads with `smem` holding Tile<L, P>::SMEM_ELEMS elements.
// build_tab = false reuses a twiddle table left in smem by a previous tile of the same L.
// wait_before_store: a programmatic grid-dependency wait precedes the store of S (the previous kernel in the
// stream may still read the buffer S is written to; raw is not written by it).
template <int L, int P>
__device__ __forceinline__ void range_tile(const float2 *__restrict__ raw, const float *__restrict__ win, int n_az,
                                           bool centred, float2 *__restrict__ S, int n0, float2 *smem, bool build_tab,
                                           bool vec_store, bool wait_before_store = false) {
    using PL = Tile<L, P>;
    constexpr int RM = PL::RM, T = PL::T;
    float2 *tab = smem;               // two-level table of exp(-j*pi*q/L), q < 2L
    float2 *buf = smem + PL::TAB;     // FFT buffer [P][LP], then transposed tile [L][TP]
    const int t = threadIdx.x % T;
    const int p = threadIdx.x / T;
    const int n = n0 + p;

    float2 v[RM];
    {
        const bool live = n < n_az;
        const float2 *src = raw + (size_t)n * L;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const int m = t + r * T;
            const float2 x = live ? ld_stream(src + m) : make_float2(0.f, 0.f);
            const float wm = win ? __ldg(win + m) : 1.f;
            v[r] = cscale(x, wm);
        }
    }
    // the twiddle table is built while the loads are in flight; the first pass needs no twiddles and
    // its barrier orders these writes before any read
    if (build_tab) build_half_twiddles<L>(tab, PL::THREADS);
    float2 *pb = buf + p * PL::LP;
    constexpr int NF = PL::NF, RR = PL::RR;
    if constexpr (L < 16) {
        stockham_pass<L, P, L, 1, true, true>(v, t, p, pb, buf, tab, centred);
    } else {
        stockham_pass<L, P, 16, 1, true, (NF == 1 && RR == 1)>(v, t, p, pb, buf, tab, centred);
        if constexpr (NF >= 2) stockham_pass<L, P, 16, 16, false, (NF == 2 && RR == 1)>(v, t, p, pb, buf, tab, centred);
        if constexpr (NF >= 3) stockham_pass<L, P, 16, 256, false, (NF == 3 && RR == 1)>(v, t, p, pb, buf, tab, centred);
        if constexpr (RR > 1) stockham_pass<L, P, RR, (L / RR), false, true>(v, t, p, pb, buf, tab, centred);
    }

    // the transform is done: a kernel that depends on S (launched for programmatic overlap) may start
    // its own prologue now; it waits for this grid's completion before reading S.
    griddep_launch_dependents();
    if (wait_before_store) griddep_wait();
    // coalesced store of the transposed tile: row l holds pulses n0..n0+P-1
    const int np = min(P, n_az - n0);
    if (vec_store && np == P) {
        // pairs of pulses as one 16-byte store; rows of an odd stride are read as two 8-byte halves
        for (int idx = threadIdx.x; idx < L * (P / 2); idx += PL::THREADS) {
            const int l = idx / (P / 2), q = idx % (P / 2);
            float4 val;
            if constexpr (PL::TP_EVEN) {
                val = *reinterpret_cast<const float4 *>(buf + l * PL::TP + 2 * q);
            } else {
                const float2 a = buf[l * PL::TP + 2 * q], b = buf[l * PL::TP + 2 * q + 1];
                val = make_float4(a.x, a.y, b.x, b.y);
            }
            *reinterpret_cast<float4 *>(S + (size_t)l * n_az + n0 + 2 * q) = val;
        }
    } else {
        for (int idx = threadIdx.x; idx < L * P; idx += PL::THREADS) {
            const int l = idx / P, q = idx % P;
            if (q < np) S[(size_t)l * n_az + n0 + q] = buf[l * PL::TP + q];
        }
    }
}

// Adjoint of range_tile for pulses n0 .. n0+P-1 (Eq. (38) transposed, conjugate-Wirtinger convention):
//   grad_raw[n][m] = win[m] * sum_l conj(c_l) * exp(+j*2*pi*l*m/L) * g[l][n]
//                  = win[m] * conj( DFT_l{ c_l * conj(g[l][n]) }[m] ).
// Reads the range-major gradient g [L][n_az] with loads coalesced along azimuth, runs the same
// Stockham passes with every result kept in the per-pulse buffer (natural order), and writes
// grad_raw [n_az][L] pulse-major.  blockDim.x == T*P; `smem` holds Tile<L, P>::SMEM_ELEMS elements.
template <int L, int P>
__device__ __forceinline__ void range_adjoint_tile(const float2 *__restrict__ g, const float *__restrict__ win,
                                                   int n_az, bool centred, float2 *__restrict__ grad_raw, int n0,
                                                   float2 *smem) {
    using PL = Tile<L, P>;
    constexpr int RM = PL::RM, T = PL::T;
    float2 *tab = smem;
    float2 *buf = smem + PL::TAB;
    const int t = threadIdx.x % T;
    const int p = threadIdx.x / T;
    const int np = min(P, n_az - n0);
    build_half_twiddles<L>(tab, PL::THREADS);
    __syncthreads();
    for (int idx = threadIdx.x; idx < L * P; idx += PL::THREADS) {
        const int l = idx / P, q = idx % P;
        float2 x = q < np ? cconj(__ldg(g + (size_t)l * n_az + n0 + q)) : make_float2(0.f, 0.f);
        if (centred) {
            const float2 c = half_twiddle(tab, l);
            x = cmul(x, (l & 1) ? make_float2(-c.x, -c.y) : c);
        }
        buf[q * PL::LP + pad16(l)] = x;
    }
    __syncthreads();
    float2 v[RM];
    float2 *pb = buf + p * PL::LP;
    constexpr int NF = PL::NF, RR = PL::RR;
    if constexpr (L < 16) {
        stockham_pass<L, P, L, 1, false, false>(v, t, p, pb, buf, tab, false);
    } else {
        stockham_pass<L, P, 16, 1, false, false>(v, t, p, pb, buf, tab, false);
        if constexpr (NF >= 2) stockham_pass<L, P, 16, 16, false, false>(v, t, p, pb, buf, tab, false);
        if constexpr (NF >= 3) stockham_pass<L, P, 16, 256, false, false>(v, t, p, pb, buf, tab, false);
        if constexpr (RR > 1) stockham_pass<L, P, RR, (L / RR), false, false>(v, t, p, pb, buf, tab, false);
    }
    for (int idx = threadIdx.x; idx < P * L; idx += PL::THREADS) {
        const int q = idx / L, m = idx % L;
        if (q < np) {
            const float wm = win ? __ldg(win + m) : 1.f;
            grad_raw[(size_t)(n0 + q) * L + m] = cscale(cconj(buf[q * PL::LP + pad16(m)]), wm);
        }
    }
}

}  // namespace fft
}  // namespace rosar
