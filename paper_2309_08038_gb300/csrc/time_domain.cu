// Time-domain comparison paths: the paper's "BPA" (Sec. II-C, Eq. (14)) and "SAS" (Sec. III-A,
// Algorithm 2 with the compensation matrix W_SA).  Both sum, over taps k (aperture pulses) and fast-time
// samples m, a per-tap coefficient times a fast-time phasor times the raw IF sample:
//
//   out[r][theta] = sum_k c[r][k] * sum_m win[m] * exp(-j*pi*phi[r][k]*(m - m_ref)) * raw[(theta + o_k) mod N][m]
//
// with phi[r][k] = 2*rho/(dR*L) (half-turns per sample; tau*K*t_s of W_BP / W_SA in these units), rho the
// nominal slant range from the tap's phase centre to pixel (r, theta) (Eq. (2)):
//   rho^2 = (r*dR)^2 + 4*R*r0*sin^2(pi*o_k/N),   R = r0 + r*dR      (no cancellation),
// and
//   BPA: taps o_k = -M/2 .. M/2-1, c = alpha * exp(-j*2*k_mid*rho), alpha = max(0, (r*dR - 2*R*sin^2)/rho)
//        (Eqs. (3), (8), (15)), m_ref = (L-1)/2.  exp(-j*2*k*rho)*exp(-j*pi*phi*m) of Eq. (14) is the same
//        product referenced to the window centre: 2*(k_mid - k)*rho = pi*phi*(L-1)/2 exactly.
//   SAS: taps o_k from the caller, c = w[r][k], m_ref = (L-1)/2 (centred) or 0 (W_SA verbatim).
// The per-(r, k) quantities are evaluated in FP64 (the two-way phase 2*k_mid*rho reaches 10^5 rad); the
// fast-time phase is reduced exactly to one turn in FP32 (phi split into two floats, product error by FMA).
//
// With offsets shared by all rows the filter is an implicit complex GEMM over the index (k, m):
//   out[theta][r] = sum_(k,m) A[theta][(k,m)] * B[(k,m)][r],  A = raw[theta + o_k][m],  B = c*win*phasor,
// tiled as 128 azimuth pixels x 32 rows per CTA.  Each stage (one tap, 16 samples) stages the A tile
// (128 pulses x 16 samples, from L2) and generates the B tile (32 rows x 16 samples, one sincospif
// each) in shared memory, double-buffered; each thread accumulates a 4 x 4 register tile (FP32 FMA).
// Per-row offsets (Algorithm 2 with a support per range bin) use a row kernel: one row per CTA, the
// row's phasors staged in shared memory by sample chunk, pulses read through L1/L2.
//
// Compute-bound on FP32 FMA: 8 flops per (pixel, tap, sample).

#include "rosar_internal.cuh"

namespace rosar {
namespace {

constexpr int TD_THREADS = 256;
constexpr int TD_BT = 128;   // azimuth pixels per CTA
constexpr int TD_BR = 32;    // range rows per CTA (= warp size: one table entry per lane of warp 0)
constexpr int TD_MC = 16;    // fast-time samples per stage
constexpr int TD_TQ = TD_BT / 32;                 // azimuth pixels per thread (4)
constexpr int TD_TI = TD_BR / (TD_THREADS / 32);  // rows per thread (4)

// (c.re, c.im, phi_hi, phi_lo) of tap offset o in row r; c is only filled for BPA.
template <bool BPA>
__device__ __forceinline__ float4 tap_entry(const TdParams &p, int r, int o) {
    const double rr = r * p.dR;
    const double R = p.r0 + rr;
    const double s = sinpi((double)o / (double)p.n_az);
    const double s2 = s * s;
    const double rho = sqrt(fma(rr, rr, 4.0 * R * p.r0 * s2));
    const double phi = rho * p.phi_scale;
    const float hi = (float)phi;
    const float lo = (float)(phi - (double)hi);
    float cr = 0.f, ci = 0.f;
    if (BPA) {
        const double alpha = rho > 0.0 ? fmax(0.0, (rr - 2.0 * R * s2) / rho) : 1.0;
        double q = p.two_f_over_c * rho;          // cycles of two-way phase
        q -= floor(q);
        double sn, cs;
        sincospi(2.0 * q, &sn, &cs);
        cr = (float)(alpha * cs);
        ci = (float)(-alpha * sn);
    }
    return make_float4(cr, ci, hi, lo);
}

// c * win * exp(-j*pi*phi*x) for x = m - m_ref (a multiple of 1/2, exact in float).  The product phi*x is
// formed as hi*x (rounded) + its exact rounding error + lo*x, and hi*x is reduced modulo 2 exactly, so
// the argument of sincospif stays within about one half-turn at full precision.
__device__ __forceinline__ float2 phasor_term(float4 t, float wm, float x) {
    const float prod = t.z * x;
    const float err = fmaf(t.z, x, -prod);
    const float red = prod - 2.f * rintf(0.5f * prod);
    const float arg = red + fmaf(t.w, x, err);
    float sn, cs;
    sincospif(arg, &sn, &cs);
    const float2 c = make_float2(t.x * wm, t.y * wm);
    return cmul(c, make_float2(cs, -sn));
}

template <bool BPA>
__global__ void __launch_bounds__(TD_THREADS, 2)
td_tile_kernel(const float2 *__restrict__ X, const float *__restrict__ win, const float2 *__restrict__ w,
               const int32_t *__restrict__ o, TdParams p, int K, float2 *__restrict__ out) {
    __shared__ __align__(16) float2 As[2][TD_MC][TD_BT];
    __shared__ __align__(16) float2 Bs[2][TD_MC][TD_BR];
    __shared__ float4 tab[3][TD_BR];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int th0 = blockIdx.x * TD_BT, r0 = blockIdx.y * TD_BR;
    const int n_az = p.n_az, L = p.L;
    const int chunks = L / TD_MC;
    const int stages = K * chunks;

    auto tap_off = [&](int k) -> int { return BPA ? k - K / 2 : pmod(__ldg(o + k), n_az); };
    auto build_tab = [&](int k) {               // warp 0: one row per lane
        const int r = r0 + lane;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < p.n_rng) {
            t = tap_entry<BPA>(p, r, tap_off(k));
            if (!BPA) {
                const float2 c = __ldg(w + (size_t)r * K + k);
                t.x = c.x;
                t.y = c.y;
            }
        }
        tab[k % 3][lane] = t;
    };

    float4 areg[4];
    float2 breg[2];
    auto load_A = [&](int s) {
        const int k = s / chunks, m0 = (s - k * chunks) * TD_MC;
        const int off = tap_off(k);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int u = tid + TD_THREADS * q;
            const int t = u & (TD_BT - 1), c = u >> 7;
            const int row = pmod(th0 + off + t, n_az);
            const float4 *src = reinterpret_cast<const float4 *>(X + (size_t)row * L + m0 + 4 * c);
            areg[2 * q] = __ldg(src);
            areg[2 * q + 1] = __ldg(src + 1);
        }
    };
    auto gen_B = [&](int s) {
        const int k = s / chunks, m0 = (s - k * chunks) * TD_MC;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int v = tid + TD_THREADS * q;
            const int j = v & (TD_BR - 1), m = v >> 5;
            const float wm = win ? __ldg(win + m0 + m) : 1.f;
            breg[q] = phasor_term(tab[k % 3][j], wm, (float)(m0 + m) - p.m_ref);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int u = tid + TD_THREADS * q;
            const int t = u & (TD_BT - 1), c = u >> 7;
            As[buf][4 * c + 0][t] = make_float2(areg[2 * q].x, areg[2 * q].y);
            As[buf][4 * c + 1][t] = make_float2(areg[2 * q].z, areg[2 * q].w);
            As[buf][4 * c + 2][t] = make_float2(areg[2 * q + 1].x, areg[2 * q + 1].y);
            As[buf][4 * c + 3][t] = make_float2(areg[2 * q + 1].z, areg[2 * q + 1].w);
            const int v = tid + TD_THREADS * q;
            Bs[buf][v >> 5][v & (TD_BR - 1)] = breg[q];
        }
    };

    if (warp == 0) {
        build_tab(0);
        if (K > 1) build_tab(1);
    }
    __syncthreads();
    load_A(0);
    gen_B(0);
    store(0);
    __syncthreads();

    float2 acc[TD_TQ][TD_TI];
#pragma unroll
    for (int q = 0; q < TD_TQ; ++q)
#pragma unroll
        for (int i = 0; i < TD_TI; ++i) acc[q][i] = make_float2(0.f, 0.f);

    for (int s = 0; s < stages; ++s) {
        const int buf = s & 1;
        const bool more = s + 1 < stages;
        if (more) load_A(s + 1);
        if (warp == 0 && s % chunks == 0) {
            const int k = s / chunks + 2;
            if (k < K) build_tab(k);
        }
#pragma unroll
        for (int m = 0; m < TD_MC; ++m) {
            float2 a[TD_TQ], b[TD_TI];
#pragma unroll
            for (int q = 0; q < TD_TQ; ++q) a[q] = As[buf][m][lane + 32 * q];
#pragma unroll
            for (int i = 0; i < TD_TI; ++i) b[i] = Bs[buf][m][warp + 8 * i];
#pragma unroll
            for (int q = 0; q < TD_TQ; ++q)
#pragma unroll
                for (int i = 0; i < TD_TI; ++i) cmac(acc[q][i], a[q], b[i]);
        }
        if (more) {
            gen_B(s + 1);
            store(buf ^ 1);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TD_TI; ++i) {
        const int r = r0 + warp + 8 * i;
        if (r >= p.n_rng) continue;
#pragma unroll
        for (int q = 0; q < TD_TQ; ++q) {
            const int th = th0 + lane + 32 * q;
            if (th < n_az) out[(size_t)r * n_az + th] = acc[q][i];
        }
    }
}

// Per-row offsets: one CTA per (row, block of TR_BT pixels), two pixels per thread.  Samples are taken in
// chunks of TR_MC: the row's B chunk (all taps x TR_MC samples; one sincospif each) is generated into
// shared memory, then every thread sweeps taps and samples, reading its pulses' samples as float4 pairs.
constexpr int TR_THREADS = 256;
constexpr int TR_TT = 2;
constexpr int TR_BT = TR_THREADS * TR_TT;
constexpr int TR_MC = 16;
constexpr int TR_KC = 64;    // taps per shared-memory chunk

__global__ void __launch_bounds__(TR_THREADS)
td_row_kernel(const float2 *__restrict__ X, const float *__restrict__ win, const float2 *__restrict__ w,
              const int32_t *__restrict__ o, int o_row_stride, TdParams p, int K, float2 *__restrict__ out) {
    __shared__ float4 tab[TR_KC];
    __shared__ int offs[TR_KC];
    __shared__ __align__(16) float2 Bs[TR_KC][TR_MC];

    const int r = blockIdx.y;
    const int th0 = blockIdx.x * TR_BT;
    const int n_az = p.n_az, L = p.L;
    const int32_t *orow = o + (size_t)r * o_row_stride;
    const float2 *wrow = w + (size_t)r * K;
    int th[TR_TT];
#pragma unroll
    for (int q = 0; q < TR_TT; ++q) th[q] = min(th0 + threadIdx.x + TR_THREADS * q, n_az - 1);

    float2 acc[TR_TT];
#pragma unroll
    for (int q = 0; q < TR_TT; ++q) acc[q] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < K; k0 += TR_KC) {
        const int nk = min(TR_KC, K - k0);
        __syncthreads();
        if (threadIdx.x < nk) {
            const int k = k0 + threadIdx.x;
            const int off = pmod(__ldg(orow + k), n_az);
            float4 t = tap_entry<false>(p, r, off);
            const float2 c = __ldg(wrow + k);
            t.x = c.x;
            t.y = c.y;
            tab[threadIdx.x] = t;
            offs[threadIdx.x] = off;
        }
        for (int m0 = 0; m0 < L; m0 += TR_MC) {
            __syncthreads();
            for (int v = threadIdx.x; v < nk * TR_MC; v += TR_THREADS) {
                const int kk = v / TR_MC, m = v - kk * TR_MC;
                const float wm = win ? __ldg(win + m0 + m) : 1.f;
                Bs[kk][m] = phasor_term(tab[kk], wm, (float)(m0 + m) - p.m_ref);
            }
            __syncthreads();
            for (int kk = 0; kk < nk; ++kk) {
                const int off = offs[kk];
#pragma unroll
                for (int q = 0; q < TR_TT; ++q) {
                    const int row = pmod(th[q] + off, n_az);
                    const float4 *src = reinterpret_cast<const float4 *>(X + (size_t)row * L + m0);
#pragma unroll
                    for (int c = 0; c < TR_MC / 2; ++c) {
                        const float4 xv = __ldg(src + c);
                        cmac(acc[q], make_float2(xv.x, xv.y), Bs[kk][2 * c]);
                        cmac(acc[q], make_float2(xv.z, xv.w), Bs[kk][2 * c + 1]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < TR_TT; ++q) {
        const int t = th0 + threadIdx.x + TR_THREADS * q;
        if (t < n_az) out[(size_t)r * n_az + t] = acc[q];
    }
}

}  // namespace

int time_domain_sample_multiple() { return TD_MC; }

rosar_status launch_time_domain(const float2 *raw, const float *win, const float2 *w, const int32_t *o,
                                int o_row_stride, const TdParams &p, int K, bool bpa, float2 *out, cudaStream_t s) {
    if (p.L % TD_MC != 0) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: L=%d is not a multiple of %d", p.L, TD_MC);
    if (bpa || o_row_stride == 0) {
        const int gy = (p.n_rng + TD_BR - 1) / TD_BR;
        if (gy > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: n_rng=%d too large", p.n_rng);
        dim3 grid((p.n_az + TD_BT - 1) / TD_BT, gy);
        if (bpa)
            td_tile_kernel<true><<<grid, TD_THREADS, 0, s>>>(raw, win, w, o, p, K, out);
        else
            td_tile_kernel<false><<<grid, TD_THREADS, 0, s>>>(raw, win, w, o, p, K, out);
        return check_launch(bpa ? "bpa_time" : "sas_time");
    }
    if (p.n_rng > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: n_rng=%d too large", p.n_rng);
    dim3 grid((p.n_az + TR_BT - 1) / TR_BT, p.n_rng);
    td_row_kernel<<<grid, TR_THREADS, 0, s>>>(raw, win, w, o, o_row_stride, p, K, out);
    return check_launch("sas_time");
}

}  // namespace rosar
