// K3: range-compressed back-projection, the FFT+BPA comparison path
// (arXiv 2309.08038, Sec. III-D after Eq. (43) with w_BP; Eq. (14); Eqs. (2), (3), (8), (37), (40)).
//
//   out[r][theta] = sum_d alpha_n * exp(-j*2*k_mid*R_n) * S(R_n/dR, n),  n = (theta + d) mod n_az
//
// Pixel (r, theta) is at R = r0 + r*dR, angle 2*pi*theta/n_az; pulse n at radius
// r0 + dr[n] and angle 2*pi*n/n_az + dphi[n].  With rho = R - r0 (the pixel's slant
// range seen from the facing pulse, exactly r bins) the kernel evaluates
//   R_n^2 - rho^2 = dr*(r_n + r0 - 2R) + 4*R*r_n*sin^2(dphi_n/2)            (no cancellation)
//   delta = R_n - rho = (R_n^2 - rho^2)/(R_n + rho),   bin x = r + delta/dR,
//   cos(theta') = ((rho - dr) - 2*R*sin^2(dphi_n/2))/R_n,   alpha = max(0, cos(theta')),
//   exp(-j*2*k_mid*R_n) = exp(-j*2*k_mid*rho) * exp(-j*2*pi*(2*f_mid/c)*delta),
// so every float32 quantity is small and well conditioned; the per-row factor
// exp(-j*2*k_mid*rho) is computed once per CTA in FP64.  sin(dphi_n/2) is
// sin(pi*d/n_az)*cos(eps/2) + cos(pi*d/n_az)*sin(eps/2) from a per-d table and a
// per-pulse table, both staged in shared memory.
//
// With no pulse errors supplied (nominal geometry) every per-pulse quantity
// depends on (r, d) only; that kernel variant tabulates (x, alpha*phase) per d
// and the pixel loop is two gathers, an interpolation and a complex MAC.
//
// With supplied errors the fine phase exp(-j*2*pi*(2*f_mid/c)*delta) of every (pixel, pulse) is taken as
// sin/cos of the phase in turns first reduced exactly by whole turns to [-1/2, 1/2] (delta spans tens of cycles)
// and then evaluated by the hardware sine and cosine (about 1e-6 absolute error there), instead of the accurate
// sincospif's software range reduction and polynomials: the per-sample work is issue-bound FP32 and SFU.
// The interpolation mode is a template parameter.
//
// Grid: (azimuth tiles of 256 pixels, rows).  Once S is staged in shared memory the nominal kernel is bound by
// shared-memory bandwidth (two 8-byte window reads per sample) and the supplied-error kernel by FP32 + SFU issue.

#include "rosar_internal.cuh"

namespace rosar {
namespace {

constexpr int BPA_THREADS = 256;
constexpr int BPA_WR = 6;     // range rows of the staged S window
// aperture offsets staged per chunk: 512 with nominal geometry; 256 with supplied errors, whose per-pulse table
// makes a CTA's shared memory the occupancy limit (256: 6 CTAs per SM instead of 3)
template <bool NOMINAL> constexpr int bpa_dc() { return NOMINAL ? 512 : 256; }
template <bool NOMINAL> constexpr int bpa_wc() { return BPA_THREADS + bpa_dc<NOMINAL>(); }   // window columns (pulses)
template <bool NOMINAL> constexpr int bpa_smem() { return BPA_WR * bpa_wc<NOMINAL>() * 8; }

__device__ __forceinline__ float2 read_bin(const float2 *__restrict__ S, int l, int L, size_t col, int n_az) {
    return (l >= 0 && l < L) ? __ldg(S + (size_t)l * n_az + col) : make_float2(0.f, 0.f);
}

// Per chunk of offsets the bins a pixel of row r reads lie in a few rows near r (x = r + (R_n - rho)/dR, within a
// couple of bins over a +-30 degree aperture): a window of rows around the chunk's range of x and the pulses
// th0 + dc .. th0 + dc + BPA_WC are staged in shared memory once.  The range of x is the nominal one widened by
// the largest distance a supplied pulse position lies from its nominal one: R_n is a distance from the pixel, so it
// moves by at most |pos_n - pos_n,nominal| <= |dr_n| + 2*r0*|sin(eps_n/2)| (triangle inequality).  When that range,
// with a bin of margin below and two above, fits the window (always with nominal geometry; with supplied errors
// unless some pulse lies more than a bin or so off), every sample's bins are in it, rows outside [0, L) are staged
// as zeros, and the pixel loop reads the window with no check.  Otherwise the window is the nominal one and each
// sample whose bins fall outside it reads S through L2.
// max that keeps a NaN (fmaxf drops it): a NaN error bound must reach the window test and fail it
__device__ __forceinline__ float nanmax(float a, float b) { return (a > b || a != a) ? a : b; }

// exp(-j*2*pi*q) for |q| up to 2^22 turns: q reduced by whole turns (q - rint(q), exact) to [-1/2, 1/2], then
// the hardware sine and cosine of 2*pi times the remainder.
__device__ __forceinline__ float2 expmj2pi_turns(float q) {
    const float r = q - rintf(q);
    float sn, cs;
    __sincosf(6.28318530717959f * r, &sn, &cs);
    return make_float2(cs, -sn);
}

template <bool NOMINAL, bool LINEAR>
__global__ void __launch_bounds__(BPA_THREADS)
bpa_kernel(const float2 *__restrict__ S, BpaParams p, const float *__restrict__ dphi, const float *__restrict__ dr,
           int L, int n_az, int M_ap, float2 *__restrict__ out) {
    constexpr int BPA_DC = bpa_dc<NOMINAL>(), BPA_WC = bpa_wc<NOMINAL>();
    extern __shared__ float2 wsm[];                           // [BPA_WR][BPA_WC]
    __shared__ float4 dtab[BPA_DC];                           // NOMINAL: (x, a.re, a.im, -); else (sin, cos, x_nominal, -)
    // per pulse, with this CTA's row folded in: (cos(eps/2), sin(eps/2), dr*(r_n + r0 - 2R), 4*R*r_n), and
    // rho - dr (the numerator of cos(theta') before its sin^2 term)
    __shared__ float4 ptab[NOMINAL ? 1 : BPA_THREADS + BPA_DC];
    __shared__ float pal[NOMINAL ? 1 : BPA_THREADS + BPA_DC];
    __shared__ float2 rowph;
    __shared__ float red_lo[BPA_THREADS / 32], red_hi[BPA_THREADS / 32], red_e[BPA_THREADS / 32];

    const int r = blockIdx.y;
    const int th0 = blockIdx.x * BPA_THREADS;
    const int th = th0 + threadIdx.x;
    const float rf = (float)r;
    const double rho_d = r * p.dR;
    const float rho = (float)rho_d;
    const float R = (float)(p.r0 + rho_d);
    const float r0 = (float)p.r0;
    if (threadIdx.x == 0) {
        double q = p.two_f_over_c_d * rho_d;
        q -= floor(q);
        double s, c;
        sincospi(2.0 * q, &s, &c);
        rowph = make_float2((float)c, (float)-s);
    }

    float2 acc = make_float2(0.f, 0.f);
    const int d_beg = -(M_ap / 2), d_end = M_ap - M_ap / 2;
    // chunks of equal size (at most BPA_DC offsets): M = 600 with BPA_DC = 256 gives 3 chunks of 200
    const int n_chunks = (M_ap + BPA_DC - 1) / BPA_DC;
    const int step = (M_ap + n_chunks - 1) / n_chunks;
    for (int dc = d_beg; dc < d_end; dc += step) {
        const int nd = min(step, d_end - dc);
        __syncthreads();
        float xlo = 1e30f, xhi = -1e30f;
        for (int i = threadIdx.x; i < nd; i += BPA_THREADS) {
            float s, c;
            sincospif((float)(dc + i) / (float)n_az, &s, &c);   // sin/cos(pi*d/n_az)
            // nominal geometry: x and the weight of this offset
            const float s2 = s * s;
            const float num = 4.f * R * r0 * s2;                // R_n^2 - rho^2
            const float Rn2 = fmaf(rho, rho, num);
            float delta, alpha;
            if (Rn2 > 0.f) {
                const float inv = rsqrtf(Rn2);
                const float Rn = Rn2 * inv;
                delta = __fdividef(num, Rn + rho);
                alpha = fmaxf(0.f, fmaf(-2.f * R, s2, rho) * inv);
            } else {
                delta = 0.f;
                alpha = 1.f;
            }
            const float x = fmaf(delta, p.inv_dR, rf);
            xlo = fminf(xlo, x);
            xhi = fmaxf(xhi, x);
            if (NOMINAL) {
                float ps, pc;
                sincospif(2.f * p.two_f_over_c * delta, &ps, &pc);
                dtab[i] = make_float4(x, alpha * pc, -alpha * ps, 0.f);
            } else {
                dtab[i] = make_float4(s, c, x, 0.f);
            }
        }
        float emax = 0.f;   // largest pulse position error of the chunk, in bins
        if (!NOMINAL) {
            for (int i = threadIdx.x; i < BPA_THREADS + nd; i += BPA_THREADS) {
                const int n = pmod(th0 + dc + i, n_az);
                const float e = dphi ? __ldg(dphi + n) : 0.f;
                float se, ce;
                sincosf(0.5f * e, &se, &ce);
                const float drn = dr ? __ldg(dr + n) : 0.f;
                const float rn = r0 + drn;
                ptab[i] = make_float4(ce, se, drn * (rn + r0 - 2.f * R), 4.f * R * rn);
                pal[i] = rho - drn;
                emax = nanmax(emax, fmaf(2.f * r0, fabsf(se), fabsf(drn)) * p.inv_dR);
            }
        }
        // the chunk's x range and error bound over the CTA
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) {
            xlo = fminf(xlo, __shfl_xor_sync(0xffffffffu, xlo, sft));
            xhi = fmaxf(xhi, __shfl_xor_sync(0xffffffffu, xhi, sft));
            if (!NOMINAL) emax = nanmax(emax, __shfl_xor_sync(0xffffffffu, emax, sft));
        }
        if ((threadIdx.x & 31) == 0) {
            red_lo[threadIdx.x >> 5] = xlo;
            red_hi[threadIdx.x >> 5] = xhi;
            red_e[threadIdx.x >> 5] = emax;
        }
        __syncthreads();
        xlo = red_lo[0];
        xhi = red_hi[0];
        emax = red_e[0];
        for (int i = 1; i < BPA_THREADS / 32; ++i) {
            xlo = fminf(xlo, red_lo[i]);
            xhi = fmaxf(xhi, red_hi[i]);
            if (!NOMINAL) emax = nanmax(emax, red_e[i]);
        }
        // covered: every sample's x lies in [xlo - emax, xhi + emax] (up to rounding, far below the margins), so
        // its bins floor(x) and floor(x) + 1 lie in rows [floor(xlo - emax) - 1, floor(xhi + emax) + 2]
        const float flo = floorf(xlo - emax), fhi = floorf(xhi + emax);
        const bool covered = fhi - flo <= (float)(BPA_WR - 4) && flo > -1e6f && fhi < 1e6f;   // false for NaN
        int wlo, nrow;
        if (covered) {
            wlo = (int)flo - 1;
            nrow = (int)(fhi - flo) + 4;
        } else {
            wlo = max(0, (int)floorf(xlo) - 1);
            nrow = min(BPA_WR, min(L - 1, (int)floorf(xhi) + 2) - wlo + 1);
        }
        const int wtop = wlo + nrow;                                  // rows [wlo, wtop) staged
        const int ncol = BPA_THREADS + nd;
        for (int e = threadIdx.x; e < nrow * ncol; e += BPA_THREADS) {
            const int rr = e / ncol, cc = e - rr * ncol;
            const int n = pmod(th0 + dc + cc, n_az);
            const int l = wlo + rr;
            wsm[rr * BPA_WC + cc] = (l >= 0 && l < L) ? __ldg(S + (size_t)l * n_az + n) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (th >= n_az) continue;
        // bin x and weight alpha * exp(-j*2*pi*(2 f/c)*delta) of offset dc + i for this thread's pixel
        auto sample = [&](int i, float &x, float2 &a) {
            const float4 t = dtab[i];
            if (NOMINAL) {
                x = t.x;
                a = make_float2(t.y, t.z);
            } else {
                const float4 pp = ptab[threadIdx.x + i];
                const float sh = fmaf(t.x, pp.x, t.y * pp.y);            // sin((pi*d/n_az) + eps/2)
                const float s2 = sh * sh;
                const float num = fmaf(pp.w, s2, pp.z);                  // R_n^2 - rho^2
                const float Rn2 = fmaf(rho, rho, num);
                // branch-free: R_n = 0 (the facing pulse of row 0, or a supplied position on the pixel) gives
                // delta = num / rho = -rho exactly, or 0 when rho = 0 too, and alpha = 1 by the select
                const float inv = rsqrtf(fmaxf(Rn2, 1e-30f));
                const float Rn = Rn2 * inv;
                const float delta = __fdividef(num, fmaxf(Rn + rho, 1e-30f));
                // alpha = max(0, cos(theta')), cos(theta') <= 1: one saturating multiply
                const float a0 = __saturatef(fmaf(-2.f * R, s2, pal[threadIdx.x + i]) * inv);
                const float alpha = Rn2 > 0.f ? a0 : 1.f;
                x = fmaf(delta, p.inv_dR, rf);
                a = cscale(expmj2pi_turns(p.two_f_over_c * delta), alpha);
            }
        };
        if (covered) {
            // in-window by construction; the unsigned clamp keeps even a NaN x's read inside the staged rows
            const float2 *colp = wsm + threadIdx.x;
#pragma unroll 4
            for (int i = 0; i < nd; ++i) {
                float x;
                float2 a;
                sample(i, x, a);
                float2 sv;
                if (LINEAR) {
                    const float fl = floorf(x);
                    const unsigned rel = min((unsigned)(int)fl - (unsigned)wlo, (unsigned)(nrow - 2));
                    const float2 s0 = colp[rel * BPA_WC + i], s1 = colp[(rel + 1) * BPA_WC + i];
                    sv = caxpy(x - fl, csub(s1, s0), s0);
                } else {
                    const unsigned rel = min((unsigned)(int)floorf(x + 0.5f) - (unsigned)wlo, (unsigned)(nrow - 1));
                    sv = colp[rel * BPA_WC + i];
                }
                cmac(acc, a, sv);
            }
        } else {
#pragma unroll 4
            for (int i = 0; i < nd; ++i) {
                float x;
                float2 a;
                sample(i, x, a);
                const int col = threadIdx.x + i;
                float2 sv;
                if (LINEAR) {
                    const float fl = floorf(x);
                    const int l0 = (int)fl;
                    const float f = x - fl;
                    float2 s0, s1;
                    if (l0 >= wlo && l0 + 1 < wtop) {
                        s0 = wsm[(l0 - wlo) * BPA_WC + col];
                        s1 = wsm[(l0 + 1 - wlo) * BPA_WC + col];
                    } else {                  // off the staged window: pulse (th + d) mod n_az through L2
                        const int n = pmod(th + dc + i, n_az);
                        s0 = read_bin(S, l0, L, n, n_az);
                        s1 = read_bin(S, l0 + 1, L, n, n_az);
                    }
                    sv = caxpy(f, csub(s1, s0), s0);
                } else {
                    const int l0 = (int)floorf(x + 0.5f);
                    sv = (l0 >= wlo && l0 < wtop) ? wsm[(l0 - wlo) * BPA_WC + col]
                                                  : read_bin(S, l0, L, pmod(th + dc + i, n_az), n_az);
                }
                cmac(acc, a, sv);
            }
        }
    }
    if (th < n_az) out[(size_t)r * n_az + th] = cmul(rowph, acc);
}

}  // namespace

rosar_status launch_bpa(const float2 *S, const BpaParams &p, const float *dphi, const float *dr, int L, int n_rng,
                        int n_az, int M_ap, int interp, float2 *out, cudaStream_t s) {
    if (n_rng > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "bpa: n_rng=%d exceeds 65535", n_rng);
    dim3 grid((n_az + BPA_THREADS - 1) / BPA_THREADS, n_rng);
    static int done[4][kMaxDevices] = {};
    const bool nominal = dphi == nullptr && dr == nullptr;
    const int v = (nominal ? 0 : 2) + (interp ? 1 : 0);
    static const void *const ks[4] = {(const void *)bpa_kernel<true, false>, (const void *)bpa_kernel<true, true>,
                                      (const void *)bpa_kernel<false, false>, (const void *)bpa_kernel<false, true>};
    const int smem = nominal ? bpa_smem<true>() : bpa_smem<false>();
    rosar_status st = ensure_smem(ks[v], smem, done[v], "bpa");
    if (st != ROSAR_OK) return st;
    switch (v) {
        case 0: bpa_kernel<true, false><<<grid, BPA_THREADS, smem, s>>>(S, p, dphi, dr, L, n_az, M_ap, out); break;
        case 1: bpa_kernel<true, true><<<grid, BPA_THREADS, smem, s>>>(S, p, dphi, dr, L, n_az, M_ap, out); break;
        case 2: bpa_kernel<false, false><<<grid, BPA_THREADS, smem, s>>>(S, p, dphi, dr, L, n_az, M_ap, out); break;
        default: bpa_kernel<false, true><<<grid, BPA_THREADS, smem, s>>>(S, p, dphi, dr, L, n_az, M_ap, out); break;
    }
    return check_launch("bpa");
}

}  // namespace rosar
