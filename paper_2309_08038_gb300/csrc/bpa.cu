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
// Grid: (azimuth tiles of 256 pixels, rows).  Compute-bound (FP32 + SFU).

#include "rosar_internal.cuh"

namespace rosar {
namespace {

constexpr int BPA_THREADS = 256;
constexpr int BPA_DC = 512;   // aperture offsets staged per chunk

__device__ __forceinline__ float2 read_bin(const float2 *__restrict__ S, int l, int L, size_t col, int n_az) {
    return (l >= 0 && l < L) ? __ldg(S + (size_t)l * n_az + col) : make_float2(0.f, 0.f);
}

template <bool NOMINAL>
__global__ void __launch_bounds__(BPA_THREADS)
bpa_kernel(const float2 *__restrict__ S, BpaParams p, const float *__restrict__ dphi, const float *__restrict__ dr,
           int L, int n_az, int M_ap, int interp, float2 *__restrict__ out) {
    __shared__ float4 dtab[BPA_DC];                           // NOMINAL: (x, a.re, a.im, -); else (sin, cos, -, -)
    __shared__ float4 ptab[NOMINAL ? 1 : BPA_THREADS + BPA_DC];   // per pulse (cos(eps/2), sin(eps/2), dr, -)
    __shared__ float2 rowph;

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
    for (int dc = d_beg; dc < d_end; dc += BPA_DC) {
        const int nd = min(BPA_DC, d_end - dc);
        __syncthreads();
        for (int i = threadIdx.x; i < nd; i += BPA_THREADS) {
            float s, c;
            sincospif((float)(dc + i) / (float)n_az, &s, &c);   // sin/cos(pi*d/n_az)
            if (NOMINAL) {
                const float s2 = s * s;
                const float num = 4.f * R * r0 * s2;            // R_n^2 - rho^2
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
                float ps, pc;
                sincospif(2.f * p.two_f_over_c * delta, &ps, &pc);
                dtab[i] = make_float4(fmaf(delta, p.inv_dR, rf), alpha * pc, -alpha * ps, 0.f);
            } else {
                dtab[i] = make_float4(s, c, 0.f, 0.f);
            }
        }
        if (!NOMINAL) {
            for (int i = threadIdx.x; i < BPA_THREADS + nd; i += BPA_THREADS) {
                const int n = pmod(th0 + dc + i, n_az);
                const float e = dphi ? __ldg(dphi + n) : 0.f;
                float se, ce;
                sincosf(0.5f * e, &se, &ce);
                ptab[i] = make_float4(ce, se, dr ? __ldg(dr + n) : 0.f, 0.f);
            }
        }
        __syncthreads();
        if (th < n_az) {
            int n = th + dc;
            n = n < 0 ? n + n_az : (n >= n_az ? n - n_az : n);
            for (int i = 0; i < nd; ++i) {
                const float4 t = dtab[i];
                float x;
                float2 a;
                if (NOMINAL) {
                    x = t.x;
                    a = make_float2(t.y, t.z);
                } else {
                    const float4 pp = ptab[threadIdx.x + i];
                    const float sh = fmaf(t.x, pp.x, t.y * pp.y);            // sin((pi*d/n_az) + eps/2)
                    const float s2 = sh * sh;
                    const float drn = pp.z;
                    const float rn = r0 + drn;
                    const float num = fmaf(drn, rn + r0 - 2.f * R, 4.f * R * rn * s2);
                    const float Rn2 = fmaf(rho, rho, num);
                    float delta, alpha;
                    if (Rn2 > 0.f) {
                        const float inv = rsqrtf(Rn2);
                        const float Rn = Rn2 * inv;
                        delta = __fdividef(num, Rn + rho);
                        alpha = fmaxf(0.f, fmaf(-2.f * R, s2, rho - drn) * inv);
                    } else {
                        delta = 0.f;
                        alpha = 1.f;
                    }
                    float ps, pc;
                    sincospif(2.f * p.two_f_over_c * delta, &ps, &pc);
                    x = fmaf(delta, p.inv_dR, rf);
                    a = make_float2(alpha * pc, -alpha * ps);
                }
                float2 sv;
                if (interp) {
                    const float fl = floorf(x);
                    const int l0 = (int)fl;
                    const float f = x - fl;
                    const float2 s0 = read_bin(S, l0, L, n, n_az);
                    const float2 s1 = read_bin(S, l0 + 1, L, n, n_az);
                    sv = make_float2(fmaf(f, s1.x - s0.x, s0.x), fmaf(f, s1.y - s0.y, s0.y));
                } else {
                    sv = read_bin(S, (int)floorf(x + 0.5f), L, n, n_az);
                }
                cmac(acc, a, sv);
                if (++n == n_az) n = 0;
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
    if (dphi == nullptr && dr == nullptr)
        bpa_kernel<true><<<grid, BPA_THREADS, 0, s>>>(S, p, dphi, dr, L, n_az, M_ap, interp, out);
    else
        bpa_kernel<false><<<grid, BPA_THREADS, 0, s>>>(S, p, dphi, dr, L, n_az, M_ap, interp, out);
    return check_launch("bpa");
}

}  // namespace rosar
