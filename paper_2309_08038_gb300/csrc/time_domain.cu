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

#include <cooperative_groups.h>

#include <cmath>

#include "rosar_internal.cuh"

namespace cg = cooperative_groups;

namespace rosar {
namespace {

constexpr int TD_THREADS = 128;
constexpr int TD_BT = 128;   // azimuth pixels per CTA
constexpr int TD_BR = 32;    // range rows per CTA (= warp size: one table entry per lane of warp 0)
constexpr int TD_MC = 16;    // fast-time samples per stage
constexpr int TD_AS = TD_MC + 1;                  // A row stride in elements (odd: conflict-free column reads)
constexpr int TD_TQ = TD_BT / 32;                 // azimuth pixels per thread (4): lane + 32 q
constexpr int TD_TI = TD_BR / (TD_THREADS / 32);  // rows per thread (8): 8 * warp + i
constexpr int TD_MAX_CLUSTER = 8;

__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// One CTA = TD_BT pixels x TD_BR rows x the taps [k_lo, k_hi) of its cluster rank.  With a cluster of G > 1
// CTAs along z the taps are split in G contiguous ranges and rank 0 adds the other ranks' partial tiles,
// read from their shared memory, in rank order (deterministic).
template <bool BPA>
__global__ void __launch_bounds__(TD_THREADS, 4)
td_tile_kernel(const float2 *__restrict__ X, const float *__restrict__ win, const float2 *__restrict__ w,
               const int32_t *__restrict__ o, TdParams p, int K, int k_per, float2 *__restrict__ out) {
    __shared__ __align__(16) float2 As[2][TD_BT * TD_AS];
    __shared__ __align__(16) float2 Bs[2][TD_MC][TD_BR];
    __shared__ float4 tab[3][TD_BR];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int th0 = blockIdx.x * TD_BT, r0 = blockIdx.y * TD_BR;
    const int n_az = p.n_az, L = p.L;
    const int chunks = L / TD_MC;
    const int k_lo = blockIdx.z * k_per;
    const int nk = max(0, min(K, k_lo + k_per) - k_lo);
    const int stages = nk * chunks;
    const bool wide = n_az >= TD_BT;            // one conditional subtraction wraps a tile row index

    auto tap_off = [&](int kk) -> int {
        const int k = k_lo + kk;
        return BPA ? k - K / 2 : pmod(__ldg(o + k), n_az);
    };
    auto build_tab = [&](int kk) {              // warp 0: one row per lane
        const int r = r0 + lane;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < p.n_rng) {
            t = tap_entry<BPA>(p, r, tap_off(kk));
            if (!BPA) {
                const float2 c = __ldg(w + (size_t)r * K + k_lo + kk);
                t.x = c.x;
                t.y = c.y;
            }
        }
        tab[kk % 3][lane] = t;
    };
    auto load_A = [&](int s, int buf) {         // 128 pulses x 16 samples by 8-byte cp.async, transposed rows
        const int kk = s / chunks, m0 = (s - kk * chunks) * TD_MC;
        const int base = pmod(th0 + tap_off(kk), n_az);
        const int m = tid & (TD_MC - 1);
#pragma unroll
        for (int j = 0; j < TD_BT * TD_MC / TD_THREADS; ++j) {
            const int t = (tid >> 4) + j * (TD_THREADS / TD_MC);
            int row = base + t;
            if (wide) row = row >= n_az ? row - n_az : row;
            else row %= n_az;
            cp_async8(&As[buf][t * TD_AS + m], X + (size_t)row * L + m0 + m);
        }
        cp_async_commit();
    };
    auto gen_B = [&](int s, int buf) {
        const int kk = s / chunks, m0 = (s - kk * chunks) * TD_MC;
#pragma unroll
        for (int q = 0; q < TD_BR * TD_MC / TD_THREADS; ++q) {
            const int v = tid + TD_THREADS * q;
            const int j = v & (TD_BR - 1), m = v >> 5;
            const float wm = win ? __ldg(win + m0 + m) : 1.f;
            Bs[buf][m][j] = phasor_term(tab[kk % 3][j], wm, (float)(m0 + m) - p.m_ref);
        }
    };

    float2 acc[TD_TQ][TD_TI];
#pragma unroll
    for (int q = 0; q < TD_TQ; ++q)
#pragma unroll
        for (int i = 0; i < TD_TI; ++i) acc[q][i] = make_float2(0.f, 0.f);

    if (stages > 0) {
        if (warp == 0) {
            build_tab(0);
            if (nk > 1) build_tab(1);
        }
        load_A(0, 0);
        __syncthreads();
        gen_B(0, 0);
        cp_async_wait_all();
        __syncthreads();
    }
    for (int s = 0; s < stages; ++s) {
        const int buf = s & 1;
        const bool more = s + 1 < stages;
        if (more) load_A(s + 1, buf ^ 1);
        if (warp == 0 && s % chunks == 0) {
            const int kk = s / chunks + 2;
            if (kk < nk) build_tab(kk);
        }
        const float2 *arow = &As[buf][lane * TD_AS];
#pragma unroll 4                                 // full unrolling overflows the instruction cache
        for (int m = 0; m < TD_MC; ++m) {
            float2 a[TD_TQ], b[TD_TI];
#pragma unroll
            for (int q = 0; q < TD_TQ; ++q) a[q] = arow[32 * q * TD_AS + m];
            const float4 *bp = reinterpret_cast<const float4 *>(&Bs[buf][m][TD_TI * warp]);
#pragma unroll
            for (int i = 0; i < TD_TI / 2; ++i) {
                const float4 v = bp[i];
                b[2 * i] = make_float2(v.x, v.y);
                b[2 * i + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int q = 0; q < TD_TQ; ++q)
#pragma unroll
                for (int i = 0; i < TD_TI; ++i) cmac(acc[q][i], a[q], b[i]);
        }
        if (more) gen_B(s + 1, buf ^ 1);
        cp_async_wait_all();
        __syncthreads();
    }

    // cluster split: every rank parks its partial tile in its own shared memory, rank 0 adds them in order
    const int G = gridDim.z;
    if (G > 1) {
        float2 *red = &As[0][0];                // 32 * 128 float2 = 32 KB <= sizeof(As)
        cg::cluster_group cluster = cg::this_cluster();
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TD_TQ; ++q)
#pragma unroll
            for (int i = 0; i < TD_TI; ++i) red[(q * TD_TI + i) * TD_THREADS + tid] = acc[q][i];
        cluster.sync();
        if (cluster.block_rank() == 0) {
            for (int rk = 1; rk < G; ++rk) {
                const float2 *rem = cluster.map_shared_rank(red, rk);
#pragma unroll
                for (int q = 0; q < TD_TQ; ++q)
#pragma unroll
                    for (int i = 0; i < TD_TI; ++i) acc[q][i] = cadd(acc[q][i], rem[(q * TD_TI + i) * TD_THREADS + tid]);
            }
        }
        cluster.sync();                         // the other ranks keep their shared memory until rank 0 is done
        if (cluster.block_rank() != 0) return;
    }
#pragma unroll
    for (int i = 0; i < TD_TI; ++i) {
        const int r = r0 + TD_TI * warp + i;
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

// Cluster size for the tap split: the G (1 .. 8, at most K, at least 8 taps per rank unless G = 1) whose
// clusters fill the co-resident cluster slots in the most nearly whole number of waves.
template <bool BPA>
int pick_cluster(int tiles, int K) {
    static int cached_dev = -1, cached_tiles = -1, cached_K = -1, cached_G = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev == cached_dev && tiles == cached_tiles && K == cached_K) return cached_G;
    int best_G = 1;
    double best = -1.0;
    for (int G = 1; G <= TD_MAX_CLUSTER; ++G) {
        if (G > 1 && (K < 8 * G)) break;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3(1, 1, G);
        cfg.blockDim = dim3(TD_THREADS);
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = G;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, td_tile_kernel<BPA>, &cfg) != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            continue;
        }
        const double waves = (double)tiles / clusters;
        const double eff = waves / std::ceil(waves);
        if (eff > best + 1e-3) {
            best = eff;
            best_G = G;
        }
    }
    cached_dev = dev;
    cached_tiles = tiles;
    cached_K = K;
    cached_G = best_G;
    return best_G;
}

template <bool BPA>
rosar_status launch_tiles(const float2 *raw, const float *win, const float2 *w, const int32_t *o, const TdParams &p,
                          int K, float2 *out, cudaStream_t s) {
    const int gx = (p.n_az + TD_BT - 1) / TD_BT, gy = (p.n_rng + TD_BR - 1) / TD_BR;
    const int G = pick_cluster<BPA>(gx * gy, K);
    const int k_per = (K + G - 1) / G;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(gx, gy, G);
    cfg.blockDim = dim3(TD_THREADS);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = G;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, td_tile_kernel<BPA>, raw, win, w, o, p, K, k_per, out);
    if (e != cudaSuccess)
        return set_error(ROSAR_ERR_CUDA, "%s: launch failed: %s", BPA ? "bpa_time" : "sas_time", cudaGetErrorString(e));
    return check_launch(BPA ? "bpa_time" : "sas_time");
}

}  // namespace

int time_domain_sample_multiple() { return TD_MC; }

rosar_status launch_time_domain(const float2 *raw, const float *win, const float2 *w, const int32_t *o,
                                int o_row_stride, const TdParams &p, int K, bool bpa, float2 *out, cudaStream_t s) {
    if (p.L % TD_MC != 0) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: L=%d is not a multiple of %d", p.L, TD_MC);
    if (bpa || o_row_stride == 0) {
        if ((p.n_rng + TD_BR - 1) / TD_BR > 65535)
            return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: n_rng=%d too large", p.n_rng);
        return bpa ? launch_tiles<true>(raw, win, w, o, p, K, out, s) : launch_tiles<false>(raw, win, w, o, p, K, out, s);
    }
    if (p.n_rng > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: n_rng=%d too large", p.n_rng);
    dim3 grid((p.n_az + TR_BT - 1) / TR_BT, p.n_rng);
    td_row_kernel<<<grid, TR_THREADS, 0, s>>>(raw, win, w, o, o_row_stride, p, K, out);
    return check_launch("sas_time");
}

}  // namespace rosar
