// Differentiable form: per-pulse phase correction and the adjoints of the sparse azimuth
// filter (arXiv 2309.08038, Sec. III-D, Eq. (43)), for a stack of scans sharing one weight set.
//
// Forward (with the gather kernel in between):
//   S_t[s][r][n]   = S[s][r][n] * exp(j * eps[s][n])                          (phase_apply)
//   out[s][r][t]   = sum_k w[r][k] * S_t[s][r][(t + o_k) mod N]
// Backward, conjugate-Wirtinger convention (grad of a real loss; grad_x = A^H grad_y):
//   grad_S_t       = sum_k conj(w[r][k]) * g[s][r][(n - o_k) mod N]           (gather kernel, adjoint mode)
//   grad_w[r][k]   = sum_s sum_t g[s][r][t] * conj(S_t[s][r][(t + o_k) mod N]) (weight_grad)
//   grad_eps[s][n] = sum_r Im(conj(S_t[s][r][n]) * grad_S_t[s][r][n])          (phase_grad)
//   grad_S         = grad_S_t * exp(-j * eps[s][n])                            (phase_grad, optional)
// Every reduction runs in a fixed order (no atomics), so gradients are bit-reproducible.

#include <limits.h>

#include "rosar_internal.cuh"

namespace rosar {
namespace {

constexpr int DG_THREADS = 256;

// One thread per (scan, pulse): the phase factor is computed once and applied down the column.
__global__ void __launch_bounds__(DG_THREADS)
phase_apply_kernel(const float2 *__restrict__ S, const float *__restrict__ eps, int n_rng, int n_az,
                   float2 *__restrict__ S_t) {
    const int n = blockIdx.x * DG_THREADS + threadIdx.x;
    const int s = blockIdx.y;
    if (n >= n_az) return;
    float sn, cs;
    sincosf(__ldg(eps + (size_t)s * n_az + n), &sn, &cs);
    const float2 e = make_float2(cs, sn);
    const size_t base = (size_t)s * n_rng * n_az + n;
#pragma unroll 4
    for (int r = 0; r < n_rng; ++r) S_t[base + (size_t)r * n_az] = cmul(__ldg(S + base + (size_t)r * n_az), e);
}

// Phase gradients: CTA = 32 consecutive pulses x 8 row groups (256 threads).  Lane c of warp g owns pulse
// n0 + c and rows g, g + 8, ...; the 8 group sums of a pulse are then added in group order, so every pulse's
// sum runs in one fixed order (rows g mod 8 ascending within a group, groups 0..7).
constexpr int PG_COLS = 32, PG_GROUPS = DG_THREADS / PG_COLS;

// grad_eps[s][n] = sum_r Im(conj(a) b), a = S_t (or S * P), b = G; grad_S = G * conj(e) with e the phase factor.
template <bool PHASOR>
__device__ __forceinline__ void phase_grad_cta(const float2 *__restrict__ S, const float2 *__restrict__ P,
                                               const float *__restrict__ eps, const float2 *__restrict__ G, int n_rng,
                                               int n_az, float *__restrict__ grad_eps, float2 *__restrict__ grad_S) {
    __shared__ float red[PG_GROUPS][PG_COLS];
    const int c = threadIdx.x % PG_COLS, g = threadIdx.x / PG_COLS;
    const int n = blockIdx.x * PG_COLS + c;
    const int s = blockIdx.y;
    float acc = 0.f;
    if (n < n_az) {
        const size_t base = (size_t)s * n_rng * n_az + n;
        float2 e = make_float2(1.f, 0.f);                        // the forward's factor exp(j eps)
        if (PHASOR) {
            e = __ldg(P + (size_t)s * n_az + n);
        } else if (grad_S) {
            float sn, cs;
            sincosf(__ldg(eps + (size_t)s * n_az + n), &sn, &cs);
            e = make_float2(cs, sn);
        }
        const float2 ec = make_float2(e.x, -e.y);
#pragma unroll 4
        for (int r = g; r < n_rng; r += PG_GROUPS) {
            const float2 sv = __ldg(S + base + (size_t)r * n_az);
            const float2 a = PHASOR ? cmul(sv, e) : sv;
            const float2 b = __ldg(G + base + (size_t)r * n_az);
            acc = fmaf(a.x, b.y, acc);          // Im(conj(a) * b) = a.x*b.y - a.y*b.x
            acc = fmaf(-a.y, b.x, acc);
            if (grad_S) grad_S[base + (size_t)r * n_az] = cmul(b, ec);
        }
    }
    red[g][c] = acc;
    __syncthreads();
    if (g == 0 && n < n_az && grad_eps) {
        float t = red[0][c];
#pragma unroll
        for (int q = 1; q < PG_GROUPS; ++q) t += red[q][c];
        grad_eps[(size_t)s * n_az + n] = t;
    }
}

__global__ void __launch_bounds__(DG_THREADS)
phase_grad_kernel(const float2 *__restrict__ S_t, const float2 *__restrict__ G, const float *__restrict__ eps,
                  int n_rng, int n_az, float *__restrict__ grad_eps, float2 *__restrict__ grad_S) {
    phase_grad_cta<false>(S_t, nullptr, eps, G, n_rng, n_az, grad_eps, grad_S);
}

// The phase factors e^{j eps} of every (scan, pulse) once, with the same sincosf as phase_apply_kernel.
__global__ void __launch_bounds__(DG_THREADS)
phasor_kernel(const float *__restrict__ eps, long long n, float2 *__restrict__ P) {
    const long long i = (long long)blockIdx.x * DG_THREADS + threadIdx.x;
    if (i >= n) return;
    float sn, cs;
    sincosf(__ldg(eps + i), &sn, &cs);
    P[i] = make_float2(cs, sn);
}

// phase_grad_kernel with the corrected rows formed at load: S_t = S * P, grad_S = G * conj(P) (the same products
// phase_apply_kernel and phase_grad_kernel compute, in the same order, so the results are identical).
__global__ void __launch_bounds__(DG_THREADS)
phase_grad_phasor_kernel(const float2 *__restrict__ S, const float2 *__restrict__ P, const float2 *__restrict__ G,
                         int n_rng, int n_az, float *__restrict__ grad_eps, float2 *__restrict__ grad_S) {
    phase_grad_cta<true>(S, P, nullptr, G, n_rng, n_az, grad_eps, grad_S);
}

// grad_w: one CTA of 1024 threads per range row.  Its 32 warps form TAPG tap groups x THG azimuth
// groups: warp (tg, hg) owns taps k0 + tg + TAPG*t (t < WT) and the azimuth positions of the current
// chunk with (theta - t0) / (CHUNK/THG) == hg.  Azimuth is processed in chunks of CHUNK outputs: the
// gradient chunk and the circular window of S_t it meets are staged in shared memory; lanes stride
// their group's positions, accumulate g * conj(S_t) per tap, reduce across lanes by shuffles and then
// across the azimuth groups in a fixed order, so results are bit-reproducible.
constexpr int WG_THREADS = 1024;
constexpr int WG_WARPS = WG_THREADS / 32;
constexpr int WG_TAPG = 4;                       // tap groups
constexpr int WG_THG = WG_WARPS / WG_TAPG;       // azimuth groups (8)
constexpr int WG_WT = 16;                        // taps per warp per sweep
constexpr int WG_SWEEP = WG_TAPG * WG_WT;        // 64 taps per sweep
constexpr int WG_CHUNK = 1024;
constexpr int WG_SPAN_CAP = 2560;

__device__ __forceinline__ int canon(int o, int n) {
    int c = pmod(o, n);
    return (c > n / 2) ? c - n : c;
}

__global__ void __launch_bounds__(WG_THREADS, 1)
weight_grad_kernel(const float2 *__restrict__ g, const float2 *__restrict__ S_t, const int32_t *__restrict__ o,
                   int o_row_stride, int n_scans, int n_rng, int n_az, int K, float2 *__restrict__ grad_w) {
    __shared__ float2 gs[WG_CHUNK];
    __shared__ float2 ws[WG_CHUNK + WG_SPAN_CAP];
    __shared__ float2 part[WG_THG][WG_SWEEP];
    __shared__ int red_lo[WG_WARPS], red_hi[WG_WARPS];
    const int r = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tg = warp % WG_TAPG, hg = warp / WG_TAPG;
    const int32_t *orow = o + (size_t)r * o_row_stride;

    int lo = INT_MAX, hi = INT_MIN;
    for (int k = threadIdx.x; k < K; k += WG_THREADS) {
        const int c = canon(__ldg(orow + k), n_az);
        lo = min(lo, c);
        hi = max(hi, c);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s));
    }
    if (lane == 0) {
        red_lo[warp] = lo;
        red_hi[warp] = hi;
    }
    __syncthreads();
    lo = red_lo[0];
    hi = red_hi[0];
    for (int i = 1; i < WG_WARPS; ++i) {
        lo = min(lo, red_lo[i]);
        hi = max(hi, red_hi[i]);
    }
    const bool staged = hi - lo <= WG_SPAN_CAP;
    constexpr int PER_G = WG_CHUNK / WG_THG;     // positions per azimuth group per chunk (128)

    for (int k0 = 0; k0 < K; k0 += WG_SWEEP) {
        int rel[WG_WT];
        float2 acc[WG_WT];
#pragma unroll
        for (int t = 0; t < WG_WT; ++t) {
            const int k = k0 + tg + WG_TAPG * t;
            const int c = k < K ? canon(__ldg(orow + k), n_az) : lo;
            rel[t] = staged ? c - lo : c;
            acc[t] = make_float2(0.f, 0.f);
        }
        for (int sc = 0; sc < n_scans; ++sc) {
            const size_t rowoff = ((size_t)sc * n_rng + r) * n_az;
            const float2 *grow = g + rowoff;
            const float2 *srow = S_t + rowoff;
            for (int t0 = 0; t0 < n_az; t0 += WG_CHUNK) {
                const int cw = min(WG_CHUNK, n_az - t0);
                __syncthreads();
                for (int i = threadIdx.x; i < cw; i += WG_THREADS) gs[i] = __ldg(grow + t0 + i);
                if (staged) {
                    const int start = pmod(t0 + lo, n_az);
                    for (int i = threadIdx.x; i < cw + hi - lo; i += WG_THREADS) {
                        int idx = start + i;
                        if (idx >= n_az) idx %= n_az;
                        ws[i] = __ldg(srow + idx);
                    }
                }
                __syncthreads();
                const int i_end = min(cw, (hg + 1) * PER_G);
                for (int i = hg * PER_G + lane; i < i_end; i += 32) {
                    const float2 gv = gs[i];
#pragma unroll
                    for (int t = 0; t < WG_WT; ++t) {
                        const float2 sv = staged ? ws[i + rel[t]] : __ldg(srow + pmod(t0 + i + rel[t], n_az));
                        acc[t].x = fmaf(gv.x, sv.x, acc[t].x);       // g * conj(s)
                        acc[t].x = fmaf(gv.y, sv.y, acc[t].x);
                        acc[t].y = fmaf(gv.y, sv.x, acc[t].y);
                        acc[t].y = fmaf(-gv.x, sv.y, acc[t].y);
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < WG_WT; ++t) {
#pragma unroll
            for (int sft = 16; sft > 0; sft >>= 1) {
                acc[t].x += __shfl_xor_sync(0xffffffffu, acc[t].x, sft);
                acc[t].y += __shfl_xor_sync(0xffffffffu, acc[t].y, sft);
            }
            if (lane == 0) part[hg][tg + WG_TAPG * t] = acc[t];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < WG_SWEEP; j += WG_THREADS) {
            const int k = k0 + j;
            if (k < K) {
                float2 sum = part[0][j];
                for (int q = 1; q < WG_THG; ++q) sum = cadd(sum, part[q][j]);
                grad_w[(size_t)r * K + k] = sum;
            }
        }
    }
}

}  // namespace

rosar_status launch_phase_apply(const float2 *S, const float *eps, int n_scans, int n_rng, int n_az, float2 *S_t,
                                cudaStream_t s) {
    if (n_scans > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "phase_apply: n_scans=%d exceeds 65535", n_scans);
    dim3 grid((n_az + DG_THREADS - 1) / DG_THREADS, n_scans);
    phase_apply_kernel<<<grid, DG_THREADS, 0, s>>>(S, eps, n_rng, n_az, S_t);
    return check_launch("phase_apply");
}

rosar_status launch_phase_grad(const float2 *S_t, const float2 *G, const float *eps, int n_scans, int n_rng, int n_az,
                               float *grad_eps, float2 *grad_S, cudaStream_t s) {
    if (n_scans > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "phase_grad: n_scans=%d exceeds 65535", n_scans);
    dim3 grid((n_az + PG_COLS - 1) / PG_COLS, n_scans);
    phase_grad_kernel<<<grid, DG_THREADS, 0, s>>>(S_t, G, eps, n_rng, n_az, grad_eps, grad_S);
    return check_launch("phase_grad");
}

rosar_status launch_phase_grad_phasor(const float2 *S, const float2 *P, const float2 *G, int n_scans, int n_rng,
                                      int n_az, float *grad_eps, float2 *grad_S, cudaStream_t s) {
    if (n_scans > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "phase_grad_phasor: n_scans=%d exceeds 65535", n_scans);
    dim3 grid((n_az + PG_COLS - 1) / PG_COLS, n_scans);
    phase_grad_phasor_kernel<<<grid, DG_THREADS, 0, s>>>(S, P, G, n_rng, n_az, grad_eps, grad_S);
    return check_launch("phase_grad_phasor");
}

rosar_status launch_phasors(const float *eps, long long n, float2 *P, cudaStream_t s) {
    const long long blocks = (n + DG_THREADS - 1) / DG_THREADS;
    if (blocks > 0x7fffffffLL) return set_error(ROSAR_ERR_UNSUPPORTED, "phasors: n=%lld too large", n);
    phasor_kernel<<<(unsigned)blocks, DG_THREADS, 0, s>>>(eps, n, P);
    return check_launch("phasors");
}

rosar_status launch_azimuth_weight_grad(const float2 *g, const float2 *S_t, const int32_t *o, int o_row_stride,
                                        int n_scans, int n_rng, int n_az, int K, float2 *grad_w, cudaStream_t s) {
    weight_grad_kernel<<<n_rng, WG_THREADS, 0, s>>>(g, S_t, o, o_row_stride, n_scans, n_rng, n_az, K, grad_w);
    return check_launch("azimuth_weight_grad");
}

}  // namespace rosar
