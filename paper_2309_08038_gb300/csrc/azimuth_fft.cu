// K2b: the sparse-aperture azimuth filter of Eq. (43) evaluated exactly as a circular
// convolution in the azimuth-frequency domain (arXiv 2309.08038, Sec. III-D; the
// pixel-parallel form of Remark 2, here per range row):
//
//   out[r][.] = sum_k w[r][k] * S[r][(. + o_k) mod N] = g_r (*) S[r][.],   g_r[(-o_k) mod N] += w[r][k]
//            = IFFT_N( FFT_N(g_r)/N . FFT_N(S[r][.]) )
//
// The same taps, the same circular modulo; only the summation order differs from the
// gather form.  Work per pixel is O(log N) instead of O(K), so at K >= 32 the
// azimuth stage turns from shared-memory/FMA bound to HBM bound (24 B/px: S, H, out).
//
// One CTA owns one range row, staged in shared memory (one pad element per 16
// against bank conflicts).  The forward transform is an in-place mixed-radix
// decimation-in-frequency FFT (radices 16, 8, 4, 2, 5, 3 and a prime-factor 15; N = 2^a 3^b 5^c <= 16384;
// a planner picks the sequence with the fewest passes, e.g. 3600 = 16*15*15).
// Every butterfly reads and writes the same R slots, so only its own R values are
// live and passes need one barrier each; its twiddles are powers of one table entry.  It leaves the spectrum in digit-reversed
// order; H is produced by the same transform (so it is stored in that order), the
// pointwise product needs no reordering, and the inverse is the transposed
// (decimation-in-time) pass sequence between two conjugations, which restores the
// natural order.  Twiddles exp(-2*pi*i*q/N) come from a two-level shared table
// (q >> 6, q & 63) built per CTA with sincospif.

#include <cooperative_groups.h>

#include "row_fft.cuh"

namespace cg = cooperative_groups;

namespace rosar {
namespace {

using namespace rowfft;

// Shared-memory layout of a row: x [padded], then (stage_h) the H row [padded], then the twiddle table.
struct Layout {
    int full_tab;
    int stage_h;
    size_t bytes;
};

// The row filter on one CTA: stage the H row and the twiddle table, wait for S, forward DIF, product with
// H (digit-reversed order, carries 1/N) between conjugations, DIT, store.  FWD/DIT run the passes.
// Row b of S/out uses row (b mod h_rows) of H (a stack of scans sharing one plan); conj_h applies conj(H), the
// adjoint filter.
// phase (optional): [n_rows / h_rows][N] per-column factors; row b is multiplied by phase row b / h_rows before
// the filter (the scans of a stack each with its own phase correction).  spec (optional): [n_rows][N] the rows'
// forward transforms (digit-reversed order, before the product with H), for the weight gradient.
struct RowMap {
    int h_rows;
    int conj_h;
    const float2 *phase;
    float2 *spec;
};

template <typename FWD, typename INV>
__device__ __forceinline__ void row_filter(const float2 *__restrict__ S, const float2 *__restrict__ H, int N, int pad_shift,
                                           const Layout &lay, RowMap map, float2 *__restrict__ out, FWD fwd, INV inv) {
    extern __shared__ float2 sm[];
    float2 *x = sm;
    float2 *hb = x + padded_len(N);
    float2 *tw = lay.stage_h ? hb + padded_len(N) : hb;
    const size_t row = (size_t)blockIdx.x * N;
    const size_t hrow = (size_t)(blockIdx.x % map.h_rows) * N;
    const float hs = map.conj_h ? -1.f : 1.f;
    // prologue independent of S: the H row and the twiddle table
    if (lay.stage_h)
        for (int n = threadIdx.x; n < N; n += blockDim.x) cp_async8(hb + rpad(n, pad_shift), H + hrow + n);
    cp_async_commit();
    const float2 *tc, *tf;
    build_twiddles(N, lay.full_tab != 0, tw, &tc, &tf);
    griddep_wait();                          // S is complete (no-op unless launched to overlap its producer)
    for (int n = threadIdx.x; n < N; n += blockDim.x) cp_async8(x + rpad(n, pad_shift), S + row + n);
    cp_async_commit();
    cp_async_wait<0>();
    if (map.phase) {                         // each thread scales the elements it staged
        const float2 *ph = map.phase + (size_t)(blockIdx.x / map.h_rows) * N;
        for (int n = threadIdx.x; n < N; n += blockDim.x) x[rpad(n, pad_shift)] = cmul(x[rpad(n, pad_shift)], __ldg(ph + n));
    }
    __syncthreads();
    fwd(x, tc, tf);
    if (map.spec)
        for (int n = threadIdx.x; n < N; n += blockDim.x) map.spec[row + n] = x[rpad(n, pad_shift)];
    if (lay.stage_h) {
        for (int n = threadIdx.x; n < N; n += blockDim.x) {   // spectrum times H (same digit-reversed order, carries 1/N), conjugated
            float2 h = hb[rpad(n, pad_shift)];
            h.y *= hs;
            const float2 y = cmul(h, x[rpad(n, pad_shift)]);
            x[rpad(n, pad_shift)] = make_float2(y.x, -y.y);
        }
    } else {
#pragma unroll 4
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            float2 h = __ldg(H + hrow + n);
            h.y *= hs;
            const float2 y = cmul(h, x[rpad(n, pad_shift)]);
            x[rpad(n, pad_shift)] = make_float2(y.x, -y.y);
        }
    }
    __syncthreads();
    inv(x, tc, tf);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const float2 y = x[rpad(n, pad_shift)];
        out[row + n] = make_float2(y.x, -y.y);
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT == 384 ? 2 : 1))
azimuth_fft_kernel(const float2 *__restrict__ S, const float2 *__restrict__ H, int N, RowPlan pl, Layout lay, RowMap map,
                   float2 *__restrict__ out) {
    row_filter(S, H, N, pl.pad_shift, lay, map, out,
               [&](float2 *x, const float2 *tc, const float2 *tf) { row_dif(x, N, pl, tc, tf); },
               [&](float2 *x, const float2 *tc, const float2 *tf) { row_dit(x, N, pl, tc, tf); });
}

// Compile-time plan for one row length (T threads, no padding: N has an odd factor, H staged): the first pass
// reads S from global memory, the last writes the image, and the last forward pass, the product with H and
// the first inverse pass run as one step (row_filter_fused): four barriers for 16.15.15.
// Rows whose staged pair (S and H) would not fit the 200 KB shared-memory cap of the row layouts read H from
// global memory in the fused step (14400-pulse rows).
template <int N>
constexpr bool stage_h_fits() { return filter_row_smem<N, true>() <= 200 * 1024; }

template <int T, int N, int... R>
__global__ void __launch_bounds__(T, (T <= 256 ? 2 : 1))
azimuth_fft_fixed_kernel(const float2 *__restrict__ S, const float2 *__restrict__ H, RowMap map,
                         float2 *__restrict__ out) {
    extern __shared__ float2 sm[];
    const size_t row = (size_t)blockIdx.x * N;
    const size_t hrow = (size_t)(blockIdx.x % map.h_rows) * N;
    filter_row_cta<T, N, stage_h_fits<N>(), R...>(S + row, H + hrow, map.conj_h != 0, out + row, sm,
                                                  map.phase ? map.phase + (size_t)(blockIdx.x / map.h_rows) * N : nullptr,
                                                  map.spec ? map.spec + row : nullptr);
}

// dl != nullptr: plane blockIdx.y of the range-migration-aware plan, built from the taps of row r whose row
// offset dl[r][k] equals d_lo + blockIdx.y, stored at H[(blockIdx.y * gridDim.x + r) * N].
template <int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT == 384 ? 2 : 1))
azimuth_plan_kernel(const float2 *__restrict__ w, const int32_t *__restrict__ o, int o_row_stride, int K, int N,
                    RowPlan pl, Layout lay, float2 *__restrict__ H, const int32_t *__restrict__ dl = nullptr,
                    int d_lo = 0) {
    extern __shared__ float2 sm[];
    float2 *x = sm;
    float2 *tw = x + padded_len(N);
    const int r = blockIdx.x;
    const int d_sel = d_lo + (int)blockIdx.y;
    H += (size_t)blockIdx.y * gridDim.x * N;
    const float2 *tc, *tf;
    build_twiddles(N, lay.full_tab != 0, tw, &tc, &tf);
    for (int n = threadIdx.x; n < padded_len(N); n += blockDim.x) x[n] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {        // g_r[(-o_k) mod N] += w[r][k]
        if (dl && __ldg(dl + (size_t)r * K + k) != d_sel) continue;
        const long long on = -(long long)__ldg(o + (size_t)r * o_row_stride + k);
        const int n = (int)(((on % N) + N) % N);
        const float2 wv = __ldg(w + (size_t)r * K + k);
        atomicAdd(&x[rpad(n, pl.pad_shift)].x, wv.x);
        atomicAdd(&x[rpad(n, pl.pad_shift)].y, wv.y);
    }
    __syncthreads();
    row_dif(x, N, pl, tc, tf);
    const float inv_n = (float)(1.0 / (double)N);
    for (int n = threadIdx.x; n < N; n += blockDim.x) H[(size_t)r * N + n] = cscale(x[rpad(n, pl.pad_shift)], inv_n);
}

// Weight gradient of the filter for a stack of scans sharing w (the differentiable form), one CTA per row:
//   corr_r[tau] = sum_s sum_t g[s][r][t] conj(S_t[s][r][(t + tau) mod N]) = (1/N) DFT( sum_s G_s . conj(S_s) )[tau]
// with G_s, S_s the forward transforms of the rows.  Both rows of each scan go through the DIF (same
// digit-reversed order, so the product needs no reordering), the cross-spectrum accumulates in shared memory,
// and one DIT pass sequence (a forward DFT of a digit-reversed row, natural-order output) gives every lag;
// grad_w[r][k] = corr_r[o_k mod N].  Work per row: 2 n_scans + 1 transforms instead of n_scans * N * K MACs.
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
azimuth_xspec_kernel(const float2 *__restrict__ g, const float2 *__restrict__ St, const int32_t *__restrict__ o,
                     int o_row_stride, int n_scans, int n_rng, int K, int N, RowPlan pl, float2 *__restrict__ grad_w,
                     const float2 *__restrict__ phase) {
    extern __shared__ float2 sm[];
    const int pn = padded_len(N), sh = pl.pad_shift;
    float2 *P = sm;
    float2 *x = P + pn;
    float2 *y = x + pn;
    float2 *tw = y + pn;
    const int r = blockIdx.x;
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    for (int n = threadIdx.x; n < pn; n += blockDim.x) P[n] = make_float2(0.f, 0.f);
    for (int sc = 0; sc < n_scans; ++sc) {
        const size_t row = ((size_t)sc * n_rng + r) * N;
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            cp_async8(x + rpad(n, sh), g + row + n);
            cp_async8(y + rpad(n, sh), St + row + n);
        }
        cp_async_commit();
        cp_async_wait<0>();
        if (phase)                            // S_t = S e^{j eps}: each thread scales the elements it staged
            for (int n = threadIdx.x; n < N; n += blockDim.x)
                y[rpad(n, sh)] = cmul(y[rpad(n, sh)], __ldg(phase + (size_t)sc * N + n));
        __syncthreads();
        row_dif(x, N, pl, tc, tf);
        row_dif(y, N, pl, tc, tf);
        for (int n = threadIdx.x; n < N; n += blockDim.x) {      // P += X . conj(Y), same digit-reversed slot
            const float2 a = x[rpad(n, sh)], b = y[rpad(n, sh)];
            float2 &p = P[rpad(n, sh)];
            p.x = fmaf(a.x, b.x, fmaf(a.y, b.y, p.x));
            p.y = fmaf(a.y, b.x, fmaf(-a.x, b.y, p.y));
        }
        __syncthreads();
    }
    row_dit(P, N, pl, tc, tf);
    const float inv_n = (float)(1.0 / (double)N);
    const int32_t *orow = o + (size_t)r * o_row_stride;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int tau = pmod(__ldg(orow + k), N);
        grad_w[(size_t)r * K + k] = cscale(P[rpad(tau, sh)], inv_n);
    }
}

// Compile-time-plan form of the weight gradient: the scans of a row are split over a cluster of G CTAs
// (rank c takes scans c, c + G, ...).  Each CTA transforms its rows with the first DIF pass read straight from
// global memory and the last DIF pass of both rows fused with the accumulation P += X . conj(Y); rank 0 then
// adds the other ranks' partial cross-spectra from distributed shared memory in rank order (deterministic),
// runs the DIT sequence and samples the taps.  grid = (G, n_rng), cluster (G, 1, 1).
template <int N, int M, int T, int R, int... Rest>
__device__ __forceinline__ void xspec_tail(float2 *x, float2 *y, float2 *P, const float2 *tc, const float2 *tf) {
    if constexpr (sizeof...(Rest) == 0) {
        static_assert(M == R, "the last radix spans the last block");
#pragma unroll 1
        for (int b = threadIdx.x; b < N / R; b += T) {
            float2 v[R], u[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                v[q] = x[b * R + q];
                u[q] = y[b * R + q];
            }
            small_dft<R>(v);
            small_dft<R>(u);
#pragma unroll
            for (int q = 0; q < R; ++q) {             // P += X . conj(Y)
                float2 &p = P[b * R + q];
                p.x = fmaf(v[q].x, u[q].x, fmaf(v[q].y, u[q].y, p.x));
                p.y = fmaf(v[q].y, u[q].x, fmaf(-v[q].x, u[q].y, p.y));
            }
        }
        __syncthreads();
    } else {
        dif_pass_c<N, M, R, false, T>(x, tc, tf);
        dif_pass_c<N, M, R, false, T>(y, tc, tf);
        xspec_tail<N, M / R, T, Rest...>(x, y, P, tc, tf);
    }
}

template <int T, int N, int R1, int... Rs>
__global__ void __launch_bounds__(T, 2)
azimuth_xspec_fixed_kernel(const float2 *__restrict__ g, const float2 *__restrict__ St, const int32_t *__restrict__ o,
                           int o_row_stride, int n_scans, int n_rng, int K, float2 *__restrict__ grad_w,
                           const float2 *__restrict__ phase) {
    extern __shared__ float2 sm[];
    cg::cluster_group cluster = cg::this_cluster();
    const int G = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int r = blockIdx.y;
    float2 *P = sm;
    float2 *x = P + padded_len(N);
    float2 *y = x + padded_len(N);
    float2 *tw = y + padded_len(N);
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    for (int n = threadIdx.x; n < N; n += T) P[n] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int sc = rank; sc < n_scans; sc += G) {
        const size_t row = ((size_t)sc * n_rng + r) * N;
        dif_first_global<N, R1, T, false>(g + row, x, tc, tf);
        dif_first_global<N, R1, T, false>(St + row, y, tc, tf, false, phase ? phase + (size_t)sc * N : nullptr);
        xspec_tail<N, N / R1, T, Rs...>(x, y, P, tc, tf);
    }
    cluster.sync();
    if (rank == 0) {
        for (int n = threadIdx.x; n < N; n += T) {
            float2 acc = P[n];
            for (int c = 1; c < G; ++c) {
                const float2 v = cluster.map_shared_rank(P, c)[n];
                acc.x += v.x;
                acc.y += v.y;
            }
            P[n] = acc;
        }
    }
    cluster.sync();                       // the other ranks' partial sums stay alive until rank 0 has read them
    if (rank != 0) return;
    dit_seq<N, N, false, T, R1, Rs...>(P, tc, tf);
    const float inv_n = (float)(1.0 / (double)N);
    const int32_t *orow = o + (size_t)r * o_row_stride;
    for (int k = threadIdx.x; k < K; k += T) {
        const int tau = pmod(__ldg(orow + k), N);
        grad_w[(size_t)r * K + k] = cscale(P[tau], inv_n);
    }
}

// Weight gradient from stored spectra (the forward filter's transforms X_s of the corrected rows and the adjoint
// filter's transforms G_s of the image gradient, both digit-reversed), in two launches: the cross-spectrum
// P[r][f] = sum_s G_s[r][f] conj(X_s[r][f]) elementwise (one thread per (row, frequency), scans in order: a pure
// stream of 16 B per pixel), then per row one inverse-order DIT of P and the taps sampled.  No forward transform
// is repeated.
__global__ void __launch_bounds__(256)
xspec_accumulate_kernel(const float2 *__restrict__ G, const float2 *__restrict__ X, int n_scans, long long plane,
                        float2 *__restrict__ P) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= plane) return;
    float2 p = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int sc = 0; sc < n_scans; ++sc) {
        const float2 a = __ldg(G + sc * plane + i), b = __ldg(X + sc * plane + i);
        p.x = fmaf(a.x, b.x, fmaf(a.y, b.y, p.x));     // P += G . conj(X)
        p.y = fmaf(a.y, b.x, fmaf(-a.x, b.y, p.y));
    }
    P[i] = p;
}

// rk > 0: the spectra came from the compile-time-plan filter, stored radix-major for its last radix rk (element
// i = q*(N/rk) + b holds digit-reversed position b*rk + q); rk == 0: stored in digit-reversed order.
template <typename INV>
__device__ __forceinline__ void xspec_taps_row(const float2 *__restrict__ Pg, const int32_t *__restrict__ o,
                                               int o_row_stride, int K, int N, int pad_shift, int rk,
                                               float2 *__restrict__ grad_w, INV inv) {
    extern __shared__ float2 sm[];
    float2 *P = sm;
    float2 *tw = P + padded_len(N);
    const int r = blockIdx.x;
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    const int nb = rk > 0 ? N / rk : N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int q = i / nb, b = i - q * nb;
        P[rpad(rk > 0 ? b * rk + q : i, pad_shift)] = __ldg(Pg + (size_t)r * N + i);
    }
    __syncthreads();
    inv(P, tc, tf);
    const float inv_n = (float)(1.0 / (double)N);
    const int32_t *orow = o + (size_t)r * o_row_stride;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int tau = pmod(__ldg(orow + k), N);
        grad_w[(size_t)r * K + k] = cscale(P[rpad(tau, pad_shift)], inv_n);
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
xspec_taps_kernel(const float2 *__restrict__ P, const int32_t *__restrict__ o, int o_row_stride, int K, int N,
                  RowPlan pl, float2 *__restrict__ grad_w) {
    xspec_taps_row(P, o, o_row_stride, K, N, pl.pad_shift, 0, grad_w,
                   [&](float2 *x, const float2 *tc, const float2 *tf) { row_dit(x, N, pl, tc, tf); });
}

template <int... R>
constexpr int last_of() {
    constexpr int r[] = {R...};
    return r[sizeof...(R) - 1];
}

template <int T, int N, int... R>
__global__ void __launch_bounds__(T, 2)
xspec_taps_fixed_kernel(const float2 *__restrict__ P, const int32_t *__restrict__ o, int o_row_stride, int K,
                        float2 *__restrict__ grad_w) {
    xspec_taps_row(P, o, o_row_stride, K, N, 31, last_of<R...>(), grad_w,
                   [](float2 *x, const float2 *tc, const float2 *tf) { dit_seq<N, N, false, T, R...>(x, tc, tf); });
}

constexpr size_t AF_SMEM_CAP = 200 * 1024;

Layout layout_for(int N, bool with_h) {
    Layout l{};
    const size_t row = sizeof(float2) * (size_t)padded_len(N);
    const size_t two = sizeof(float2) * (size_t)(64 + coarse_len(N));
    l.stage_h = with_h && (2 * row + two <= AF_SMEM_CAP);
    l.full_tab = 0;      // two-level table: ~N/64 + 64 sincospif per CTA instead of N
    l.bytes = row * (l.stage_h ? 2 : 1) + two;
    return l;
}

template <typename F256, typename F384, typename F512, typename F1024>
rosar_status launch_rows(int N, int rows, size_t sm, F256 f256, F384 f384, F512 f512, F1024 f1024,
                         const void *const k[4], int (*done)[kMaxDevices], const char *what) {
    const int T = threads_for(N);
    const int v = T <= 256 ? 0 : T <= 384 ? 1 : T <= 512 ? 2 : 3;
    rosar_status st = ensure_smem(k[v], sm, done[v], what);
    if (st != ROSAR_OK) return st;
    if (v == 0) f256(rows, T, sm);
    else if (v == 1) f384(rows, T, sm);
    else if (v == 2) f512(rows, T, sm);
    else f1024(rows, T, sm);
    return check_launch(what);
}

}  // namespace

int azimuth_fft_supported(int n_az) {
    RowPlan pl;
    return make_plan(n_az, &pl) ? 1 : 0;
}

template <int MAXT>
cudaError_t launch_fft_rows(int g, int t, size_t sm, cudaStream_t s, bool overlap, const float2 *S, const float2 *H,
                            int N, const RowPlan &pl, const Layout &lay, RowMap map, float2 *out) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g);
    cfg.blockDim = dim3(t);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = overlap ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, azimuth_fft_kernel<MAXT>, S, H, N, pl, lay, map, out);
}

namespace {

// Launches the compile-time-plan kernel when the run-time planner picks exactly its radices for n_az (so H,
// made by the run-time plan, is in the same order); returns false to fall back to the run-time plan.
template <int T, int N, int... R>
bool try_fixed(int n_az, const RowPlan &pl, int n_rng, RowMap map, bool ov, const float2 *S, const float2 *H,
               float2 *out, cudaStream_t s, cudaError_t *le, rosar_status *st) {
    constexpr int rad[] = {R...};
    if (n_az != N || threads_for(N) != T || pl.pad_shift != pad_shift_for(N) || pad_shift_for(N) != 31 ||
        pl.npass != (int)sizeof...(R))
        return false;
    for (int i = 0; i < pl.npass; ++i)
        if (pl.rad[i] != rad[i]) return false;
    static int done[kMaxDevices] = {};
    const void *k = (const void *)azimuth_fft_fixed_kernel<T, N, R...>;
    constexpr size_t smem = filter_row_smem<N, stage_h_fits<N>()>();
    *st = ensure_smem(k, smem, done, "azimuth_fft");
    if (*st != ROSAR_OK) return true;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_rng);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = ov ? 1 : 0;
    *le = cudaLaunchKernelEx(&cfg, azimuth_fft_fixed_kernel<T, N, R...>, S, H, map, out);
    *st = check_launch("azimuth_fft");
    return true;
}

}  // namespace

rosar_status launch_azimuth_fft(const float2 *S, const float2 *H, int n_rng, int n_az, float2 *out, cudaStream_t s,
                                bool overlap_predecessor, int h_rows, bool conj_h, const float2 *phase, float2 *spec) {
    const RowMap map{h_rows > 0 ? h_rows : n_rng, conj_h ? 1 : 0, phase, spec};
    RowPlan pl;
    if (!make_plan(n_az, &pl))
        return set_error(ROSAR_ERR_UNSUPPORTED, "azimuth_fft: n_az=%d is not 2^a 3^b 5^c in [2, %d]", n_az, AF_MAX_N);
    static int done[4][kMaxDevices] = {};
    const Layout lay = layout_for(n_az, true);
    const bool ov = overlap_predecessor;
    {
        cudaError_t fle = cudaSuccess;
        rosar_status fst = ROSAR_OK;
        if (try_fixed<256, 3600, 16, 15, 15>(n_az, pl, n_rng, map, ov, S, H, out, s, &fle, &fst) ||
            try_fixed<256, 1800, 8, 15, 15>(n_az, pl, n_rng, map, ov, S, H, out, s, &fle, &fst) ||
            try_fixed<512, 7200, 8, 4, 15, 15>(n_az, pl, n_rng, map, ov, S, H, out, s, &fle, &fst) ||
            try_fixed<1024, 14400, 8, 8, 15, 15>(n_az, pl, n_rng, map, ov, S, H, out, s, &fle, &fst) ||
            try_fixed<256, 360, 8, 3, 15>(n_az, pl, n_rng, map, ov, S, H, out, s, &fle, &fst)) {
            if (fst == ROSAR_OK && fle != cudaSuccess)
                return set_error(ROSAR_ERR_CUDA, "azimuth_fft: launch failed: %s", cudaGetErrorString(fle));
            return fst;
        }
    }
    cudaError_t le = cudaSuccess;
    static const void *const ks[4] = {(const void *)azimuth_fft_kernel<256>, (const void *)azimuth_fft_kernel<384>,
                                      (const void *)azimuth_fft_kernel<512>, (const void *)azimuth_fft_kernel<1024>};
    rosar_status st = launch_rows(
        n_az, n_rng, lay.bytes,
        [&](int g, int t, size_t sm) { le = launch_fft_rows<256>(g, t, sm, s, ov, S, H, n_az, pl, lay, map, out); },
        [&](int g, int t, size_t sm) { le = launch_fft_rows<384>(g, t, sm, s, ov, S, H, n_az, pl, lay, map, out); },
        [&](int g, int t, size_t sm) { le = launch_fft_rows<512>(g, t, sm, s, ov, S, H, n_az, pl, lay, map, out); },
        [&](int g, int t, size_t sm) { le = launch_fft_rows<1024>(g, t, sm, s, ov, S, H, n_az, pl, lay, map, out); },
        ks, done, "azimuth_fft");
    if (st == ROSAR_OK && le != cudaSuccess)
        return set_error(ROSAR_ERR_CUDA, "azimuth_fft: launch failed: %s", cudaGetErrorString(le));
    return st;
}

namespace {

// Launches the cluster-split weight gradient when n_az has this compile-time plan (the planner's radices);
// returns false to fall back to one CTA per row.
template <int T, int N, int... R>
bool try_xspec_fixed(int n_az, const RowPlan &pl, const float2 *g, const float2 *S_t, const int32_t *o,
                     int o_row_stride, int n_scans, int n_rng, int K, float2 *grad_w, cudaStream_t s,
                     rosar_status *st, const float2 *phase) {
    constexpr int rad[] = {R...};
    if (n_az != N || threads_for(N) != T || pl.npass != (int)sizeof...(R) || n_rng > 65535) return false;
    for (int i = 0; i < pl.npass; ++i)
        if (pl.rad[i] != rad[i]) return false;
    static int done[kMaxDevices] = {};
    const void *k = (const void *)azimuth_xspec_fixed_kernel<T, N, R...>;
    constexpr size_t smem = sizeof(float2) * (3 * (size_t)padded_len(N) + 64 + coarse_len(N));
    *st = ensure_smem(k, smem, done, "weight_grad_fft");
    if (*st != ROSAR_OK) return true;
    // scans per CTA: about 4 (G = 4 at 16 scans), G a power of two <= 8 and <= n_scans
    int G = 1;
    while (G < 8 && 2 * G <= n_scans && 4 * G < n_scans) G *= 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G, n_rng);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = G;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, azimuth_xspec_fixed_kernel<T, N, R...>, g, S_t, o, o_row_stride,
                                             n_scans, n_rng, K, grad_w, phase);
    *st = e != cudaSuccess ? set_error(ROSAR_ERR_CUDA, "weight_grad_fft: launch failed: %s", cudaGetErrorString(e))
                           : check_launch("weight_grad_fft");
    return true;
}

}  // namespace

rosar_status launch_azimuth_weight_grad_fft(const float2 *g, const float2 *S_t, const int32_t *o, int o_row_stride,
                                            int n_scans, int n_rng, int n_az, int K, float2 *grad_w, cudaStream_t s,
                                            const float2 *phase) {
    RowPlan pl;
    if (!make_plan(n_az, &pl))
        return set_error(ROSAR_ERR_UNSUPPORTED, "weight_grad_fft: n_az=%d is not 2^a 3^b 5^c in [2, %d]", n_az, AF_MAX_N);
    {
        rosar_status st = ROSAR_OK;
        if (try_xspec_fixed<256, 3600, 16, 15, 15>(n_az, pl, g, S_t, o, o_row_stride, n_scans, n_rng, K, grad_w, s,
                                                   &st, phase) ||
            try_xspec_fixed<256, 1800, 8, 15, 15>(n_az, pl, g, S_t, o, o_row_stride, n_scans, n_rng, K, grad_w, s,
                                                  &st, phase) ||
            try_xspec_fixed<256, 360, 8, 3, 15>(n_az, pl, g, S_t, o, o_row_stride, n_scans, n_rng, K, grad_w, s, &st,
                                                phase))
            return st;
    }
    const size_t bytes = sizeof(float2) * (3 * (size_t)padded_len(n_az) + 64 + coarse_len(n_az));
    if (bytes > AF_SMEM_CAP)
        return set_error(ROSAR_ERR_UNSUPPORTED, "weight_grad_fft: n_az=%d needs %zu bytes of shared memory", n_az, bytes);
    static int done[4][kMaxDevices] = {};
    static const void *const ks[4] = {(const void *)azimuth_xspec_kernel<256>, (const void *)azimuth_xspec_kernel<384>,
                                      (const void *)azimuth_xspec_kernel<512>, (const void *)azimuth_xspec_kernel<1024>};
    return launch_rows(
        n_az, n_rng, bytes,
        [&](int gr, int t, size_t sm) { azimuth_xspec_kernel<256><<<gr, t, sm, s>>>(g, S_t, o, o_row_stride, n_scans, n_rng, K, n_az, pl, grad_w, phase); },
        [&](int gr, int t, size_t sm) { azimuth_xspec_kernel<384><<<gr, t, sm, s>>>(g, S_t, o, o_row_stride, n_scans, n_rng, K, n_az, pl, grad_w, phase); },
        [&](int gr, int t, size_t sm) { azimuth_xspec_kernel<512><<<gr, t, sm, s>>>(g, S_t, o, o_row_stride, n_scans, n_rng, K, n_az, pl, grad_w, phase); },
        [&](int gr, int t, size_t sm) { azimuth_xspec_kernel<1024><<<gr, t, sm, s>>>(g, S_t, o, o_row_stride, n_scans, n_rng, K, n_az, pl, grad_w, phase); },
        ks, done, "weight_grad_fft");
}

namespace {
template <int T, int N, int... R>
bool try_xspec_taps_fixed(int n_az, const RowPlan &pl, const float2 *P, const int32_t *o, int o_row_stride, int n_rng,
                          int K, float2 *grad_w, cudaStream_t s, rosar_status *st) {
    constexpr int rad[] = {R...};
    if (n_az != N || threads_for(N) != T || pl.pad_shift != 31 || pl.npass != (int)sizeof...(R)) return false;
    for (int i = 0; i < pl.npass; ++i)
        if (pl.rad[i] != rad[i]) return false;
    static int done[kMaxDevices] = {};
    const size_t smem = sizeof(float2) * ((size_t)padded_len(N) + 64 + coarse_len(N));
    *st = ensure_smem((const void *)xspec_taps_fixed_kernel<T, N, R...>, smem, done, "weight_grad_spectra");
    if (*st != ROSAR_OK) return true;
    xspec_taps_fixed_kernel<T, N, R...><<<n_rng, T, smem, s>>>(P, o, o_row_stride, K, grad_w);
    *st = check_launch("weight_grad_spectra");
    return true;
}
}  // namespace

rosar_status launch_azimuth_weight_grad_spectra(const float2 *G, const float2 *X, const int32_t *o, int o_row_stride,
                                                int n_scans, int n_rng, int n_az, int K, float2 *P, float2 *grad_w,
                                                cudaStream_t s) {
    RowPlan pl;
    if (!make_plan(n_az, &pl))
        return set_error(ROSAR_ERR_UNSUPPORTED, "weight_grad_spectra: n_az=%d is not 2^a 3^b 5^c in [2, %d]", n_az,
                         AF_MAX_N);
    const long long plane = (long long)n_rng * n_az;
    xspec_accumulate_kernel<<<(unsigned)((plane + 255) / 256), 256, 0, s>>>(G, X, n_scans, plane, P);
    rosar_status st = check_launch("weight_grad_spectra");
    if (st != ROSAR_OK) return st;
    if (try_xspec_taps_fixed<256, 3600, 16, 15, 15>(n_az, pl, P, o, o_row_stride, n_rng, K, grad_w, s, &st) ||
        try_xspec_taps_fixed<256, 1800, 8, 15, 15>(n_az, pl, P, o, o_row_stride, n_rng, K, grad_w, s, &st) ||
        try_xspec_taps_fixed<512, 7200, 8, 4, 15, 15>(n_az, pl, P, o, o_row_stride, n_rng, K, grad_w, s, &st) ||
        try_xspec_taps_fixed<256, 360, 8, 3, 15>(n_az, pl, P, o, o_row_stride, n_rng, K, grad_w, s, &st))
        return st;
    const size_t bytes = sizeof(float2) * ((size_t)padded_len(n_az) + 64 + coarse_len(n_az));
    static int done[4][kMaxDevices] = {};
    static const void *const ks[4] = {(const void *)xspec_taps_kernel<256>, (const void *)xspec_taps_kernel<384>,
                                      (const void *)xspec_taps_kernel<512>, (const void *)xspec_taps_kernel<1024>};
    return launch_rows(
        n_az, n_rng, bytes,
        [&](int gr, int t, size_t sm) { xspec_taps_kernel<256><<<gr, t, sm, s>>>(P, o, o_row_stride, K, n_az, pl, grad_w); },
        [&](int gr, int t, size_t sm) { xspec_taps_kernel<384><<<gr, t, sm, s>>>(P, o, o_row_stride, K, n_az, pl, grad_w); },
        [&](int gr, int t, size_t sm) { xspec_taps_kernel<512><<<gr, t, sm, s>>>(P, o, o_row_stride, K, n_az, pl, grad_w); },
        [&](int gr, int t, size_t sm) { xspec_taps_kernel<1024><<<gr, t, sm, s>>>(P, o, o_row_stride, K, n_az, pl, grad_w); },
        ks, done, "weight_grad_spectra");
}

rosar_status launch_azimuth_plan(const float2 *w, const int32_t *o, int o_row_stride, int n_rng, int n_az, int K,
                                 float2 *H, cudaStream_t s, const int32_t *dl, int d_lo, int n_d) {
    RowPlan pl;
    if (!make_plan(n_az, &pl))
        return set_error(ROSAR_ERR_UNSUPPORTED, "azimuth_plan: n_az=%d is not 2^a 3^b 5^c in [2, %d]", n_az, AF_MAX_N);
    static int done[4][kMaxDevices] = {};
    const Layout lay = layout_for(n_az, false);
    static const void *const ks[4] = {(const void *)azimuth_plan_kernel<256>, (const void *)azimuth_plan_kernel<384>,
                                      (const void *)azimuth_plan_kernel<512>, (const void *)azimuth_plan_kernel<1024>};
    const dim3 grid(n_rng, dl ? n_d : 1);
    return launch_rows(
        n_az, n_rng, lay.bytes,
        [&](int, int t, size_t sm) { azimuth_plan_kernel<256><<<grid, t, sm, s>>>(w, o, o_row_stride, K, n_az, pl, lay, H, dl, d_lo); },
        [&](int, int t, size_t sm) { azimuth_plan_kernel<384><<<grid, t, sm, s>>>(w, o, o_row_stride, K, n_az, pl, lay, H, dl, d_lo); },
        [&](int, int t, size_t sm) { azimuth_plan_kernel<512><<<grid, t, sm, s>>>(w, o, o_row_stride, K, n_az, pl, lay, H, dl, d_lo); },
        [&](int, int t, size_t sm) { azimuth_plan_kernel<1024><<<grid, t, sm, s>>>(w, o, o_row_stride, K, n_az, pl, lay, H, dl, d_lo); },
        ks, done, "azimuth_plan");
}

}  // namespace rosar
