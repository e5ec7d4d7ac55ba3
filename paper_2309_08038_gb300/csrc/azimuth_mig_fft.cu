// K2mf: the range-migration-aware azimuth filter (arXiv 2309.08038, Sec. III-D: the
// per-pulse peak bin l*_n of Eq. (40) inside Eq. (43)) evaluated exactly in the
// azimuth-frequency domain.  Tap k of output row r reads range row r + dl[r][k];
// grouping the taps of row r by their row offset d,
//
//   out[r][.] = sum_d sum_{k: dl[r][k] = d} w[r][k] * S[r+d][(. + o_k) mod N]
//             = sum_d g_{r,d} (*) S[r+d][.],        g_{r,d}[(-o_k) mod N] += w[r][k]
//             = IFFT( sum_d FFT(S[r+d][.]) . FFT(g_{r,d})/N ),
//
// so one forward transform per S row (shared by every output row that reads it) and one
// inverse per output row replace the K-tap gather: the cost of the fixed-row FFT filter
// plus one product per plane d.  Rows r+d outside [0, n_bins) contribute nothing (they
// read zero, as in the gather form).
//
//   plan     H_d[r] = FFT(g_{r,d})/N for d = d_lo .. d_lo+n_d-1 (azimuth_plan_kernel with a
//            row-offset filter, azimuth_fft.cu), digit-reversed order as every plan here;
//   kernel 1 X[b] = DIF(S[b]) for every row b of S (the forward transform, same order);
//   kernel 2 Y_r = sum_d X[r+d] . H_d[r] in increasing d, then conj, DIT, conj (the
//            inverse, natural order), written to out[r].
// Rows with a compile-time plan (360, 1800, 3600, 7200 pulses) run the pass sequence with
// constant strides, the first and last passes of each transform on global memory, the
// inverse launched to overlap the forward kernel's tail; the others the run-time plan.

#include "row_fft.cuh"

namespace rosar {
namespace {

using namespace rowfft;

// One CTA per S row: stage the row (cp.async), build the twiddle table, forward transform, store.
template <typename FWD>
__device__ __forceinline__ void spectrum_row(const float2 *__restrict__ S, float2 *__restrict__ X, int N, int pad_shift,
                                             FWD fwd) {
    extern __shared__ float2 sm[];
    float2 *x = sm;
    float2 *tw = x + padded_len(N);
    const size_t row = (size_t)blockIdx.x * N;
    for (int n = threadIdx.x; n < N; n += blockDim.x) cp_async8(x + rpad(n, pad_shift), S + row + n);
    cp_async_commit();
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    cp_async_wait<0>();
    __syncthreads();
    fwd(x, tc, tf);                                  // ends with a barrier
    for (int n = threadIdx.x; n < N; n += blockDim.x) X[row + n] = x[rpad(n, pad_shift)];
}

// One CTA per output row r: the planes' products summed in increasing d (each thread owns its frequencies,
// so no barrier between planes), conjugated, inverse transform, conjugated store.
template <typename INV>
__device__ __forceinline__ void combine_row(const float2 *__restrict__ X, const float2 *__restrict__ H, int n_bins,
                                            int n_rng, int d_lo, int n_d, int N, int pad_shift, float2 *__restrict__ out,
                                            INV inv) {
    extern __shared__ float2 sm[];
    float2 *x = sm;
    float2 *tw = x + padded_len(N);
    const int r = blockIdx.x;
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        bool any = false;
        for (int i = 0; i < n_d; ++i) {
            const int b = r + d_lo + i;
            if (b < 0 || b >= n_bins) continue;
            const float2 p = cmul(__ldg(H + ((size_t)i * n_rng + r) * N + n), __ldg(X + (size_t)b * N + n));
            acc = any ? cadd(acc, p) : p;
            any = true;
        }
        x[rpad(n, pad_shift)] = make_float2(acc.x, -acc.y);
    }
    __syncthreads();
    inv(x, tc, tf);                                  // ends with a barrier
    const size_t row = (size_t)r * N;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const float2 y = x[rpad(n, pad_shift)];
        out[row + n] = make_float2(y.x, -y.y);
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
azimuth_spectrum_kernel(const float2 *__restrict__ S, int N, RowPlan pl, float2 *__restrict__ X) {
    spectrum_row(S, X, N, pl.pad_shift, [&](float2 *x, const float2 *tc, const float2 *tf) { row_dif(x, N, pl, tc, tf); });
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
azimuth_mig_combine_kernel(const float2 *__restrict__ X, const float2 *__restrict__ H, int n_bins, int n_rng, int d_lo,
                           int n_d, int N, RowPlan pl, float2 *__restrict__ out) {
    combine_row(X, H, n_bins, n_rng, d_lo, n_d, N, pl.pad_shift, out,
                [&](float2 *x, const float2 *tc, const float2 *tf) { row_dit(x, N, pl, tc, tf); });
}

// Compile-time plans (radices R1 .. Rk, no padding).  The forward transform reads S straight into the first DIF
// pass (dif_first_global) and writes its last pass (blocks of Rk, twiddles 1) straight to X; the inverse reads
// the planes' products straight into its first DIT pass (blocks of Rk, twiddles 1) and writes its last pass to
// out (dit_last_global): two shared-memory round trips per transform fewer than staging the rows.

// DIF passes on blocks of M for the radices R, Rest..., the innermost one (M == R) left out.
template <int N, int M, int T, int R, int... Rest>
__device__ __forceinline__ void dif_middle(float2 *x, const float2 *tc, const float2 *tf) {
    if constexpr (sizeof...(Rest) > 0) {
        dif_pass_c<N, M, R, false, T>(x, tc, tf);
        dif_middle<N, M / R, T, Rest...>(x, tc, tf);
    }
}

// DIT passes for the radices R, Rest... (plan order; blocks of M for R), the innermost one left out.
template <int N, int M, int T, int R, int... Rest>
__device__ __forceinline__ void dit_middle(float2 *x, const float2 *tc, const float2 *tf) {
    if constexpr (sizeof...(Rest) > 0) {
        dit_middle<N, M / R, T, Rest...>(x, tc, tf);
        dit_pass_c<N, M, R, false, T>(x, tc, tf);
    }
}

template <int... R>
struct LastRadix;
template <int R>
struct LastRadix<R> {
    static constexpr int value = R;
};
template <int R, int... Rest>
struct LastRadix<R, Rest...> {
    static constexpr int value = sizeof...(Rest) ? LastRadix<Rest...>::value : R;
};

template <int T, int N, int R1, int... Rs>
__global__ void __launch_bounds__(T, 2)
azimuth_spectrum_fixed_kernel(const float2 *__restrict__ S, float2 *__restrict__ X) {
    extern __shared__ float2 sm[];
    constexpr int RK = LastRadix<R1, Rs...>::value;
    float2 *x = sm;
    float2 *tw = x + padded_len(N);
    const size_t row = (size_t)blockIdx.x * N;
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    __syncthreads();
    griddep_launch_dependents();
    griddep_wait();                                  // S is complete (no-op without a programmatic predecessor)
    dif_first_global<N, R1, T, false>(S + row, x, tc, tf);
    dif_middle<N, N / R1, T, Rs...>(x, tc, tf);
#pragma unroll 1
    for (int b = threadIdx.x; b < N / RK; b += T) {   // last DIF pass: blocks of RK, twiddles 1, to X
        float2 v[RK];
#pragma unroll
        for (int q = 0; q < RK; ++q) v[q] = x[b * RK + q];
        small_dft<RK>(v);
#pragma unroll
        for (int q = 0; q < RK; ++q) X[row + b * RK + q] = v[q];
    }
}

template <int T, int N, int R1, int... Rs>
__global__ void __launch_bounds__(T, 2)
azimuth_mig_combine_fixed_kernel(const float2 *__restrict__ X, const float2 *__restrict__ H, int n_bins, int n_rng,
                                 int d_lo, int n_d, float2 *__restrict__ out) {
    extern __shared__ float2 sm[];
    constexpr int RK = LastRadix<R1, Rs...>::value;
    float2 *x = sm;
    float2 *tw = x + padded_len(N);
    const int r = blockIdx.x;
    const float2 *tc, *tf;
    build_twiddles(N, false, tw, &tc, &tf);
    griddep_wait();                                  // X is complete
#pragma unroll 1
    for (int b = threadIdx.x; b < N / RK; b += T) {   // first DIT pass on the planes' products: blocks of RK
        float2 v[RK];
#pragma unroll
        for (int q = 0; q < RK; ++q) v[q] = make_float2(0.f, 0.f);
        bool any = false;
        for (int i = 0; i < n_d; ++i) {
            const int bin = r + d_lo + i;
            if (bin < 0 || bin >= n_bins) continue;
            const float2 *Xr = X + (size_t)bin * N + b * RK;
            const float2 *Hr = H + ((size_t)i * n_rng + r) * N + b * RK;
#pragma unroll
            for (int q = 0; q < RK; ++q) {
                const float2 p = cmul(__ldg(Hr + q), __ldg(Xr + q));
                v[q] = any ? cadd(v[q], p) : p;
            }
            any = true;
        }
#pragma unroll
        for (int q = 0; q < RK; ++q) v[q].y = -v[q].y;
        small_dft<RK>(v);
#pragma unroll
        for (int q = 0; q < RK; ++q) x[b * RK + q] = v[q];
    }
    __syncthreads();
    dit_middle<N, N / R1, T, Rs...>(x, tc, tf);
    dit_last_global<N, R1, T>(x, out + (size_t)r * N, tc, tf);
}

size_t row_smem(int N) { return sizeof(float2) * (size_t)(padded_len(N) + 64 + coarse_len(N)); }

// Both kernels with the compile-time plan when the run-time planner picks exactly these radices for n_az (so the
// spectra and the plans share one order); false to fall back to the run-time plan.
template <int T, int N, int... R>
bool try_fixed_mig(int n_az, const RowPlan &pl, const float2 *S, int n_bins, const float2 *H, int d_lo, int n_d,
                   int n_rng, float2 *X, float2 *out, cudaStream_t s, rosar_status *st) {
    constexpr int rad[] = {R...};
    if (n_az != N || threads_for(N) != T || pl.pad_shift != 31 || pad_shift_for(N) != 31 || pl.npass != (int)sizeof...(R))
        return false;
    for (int i = 0; i < pl.npass; ++i)
        if (pl.rad[i] != rad[i]) return false;
    static int done_a[kMaxDevices] = {}, done_b[kMaxDevices] = {};
    const size_t sm = row_smem(N);
    *st = ensure_smem((const void *)azimuth_spectrum_fixed_kernel<T, N, R...>, sm, done_a, "sparse_azimuth_migrating_fft");
    if (*st == ROSAR_OK)
        *st = ensure_smem((const void *)azimuth_mig_combine_fixed_kernel<T, N, R...>, sm, done_b,
                          "sparse_azimuth_migrating_fft");
    if (*st != ROSAR_OK) return true;
    azimuth_spectrum_fixed_kernel<T, N, R...><<<n_bins, T, sm, s>>>(S, X);
    // the combine kernel's twiddle table overlaps the spectrum kernel's tail (programmatic dependent launch)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_rng);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, azimuth_mig_combine_fixed_kernel<T, N, R...>, (const float2 *)X, H,
                                             n_bins, n_rng, d_lo, n_d, out);
    *st = e != cudaSuccess ? set_error(ROSAR_ERR_CUDA, "sparse_azimuth_migrating_fft: launch failed: %s",
                                       cudaGetErrorString(e))
                           : check_launch("sparse_azimuth_migrating_fft");
    return true;
}

}  // namespace

rosar_status launch_sparse_azimuth_migrating_fft(const float2 *S, int n_bins, const float2 *H, int d_lo, int n_d,
                                                 int n_rng, int n_az, float2 *X, float2 *out, cudaStream_t s) {
    RowPlan pl;
    if (!make_plan(n_az, &pl))
        return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth_migrating_fft: n_az=%d is not 2^a 3^b 5^c in [2, %d]",
                         n_az, AF_MAX_N);
    {
        rosar_status st = ROSAR_OK;
        if (try_fixed_mig<256, 3600, 16, 15, 15>(n_az, pl, S, n_bins, H, d_lo, n_d, n_rng, X, out, s, &st) ||
            try_fixed_mig<256, 1800, 8, 15, 15>(n_az, pl, S, n_bins, H, d_lo, n_d, n_rng, X, out, s, &st) ||
            try_fixed_mig<512, 7200, 8, 4, 15, 15>(n_az, pl, S, n_bins, H, d_lo, n_d, n_rng, X, out, s, &st) ||
            try_fixed_mig<256, 360, 8, 3, 15>(n_az, pl, S, n_bins, H, d_lo, n_d, n_rng, X, out, s, &st))
            return st;
    }
    const size_t sm = row_smem(n_az);
    if (sm > 200 * 1024)
        return set_error(ROSAR_ERR_UNSUPPORTED, "sparse_azimuth_migrating_fft: n_az=%d needs %zu bytes of shared memory",
                         n_az, sm);
    const int T = threads_for(n_az);
    static int done[8][kMaxDevices] = {};
    auto go = [&](auto ka, auto kb, int v) -> rosar_status {
        rosar_status st = ensure_smem((const void *)ka, sm, done[2 * v], "sparse_azimuth_migrating_fft");
        if (st == ROSAR_OK) st = ensure_smem((const void *)kb, sm, done[2 * v + 1], "sparse_azimuth_migrating_fft");
        if (st != ROSAR_OK) return st;
        ka<<<n_bins, T, sm, s>>>(S, n_az, pl, X);
        kb<<<n_rng, T, sm, s>>>(X, H, n_bins, n_rng, d_lo, n_d, n_az, pl, out);
        return check_launch("sparse_azimuth_migrating_fft");
    };
    if (T <= 256) return go(azimuth_spectrum_kernel<256>, azimuth_mig_combine_kernel<256>, 0);
    if (T <= 384) return go(azimuth_spectrum_kernel<384>, azimuth_mig_combine_kernel<384>, 1);
    if (T <= 512) return go(azimuth_spectrum_kernel<512>, azimuth_mig_combine_kernel<512>, 2);
    return go(azimuth_spectrum_kernel<1024>, azimuth_mig_combine_kernel<1024>, 3);
}

}  // namespace rosar
