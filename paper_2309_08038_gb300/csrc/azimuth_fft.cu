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
// decimation-in-frequency FFT (radices 16, 8, 4, 2, 5, 3; N = 2^a 3^b 5^c <= 16384):
// every butterfly reads and writes the same R slots, so only its own R values are
// live and passes need one barrier each.  It leaves the spectrum in digit-reversed
// order; H is produced by the same transform (so it is stored in that order), the
// pointwise product needs no reordering, and the inverse is the transposed
// (decimation-in-time) pass sequence between two conjugations, which restores the
// natural order.  Twiddles exp(-2*pi*i*q/N) come from a two-level shared table
// (q >> 6, q & 63) built per CTA with sincospif.

#include "fft_tile.cuh"

namespace rosar {
namespace {

constexpr int AF_MAX_N = 16384;
constexpr int AF_MAXPASS = 16;

struct RowPlan {
    int npass;
    int rad[AF_MAXPASS];
};

__host__ __device__ constexpr int padded_len(int n) { return n + n / 16 + 1; }
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
    const float2 a = make_float2(fmaf(-0.5f, t1.x, v[0].x), fmaf(-0.5f, t1.y, v[0].y));
    const float2 b = make_float2(h * t2.x, h * t2.y);           // y1 = a - i b, y2 = a + i b
    v[0] = y0;
    v[1] = make_float2(a.x + b.y, a.y - b.x);
    v[2] = make_float2(a.x - b.y, a.y + b.x);
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
    const float2 a1 = make_float2(fmaf(c1, t1.x, fmaf(c2, t2.x, x0.x)), fmaf(c1, t1.y, fmaf(c2, t2.y, x0.y)));
    const float2 a2 = make_float2(fmaf(c2, t1.x, fmaf(c1, t2.x, x0.x)), fmaf(c2, t1.y, fmaf(c1, t2.y, x0.y)));
    const float2 b1 = make_float2(fmaf(s1, t3.x, s2 * t4.x), fmaf(s1, t3.y, s2 * t4.y));
    const float2 b2 = make_float2(fmaf(s2, t3.x, -s1 * t4.x), fmaf(s2, t3.y, -s1 * t4.y));
    v[0] = make_float2(x0.x + t1.x + t2.x, x0.y + t1.y + t2.y);
    v[1] = make_float2(a1.x + b1.y, a1.y - b1.x);              // a1 - i b1
    v[4] = make_float2(a1.x - b1.y, a1.y + b1.x);              // a1 + i b1
    v[2] = make_float2(a2.x + b2.y, a2.y - b2.x);              // a2 - i b2
    v[3] = make_float2(a2.x - b2.y, a2.y + b2.x);              // a2 + i b2
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

__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

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

// exp(-2*pi*i*q/N), 0 <= q < N, from the coarse (q >> 6) and fine (q & 63) tables
__device__ __forceinline__ float2 twiddle(int q, const float2 *tc, const float2 *tf) {
    return cmul(tc[q >> 6], tf[q & 63]);
}

// One in-place decimation-in-frequency stage: radix R on blocks of length M (stride s = M/R):
// v = DFT_R(x[base + r*s]); x[base + q*s] = v[q] * W_M^(j*q).
template <int R>
__device__ __forceinline__ void dif_pass(float2 *x, int N, int M, const float2 *tc, const float2 *tf) {
    const int s = M / R, tstep = N / M, nb = N / R;
    const float inv_s = 1.f / (float)s;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int blk = quot(idx, inv_s), j = idx - blk * s;
        const int base = blk * M + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[pad16(base + r * s)];
        small_dft<R>(v);
        x[pad16(base)] = v[0];
#pragma unroll
        for (int q = 1; q < R; ++q) x[pad16(base + q * s)] = cmul(v[q], twiddle(j * q * tstep, tc, tf));
    }
    __syncthreads();
}

// The transposed stage (decimation in time): v[q] = x[base + q*s] * W_M^(j*q); x[base + r*s] = DFT_R(v)[r].
template <int R>
__device__ __forceinline__ void dit_pass(float2 *x, int N, int M, const float2 *tc, const float2 *tf) {
    const int s = M / R, tstep = N / M, nb = N / R;
    const float inv_s = 1.f / (float)s;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int blk = quot(idx, inv_s), j = idx - blk * s;
        const int base = blk * M + j;
        float2 v[R];
        v[0] = x[pad16(base)];
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmul(x[pad16(base + q * s)], twiddle(j * q * tstep, tc, tf));
        small_dft<R>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) x[pad16(base + r * s)] = v[r];
    }
    __syncthreads();
}

template <bool DIF>
__device__ __forceinline__ void stage(int R, float2 *x, int N, int M, const float2 *tc, const float2 *tf) {
    switch (R) {
        case 16: DIF ? dif_pass<16>(x, N, M, tc, tf) : dit_pass<16>(x, N, M, tc, tf); break;
        case 8: DIF ? dif_pass<8>(x, N, M, tc, tf) : dit_pass<8>(x, N, M, tc, tf); break;
        case 4: DIF ? dif_pass<4>(x, N, M, tc, tf) : dit_pass<4>(x, N, M, tc, tf); break;
        case 2: DIF ? dif_pass<2>(x, N, M, tc, tf) : dit_pass<2>(x, N, M, tc, tf); break;
        case 5: DIF ? dif_pass<5>(x, N, M, tc, tf) : dit_pass<5>(x, N, M, tc, tf); break;
        default: DIF ? dif_pass<3>(x, N, M, tc, tf) : dit_pass<3>(x, N, M, tc, tf); break;
    }
}

// Forward DFT of the row, output in digit-reversed order.
__device__ __forceinline__ void row_dif(float2 *x, int N, const RowPlan &pl, const float2 *tc, const float2 *tf) {
    int M = N;
    for (int p = 0; p < pl.npass; ++p) {
        stage<true>(pl.rad[p], x, N, M, tc, tf);
        M /= pl.rad[p];
    }
}

// Forward DFT of a row held in digit-reversed order, output in natural order.
__device__ __forceinline__ void row_dit(float2 *x, int N, const RowPlan &pl, const float2 *tc, const float2 *tf) {
    int M = 1;
    for (int p = pl.npass - 1; p >= 0; --p) {
        M *= pl.rad[p];
        stage<false>(pl.rad[p], x, N, M, tc, tf);
    }
}

__device__ __forceinline__ void build_twiddles(int N, float2 *tc, float2 *tf) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        float s, c;
        sincospif(2.f * (float)i / (float)N, &s, &c);
        tf[i] = make_float2(c, -s);
    }
    for (int i = threadIdx.x; i < coarse_len(N); i += blockDim.x) {
        float s, c;
        sincospif(2.f * (float)(64 * i) / (float)N, &s, &c);
        tc[i] = make_float2(c, -s);
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT)
azimuth_fft_kernel(const float2 *__restrict__ S, const float2 *__restrict__ H, int N, RowPlan pl, int stage_h,
                   float2 *__restrict__ out) {
    extern __shared__ float2 sm[];
    float2 *x = sm;
    float2 *tf = x + padded_len(N);
    float2 *tc = tf + 64;
    float2 *hb = tc + coarse_len(N);        // H row, staged while the forward transform runs (stage_h)
    const size_t row = (size_t)blockIdx.x * N;
    for (int n = threadIdx.x; n < N; n += blockDim.x) cp_async8(x + pad16(n), S + row + n);
    cp_async_commit();
    if (stage_h)
        for (int n = threadIdx.x; n < N; n += blockDim.x) cp_async8(hb + pad16(n), H + row + n);
    cp_async_commit();
    build_twiddles(N, tc, tf);
    cp_async_wait<1>();
    __syncthreads();
    row_dif(x, N, pl, tc, tf);
    cp_async_wait<0>();
    __syncthreads();
    if (stage_h) {
        for (int n = threadIdx.x; n < N; n += blockDim.x) {   // spectrum times H (same digit-reversed order, carries 1/N), conjugated
            const float2 y = cmul(hb[pad16(n)], x[pad16(n)]);
            x[pad16(n)] = make_float2(y.x, -y.y);
        }
    } else {
#pragma unroll 4
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            const float2 y = cmul(__ldg(H + row + n), x[pad16(n)]);
            x[pad16(n)] = make_float2(y.x, -y.y);
        }
    }
    __syncthreads();
    row_dit(x, N, pl, tc, tf);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const float2 y = x[pad16(n)];
        out[row + n] = make_float2(y.x, -y.y);
    }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT)
azimuth_plan_kernel(const float2 *__restrict__ w, const int32_t *__restrict__ o, int o_row_stride, int K, int N,
                    RowPlan pl, float2 *__restrict__ H) {
    extern __shared__ float2 sm[];
    float2 *x = sm;
    float2 *tf = x + padded_len(N);
    float2 *tc = tf + 64;
    const int r = blockIdx.x;
    build_twiddles(N, tc, tf);
    for (int n = threadIdx.x; n < padded_len(N); n += blockDim.x) x[n] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {        // g_r[(-o_k) mod N] += w[r][k]
        const long long on = -(long long)__ldg(o + (size_t)r * o_row_stride + k);
        const int n = (int)(((on % N) + N) % N);
        const float2 wv = __ldg(w + (size_t)r * K + k);
        atomicAdd(&x[pad16(n)].x, wv.x);
        atomicAdd(&x[pad16(n)].y, wv.y);
    }
    __syncthreads();
    row_dif(x, N, pl, tc, tf);
    const float inv_n = (float)(1.0 / (double)N);
    for (int n = threadIdx.x; n < N; n += blockDim.x) H[(size_t)r * N + n] = cscale(x[pad16(n)], inv_n);
}

bool make_plan(int N, RowPlan *pl) {
    if (N < 2 || N > AF_MAX_N) return false;
    int n = N, np = 0;
    while (n % 16 == 0 && np < AF_MAXPASS) { pl->rad[np++] = 16; n /= 16; }
    for (int p : {8, 4, 2})
        while (n % p == 0 && np < AF_MAXPASS) { pl->rad[np++] = p; n /= p; }
    for (int p : {5, 3})
        while (n % p == 0 && np < AF_MAXPASS) { pl->rad[np++] = p; n /= p; }
    pl->npass = np;
    return n == 1;
}

int threads_for(int N) { return N <= 4096 ? 256 : N <= 8192 ? 512 : 1024; }

size_t smem_for(int N) { return sizeof(float2) * (size_t)(padded_len(N) + 64 + coarse_len(N)); }

constexpr size_t AF_SMEM_CAP = 200 * 1024;
bool stage_h_for(int N) { return smem_for(N) + sizeof(float2) * (size_t)padded_len(N) <= AF_SMEM_CAP; }
size_t fft_smem_for(int N) { return smem_for(N) + (stage_h_for(N) ? sizeof(float2) * (size_t)padded_len(N) : 0); }

template <typename F256, typename F512, typename F1024>
rosar_status launch_rows(int N, int rows, size_t sm, F256 f256, F512 f512, F1024 f1024, const void *k256,
                         const void *k512, const void *k1024, int (*done)[kMaxDevices], const char *what) {
    const int T = threads_for(N);
    const void *k = T <= 256 ? k256 : T <= 512 ? k512 : k1024;
    rosar_status st = ensure_smem(k, sm, done[T <= 256 ? 0 : T <= 512 ? 1 : 2], what);
    if (st != ROSAR_OK) return st;
    if (T <= 256) f256(rows, T, sm);
    else if (T <= 512) f512(rows, T, sm);
    else f1024(rows, T, sm);
    return check_launch(what);
}

}  // namespace

int azimuth_fft_supported(int n_az) {
    RowPlan pl;
    return make_plan(n_az, &pl) ? 1 : 0;
}

rosar_status launch_azimuth_fft(const float2 *S, const float2 *H, int n_rng, int n_az, float2 *out, cudaStream_t s) {
    RowPlan pl;
    if (!make_plan(n_az, &pl))
        return set_error(ROSAR_ERR_UNSUPPORTED, "azimuth_fft: n_az=%d is not 2^a 3^b 5^c in [2, %d]", n_az, AF_MAX_N);
    static int done[3][kMaxDevices] = {};
    const int sh = stage_h_for(n_az) ? 1 : 0;
    return launch_rows(
        n_az, n_rng, fft_smem_for(n_az),
        [&](int g, int t, size_t sm) { azimuth_fft_kernel<256><<<g, t, sm, s>>>(S, H, n_az, pl, sh, out); },
        [&](int g, int t, size_t sm) { azimuth_fft_kernel<512><<<g, t, sm, s>>>(S, H, n_az, pl, sh, out); },
        [&](int g, int t, size_t sm) { azimuth_fft_kernel<1024><<<g, t, sm, s>>>(S, H, n_az, pl, sh, out); },
        (const void *)azimuth_fft_kernel<256>, (const void *)azimuth_fft_kernel<512>,
        (const void *)azimuth_fft_kernel<1024>, done, "azimuth_fft");
}

rosar_status launch_azimuth_plan(const float2 *w, const int32_t *o, int o_row_stride, int n_rng, int n_az, int K,
                                 float2 *H, cudaStream_t s) {
    RowPlan pl;
    if (!make_plan(n_az, &pl))
        return set_error(ROSAR_ERR_UNSUPPORTED, "azimuth_plan: n_az=%d is not 2^a 3^b 5^c in [2, %d]", n_az, AF_MAX_N);
    static int done[3][kMaxDevices] = {};
    return launch_rows(
        n_az, n_rng, smem_for(n_az),
        [&](int g, int t, size_t sm) { azimuth_plan_kernel<256><<<g, t, sm, s>>>(w, o, o_row_stride, K, n_az, pl, H); },
        [&](int g, int t, size_t sm) { azimuth_plan_kernel<512><<<g, t, sm, s>>>(w, o, o_row_stride, K, n_az, pl, H); },
        [&](int g, int t, size_t sm) { azimuth_plan_kernel<1024><<<g, t, sm, s>>>(w, o, o_row_stride, K, n_az, pl, H); },
        (const void *)azimuth_plan_kernel<256>, (const void *)azimuth_plan_kernel<512>,
        (const void *)azimuth_plan_kernel<1024>, done, "azimuth_plan");
}

}  // namespace rosar
