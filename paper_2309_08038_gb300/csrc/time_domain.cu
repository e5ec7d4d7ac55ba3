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
// run on the tensor cores: 128 azimuth pixels x 64 rows per CTA, per stage (one tap, 16 samples) an A tile of
// raw samples and a B tile of coefficients in shared memory, tcgen05 MMAs into a tensor-memory accumulator.
// Three kernels share that tiling: td_tcg_kernel (the unplanned calls: B generated per stage, A from a window
// of raw pulses shared by the taps of a group), td_tcw_kernel (the planned calls: B precomputed once per weight
// design and bulk-copied) and td_tc_kernel (A and B both built per stage; taken when a CTA's taps exceed the
// others' sorted-tap list).  Per-row offsets (Algorithm 2 with a support per range bin) use a row kernel on the
// CUDA cores: one row per CTA, the row's phasors staged in shared memory by sample chunk, pulses read through
// L1/L2.
//
// 8 flops per (pixel, tap, sample).

#include <cooperative_groups.h>

#include <cmath>
#include <mutex>

#include <cuda_bf16.h>

#include "rosar_internal.cuh"

namespace cg = cooperative_groups;

namespace rosar {
namespace {

constexpr int TD_MC = 16;    // fast-time samples per stage
constexpr int TD_MAX_CLUSTER = 8;

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

// ------------------------------------------------------------------ tensor-core form (tcgen05) --
// The same implicit GEMM on the 5th-generation tensor cores.  A complex product a*b is the real product of
// [a.re a.im] (two K entries of A) with [[b.re, b.im], [-b.im, b.re]] (a 2 x 2 block of B: K = (sample, re/im),
// N = (row, re/im)), so D[theta][(row, re/im)] accumulates the complex sum in fp32 in tensor memory.  bf16
// operands hold 8 significant bits; each operand is split as x = hi + lo (bf16 each, x - hi exact to 2^-16 of
// x) and the product taken as hi*hi + hi*lo + lo*hi (three MMAs per K step), which keeps products within a few
// 10^-5 of fp32 (the dropped lo*lo term is 2^-16 smaller).  Per stage (one tap, 16 samples) the threads write
// the A tiles (128 pulses x 32 reals, split) and the B tiles (128 (row, re/im) x 32 reals: coefficient x window
// x fast-time phasor, split) into shared memory in the canonical no-swizzle K-major layout (8 x 16-byte core
// matrices; K-adjacent ones 128 B apart, 8-row groups 512 B apart), double-buffered; one thread issues the 2 K
// steps x 3 MMAs (M = 128, N = 128, K = 16) and commits them to the stage buffer's mbarrier, which the
// producers wait on before refilling that buffer.  Taps split across a cluster of CTAs whose partial tiles
// rank 0 adds in rank order.
namespace tcg {
constexpr int PRODUCERS = 256;               // warps 0-7 stage the operands and read the accumulator
constexpr int THREADS = PRODUCERS + 32;      // warp 8 issues the MMAs
constexpr int BT = 128;                      // azimuth pixels per CTA = MMA M
constexpr int BR = 64;                       // rows per CTA
constexpr int NN = 2 * BR;                   // MMA N
constexpr int MC = 16;                       // samples per stage
constexpr int KR = 2 * MC;                   // K entries (reals) per stage
constexpr int SBO = (KR / 8) * 128;          // byte stride of 8-row groups
constexpr int LBO = 128;                     // byte stride of K-adjacent core matrices
constexpr int TILE = BT * KR * 2;            // bytes of one operand tile (A: 128 x 32 bf16; B: NN = 128 rows)
constexpr int STAGE = 4 * TILE;              // A hi, A lo, B hi, B lo
constexpr int AFS = MC + 4;                  // fp32 A staging row stride (160 B: 16-byte lane accesses spread banks)
constexpr int AF = BT * AFS * 8;             // fp32 A staging of one stage (cp.async target): 20 KB
constexpr int SMEM = 2 * STAGE + 2 * AF + 6 * BR * 16 + 64;   // + [3][BR] tap table and [3][BR] phasor steps
constexpr int TMEM_COLS = 2 * NN;             // period accumulator X, running sum Y
constexpr int PERIOD = 128;                  // stages per period: 768 MMA steps accumulate in X before X is added into Y
constexpr long long SPIN_LIMIT = 1LL << 26;
static_assert(NN == BT, "one tile size serves both operands");

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int off(int row, int kk) {
    return (row >> 3) * SBO + (kk >> 3) * LBO + (row & 7) * 16 + (kk & 7) * 2;
}
__device__ __forceinline__ uint64_t desc(uint32_t a) {
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}
// D fp32, A and B bf16, both K-major, N = NN, M = BT
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(BT >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void ld16(uint32_t ta, float *v) {
    uint32_t rr[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
                   "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
                   "=r"(rr[15])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(rr[j]);
}
__device__ __forceinline__ void st16(uint32_t ta, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                   "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                   "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                   "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                   "r"(__float_as_uint(v[15]))
                 : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
// bounded wait for the completion of phase `parity` of an mbarrier; false after SPIN_LIMIT polls
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity) {
    for (long long it = 0; it < SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(saddr(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
// hi and lo bf16 pairs of (x, y): hi = RN(x, y), lo = RN(x - hi.x, y - hi.y)
__device__ __forceinline__ void split2(float x, float y, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}
}  // namespace tcg

// Warp-specialised pipeline: warps 0-7 (producers) wait until the MMAs of stage s-2 have released buffer s & 1
// (its `empty` mbarrier, armed by tcgen05.commit), fill it and arrive on its `full` mbarrier; warp 8 waits on
// `full`, issues the stage's MMAs and commits them to `empty`.  Producers meet at a named barrier once per tap,
// where two warps refresh the per-(row, tap) table two taps ahead.  At the end of each period of PERIOD stages the
// producers wait for the period's MMAs, fold X into Y and arrive on `fold`, which the issuer waits on before the
// next period's first MMA overwrites X.
template <bool BPA>
__global__ void __launch_bounds__(tcg::THREADS, 2)
td_tc_kernel(const float2 *__restrict__ X, const float *__restrict__ win, const float2 *__restrict__ w,
             const int32_t *__restrict__ o, TdParams p, int K, int k_per, float2 *__restrict__ out) {
    using namespace tcg;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *stage_base = smem;                                  // [2][A hi, A lo, B hi, B lo]
    float2 *af = reinterpret_cast<float2 *>(smem + 2 * STAGE);   // [2][BT][AFS] raw samples, one stage ahead
    float4 *tab = reinterpret_cast<float4 *>(smem + 2 * STAGE + 2 * AF);  // [3][BR]
    float4 *stp = tab + 3 * BR;              // [3][BR]: exp(-j pi phi), exp(-j pi 16 phi) of the same (row, tap)
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * STAGE + 2 * AF + 6 * BR * 16);
    uint64_t *full = bars, *empty = bars + 2, *fold_bar = bars + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 5);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool producer = warp < PRODUCERS / 32;
    const int th0 = blockIdx.x * BT, r0 = blockIdx.y * BR;
    const int n_az = p.n_az, L = p.L;
    const int chunks = L / MC;
    const int k_lo = blockIdx.z * k_per;
    const int nk = max(0, min(K, k_lo + k_per) - k_lo);
    const int stages = nk * chunks;
    const bool wide = n_az >= BT;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&full[i])), "r"(PRODUCERS / 32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&empty[i])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(fold_bar)), "r"(PRODUCERS / 32));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    auto tap_off = [&](int kk) -> int {
        const int k = k_lo + kk;
        return BPA ? k - K / 2 : pmod(__ldg(o + k), n_az);
    };
    auto build_tab = [&](int kk) {           // warps 0-1: one row per thread
        const int j = tid;
        const int r = r0 + j;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < p.n_rng) {
            t = tap_entry<BPA>(p, r, tap_off(kk));
            if (!BPA) {
                const float2 c = __ldg(w + (size_t)r * K + k_lo + kk);
                t.x = c.x;
                t.y = c.y;
            }
        }
        tab[(kk % 3) * BR + j] = t;
        // fast-time phasor steps of one and of MC samples, from the exactly reduced phase (zero rows: 1)
        const float4 u = make_float4(1.f, 0.f, t.z, t.w);
        const float2 s1 = phasor_term(u, 1.f, 1.f), s16 = phasor_term(u, 1.f, (float)MC);
        stp[(kk % 3) * BR + j] = make_float4(s1.x, s1.y, s16.x, s16.y);
    };
    if (warp < 2 && stages > 0) {
        build_tab(0);
        if (nk > 1) build_tab(1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int q = warp & 3, h = (warp >> 2) & 1;
    const uint32_t x_ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h);
    const uint32_t y_ta = x_ta + (uint32_t)NN;
    bool have_y = false;
    bool ok = true;

    if (producer) {
        // A copies of one stage: pair e = tid + PRODUCERS*it (it < 4) is row t = t_a + 32 it, samples m_a, m_a + 1,
        // with t_a = 8 (tid >> 6) + ((tid >> 1) & 7) and m_a = 4 ((tid >> 4) & 3) + 2 (tid & 1): the same samples and
        // 8-row group position for every it, so the staging and tile offsets advance by constants
        constexpr int A_IT = BT * MC / 2 / PRODUCERS;
        static_assert(A_IT == 4 && PRODUCERS == 256, "the closed form of the A pairs assumes 256 producers");
        const int m_a = ((tid >> 4) & 3) * 4 + (tid & 1) * 2;
        const int t_a = (tid >> 6) * 8 + ((tid >> 1) & 7);
        const int a_src = t_a * AFS + m_a;        // float2 offset in the fp32 staging of a stage, + 32 AFS per it
        const int a_dst = off(t_a, 2 * m_a);      // byte offset in the operand tiles, + 4 SBO per it
        // stage s2 = (tap kk2, samples m02 ..): the caller tracks both (no division per stage); the first pulse of
        // the tap's rows is recomputed only when the tap changes
        int base_kk = -1, base_row = 0;
        auto prefetch_A = [&](int s2, int kk2, int m02) {
            if (kk2 != base_kk) {
                base_kk = kk2;
                base_row = pmod(th0 + tap_off(kk2), n_az);
            }
            const int base2 = base_row;
            const uint32_t dst = saddr(af + (s2 & 1) * (BT * AFS) + a_src);
            const float2 *colp = X + m02 + m_a;
#pragma unroll
            for (int it = 0; it < A_IT; ++it) {
                int row = base2 + t_a + 32 * it;
                if (wide) row = row >= n_az ? row - n_az : row;
                else row %= n_az;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (uint32_t)(it * 32 * AFS * 8)),
                             "l"(colp + (size_t)row * L) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        auto fold = [&]() {                   // Y (+)= X, this warp's 32 lanes x 64 columns
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float xv[16], yv[16];
                ld16(x_ta + 16 * c, xv);
                if (have_y) {
                    ld16(y_ta + 16 * c, yv);
#pragma unroll
                    for (int j = 0; j < 16; ++j) xv[j] += yv[j];
                }
                st16(y_ta + 16 * c, xv);
            }
            have_y = true;
        };
        // B: this thread's (row, 4 samples) slot and its two 16-byte tile offsets, the same every stage
        const int b_r = 8 * warp + (lane & 7), b_c = lane >> 3;
        const bool b_swap = (b_r & 4) != 0;
        const int b_re = off(2 * b_r, 8 * b_c), b_im = off(2 * b_r + 1, 8 * b_c);
        const int b_first = b_swap ? b_im : b_re, b_second = b_swap ? b_re : b_im;
        if (stages > 0) prefetch_A(0, 0, 0);
        float2 e_run = make_float2(1.f, 0.f);  // fast-time phasor at this thread's first sample of the stage
        int kk = 0, m0 = 0, slot = 0;          // tap, first sample of stage s, and the tap's table slot (kk mod 3)
        for (int s = 0; s < stages; ++s, m0 += MC) {
            if (m0 == L) {
                m0 = 0;
                ++kk;
                slot = slot == 2 ? 0 : slot + 1;
            }
            const int b = s & 1;
            uint8_t *st = stage_base + b * STAGE;
            // a wait that gives up clears ok and every later wait is skipped, but every thread still runs the loop
            // to its end, so the named barriers stay matched (the tile then reads NaN)
            if (s >= 2 && ok) ok = wait_bar(&empty[b], (uint32_t)(((s - 2) >> 1) & 1));
            if (m0 == 0) {                     // tap boundary: the table of tap kk-1 is no longer read
                asm volatile("bar.sync 1, %0;" ::"n"(PRODUCERS) : "memory");
                if (warp < 2 && kk + 2 < nk) build_tab(kk + 2);
            }
            if (s + 1 < stages) {
                prefetch_A(s + 1, m0 + MC == L ? kk + 1 : kk, m0 + MC == L ? 0 : m0 + MC);
                asm volatile("cp.async.wait_group 1;" ::: "memory");       // this thread's copies of stage s
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            // A: the thread's own 4 pairs of samples, split into the hi and lo tiles
            const float2 *src = af + b * (BT * AFS) + a_src;
#pragma unroll
            for (int it = 0; it < A_IT; ++it) {
                const float4 a = *reinterpret_cast<const float4 *>(src + it * 32 * AFS);
                uint2 hi, lo;
                split2(a.x, a.y, hi.x, lo.x);
                split2(a.z, a.w, hi.y, lo.y);
                *reinterpret_cast<uint2 *>(st + a_dst + it * 4 * SBO) = hi;
                *reinterpret_cast<uint2 *>(st + TILE + a_dst + it * 4 * SBO) = lo;
            }
            // B: thread = (row r = 8 warp + (lane & 7), samples 4 (lane >> 3) ..): coefficient x window x phasor by a
            // recurrence over the 4 samples, rows (r, re) = [b.re, -b.im] and (r, im) = [b.im, b.re]; lanes with r & 4
            // write the im row first, so each 8-lane phase of a 16-byte store hits 8 distinct rows
            {
                const int r = b_r;
                const float4 t4 = tab[slot * BR + r];
                const float4 st4 = stp[slot * BR + r];
                const int mb = m0 + 4 * b_c;
                // the thread keeps the same (row, 4 samples) slot every stage: the phasor at its first sample is
                // taken exactly at the tap's first stage and advanced by MC samples per stage after that
                e_run = m0 == 0 ? phasor_term(make_float4(1.f, 0.f, t4.z, t4.w), 1.f, (float)mb - p.m_ref)
                                : cmul(e_run, make_float2(st4.z, st4.w));
                const float2 step = make_float2(st4.x, st4.y);               // exp(-j pi phi), one sample
                float2 e = e_run;
                uint32_t re_hi[4], re_lo[4], im_hi[4], im_lo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float wm = win ? __ldg(win + mb + i) : 1.f;
                    const float2 v = cmul(make_float2(t4.x * wm, t4.y * wm), e);
                    // one split of (v.re, v.im); rounding is symmetric and per component, so the row (re) =
                    // (v.re, -v.im) is the same pairs with the high half's sign flipped and the row (im) =
                    // (v.im, v.re) the same pairs with the halves swapped
                    uint32_t hi, lo;
                    split2(v.x, v.y, hi, lo);
                    re_hi[i] = hi ^ 0x80000000u;
                    re_lo[i] = lo ^ 0x80000000u;
                    im_hi[i] = __byte_perm(hi, 0, 0x1032);
                    im_lo[i] = __byte_perm(lo, 0, 0x1032);
                    e = cmul(e, step);
                }
                const uint4 rh = make_uint4(re_hi[0], re_hi[1], re_hi[2], re_hi[3]);
                const uint4 rl = make_uint4(re_lo[0], re_lo[1], re_lo[2], re_lo[3]);
                const uint4 ih = make_uint4(im_hi[0], im_hi[1], im_hi[2], im_hi[3]);
                const uint4 il = make_uint4(im_lo[0], im_lo[1], im_lo[2], im_lo[3]);
                *reinterpret_cast<uint4 *>(st + 2 * TILE + b_first) = b_swap ? ih : rh;
                *reinterpret_cast<uint4 *>(st + 3 * TILE + b_first) = b_swap ? il : rl;
                *reinterpret_cast<uint4 *>(st + 2 * TILE + b_second) = b_swap ? rh : ih;
                *reinterpret_cast<uint4 *>(st + 3 * TILE + b_second) = b_swap ? rl : il;
            }
            // every thread makes its tile stores visible to the tensor core's (async) proxy; the warp then arrives
            // once (one arrival per warp: 256 arrivals on one word would serialise in shared memory)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&full[b])) : "memory");
            if ((s + 1) % PERIOD == 0 && s + 1 < stages) {   // end of a period: its MMAs done, fold X into Y
                if (ok) ok = wait_bar(&empty[b], (uint32_t)((s >> 1) & 1));
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (ok) fold();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(fold_bar)) : "memory");
            }
        }
        if (ok && stages > 0) ok = wait_bar(&empty[(stages - 1) & 1], (uint32_t)(((stages - 1) >> 1) & 1));
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (lane == 0) {                   // the MMA issuer
        for (int s = 0; s < stages; ++s) {
            const int b = s & 1;
            if (ok) ok = wait_bar(&full[b], (uint32_t)((s >> 1) & 1));
            if (ok && s % PERIOD == 0 && s > 0) ok = wait_bar(fold_bar, (uint32_t)((s / PERIOD - 1) & 1));
            if (!ok) break;                       // the issuer meets no named barrier; producers time out on empty
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = saddr(stage_base + b * STAGE), a_lo = a_hi + TILE, b_hi = a_hi + 2 * TILE,
                           b_lo = a_hi + 3 * TILE;
#pragma unroll
            for (int ks = 0; ks < KR / 16; ++ks) {
                const uint32_t ko = ks * 2 * LBO;                     // 16 K entries = two core-matrix columns
                mma(tmem, desc(a_hi + ko), desc(b_hi + ko), (s % PERIOD != 0 || ks > 0) ? 1u : 0u);
                mma(tmem, desc(a_hi + ko), desc(b_lo + ko), 1u);
                mma(tmem, desc(a_lo + ko), desc(b_hi + ko), 1u);
            }
            commit(&empty[b]);
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // accumulator -> registers (producer warps): warp w reads TMEM lanes 32 (w % 4).. and columns 64 ((w / 4) % 2)..
    const int th = 32 * q + lane;
    float v[64];
    if (producer) {
        if (ok && stages > 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                ld16(x_ta + 16 * c, v + 16 * c);
                if (have_y) {
                    float yv[16];
                    ld16(y_ta + 16 * c, yv);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[16 * c + j] += yv[j];
                }
            }
        } else {
            const float f = ok ? 0.f : __int_as_float(0x7fc00000);   // no taps: zero; a wait that gave up: NaN
#pragma unroll
            for (int j = 0; j < 64; ++j) v[j] = f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));

    const int G = gridDim.z;
    bool writer = producer;
    if (G > 1) {                              // partial tiles parked in the stage buffers, rank 0 adds in rank order
        float *red = reinterpret_cast<float *>(smem);            // [128 columns][128 pixels] = 64 KB
        cg::cluster_group cluster = cg::this_cluster();
        if (producer) {
#pragma unroll
            for (int j = 0; j < 64; ++j) red[(64 * h + j) * BT + th] = v[j];
        }
        cluster.sync();
        if (producer && cluster.block_rank() == 0) {
            for (int rk = 1; rk < G; ++rk) {
                const float *rem = cluster.map_shared_rank(red, rk);
#pragma unroll
                for (int j = 0; j < 64; ++j) v[j] += rem[(64 * h + j) * BT + th];
            }
        }
        cluster.sync();
        writer = producer && cluster.block_rank() == 0;
    }
    const int tcol = th0 + th;
    if (writer && tcol < n_az) {
#pragma unroll
        for (int j = 0; j < 64; j += 2) {
            const int r = r0 + (64 * h + j) / 2;
            if (r < p.n_rng) out[(size_t)r * n_az + tcol] = make_float2(v[j], v[j + 1]);
        }
    }
}

// ------------------------------------------------------------ planned tensor-core form (sliding A window) --
// With the B operand prepared once per weight design the A operand becomes the only per-scan input, and it is
// shared between taps: the A tile of tap k is the raw pulses th0 + o_k + t (t < 128), so taps whose offsets lie
// within a span d of each other read rows of ONE window of 128 + d pulses.  In the no-swizzle K-major layout with
// 8-row groups 128 B apart (rows 16 B apart throughout), the tile of tap k is that window from row o_k - o_first:
// a start address 16 (o_k - o_first) bytes further on, same descriptor otherwise.  The loop runs sample chunks
// outermost and the taps (sorted by offset, cut into segments whose span fits the window) inside: per chunk and
// segment the producer warps stage one window (raw fp32 split into bf16 hi and lo), and per (chunk, tap) one thread
// copies the planned B block (16 KB: hi tile then lo tile, canonical layout) with one bulk copy completing on the
// stage's mbarrier.  A costs 128 + d rows per chunk and segment instead of 128 per chunk and tap.
namespace tcw {
using namespace tcg;
constexpr int NS = 3;                              // B stage buffers
constexpr int WMAX = 248;                          // window rows: 128 pixels + the segment's offset span
constexpr int SPAN = WMAX - BT;                    // largest offset span of one segment
constexpr int ALBO = WMAX * 16 + 32;               // K-adjacent core matrices of the window (+32 B: a half-warp's
                                                   // 8-byte window stores, 2 rows x 4 groups, cover 32 banks once)
constexpr int ASBO = 128;                          // 8-row groups of the window
constexpr int APLANE = 4 * ALBO;                   // hi plane, then lo plane
constexpr int WSLOT = 2 * APLANE;
constexpr int BTILE = 2 * TILE;                    // planned B block (hi, lo)
constexpr int WROUNDS = (WMAX + PRODUCERS / 8 - 1) / (PRODUCERS / 8);   // window rows per producer thread
constexpr int THREADS = PRODUCERS + 64;            // warps 0-7 windows / fold / epilogue, 8 MMA issuer, 9 B copies
constexpr int SMEM = NS * BTILE + 2 * WSLOT + 128; // + mbarriers and the TMEM slot
static_assert((2 * NS + 6) * 8 + 4 <= 128, "barriers and the TMEM slot fit their area");
static_assert(SMEM <= 232448 / 2 - 1024, "two CTAs per SM");
static_assert(BT * NN * 4 <= NS * BTILE + 2 * WSLOT, "the cluster reduction parks a tile in the stage buffers");

__device__ __forceinline__ uint64_t descA(uint32_t a) {
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)(ALBO >> 4) << 16) | ((uint64_t)(ASBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}
}  // namespace tcw

template <bool BPA>
__global__ void __launch_bounds__(tcw::THREADS, 2)
td_tcw_kernel(const float2 *__restrict__ X, const uint8_t *__restrict__ Bt, const int32_t *__restrict__ offs,
              TdParams p, int K, int k_per, float2 *__restrict__ out) {
    using namespace tcw;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *bstage = smem;                                      // [NS][B hi, B lo]
    uint8_t *wbase = smem + NS * BTILE;                          // [2][hi, lo][4 groups][ALBO]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * BTILE + 2 * WSLOT);
    uint64_t *full = bars, *empty = bars + NS, *wfull = bars + 2 * NS, *wempty = bars + 2 * NS + 2,
             *fold_bar = bars + 2 * NS + 4, *acc_bar = bars + 2 * NS + 5;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 6);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool producer = warp < PRODUCERS / 32;
    const int th0 = blockIdx.x * BT, rb = blockIdx.y, r0 = rb * BR;
    const int n_az = p.n_az, L = p.L;
    const int chunks = L / MC;
    const int k_lo = blockIdx.z * k_per;
    const int k_end = min(K, k_lo + k_per);
    const int nk = max(0, k_end - k_lo);
    const int stages = nk * chunks;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&full[i])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&empty[i])), "r"(1));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&wfull[i])), "r"(PRODUCERS / 32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&wempty[i])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(fold_bar)), "r"(PRODUCERS / 32));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(acc_bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int q = warp & 3, h = (warp >> 2) & 1;
    const uint32_t x_ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h);
    // The producer warps do not follow every stage, so they learn that a period's MMAs are done from acc_bar (one
    // phase per period end and one at the last stage, each waited for in order); a parity wait on a stage's
    // `empty` barrier could match a later phase.
    const uint32_t y_ta = x_ta + (uint32_t)NN;
    bool have_y = false;
    bool ok = true;

    // segment of taps starting at ka: the longest run of (sorted) taps within SPAN of offs[ka]
    auto seg_end = [&](int ka) {
        const long long base = __ldg(offs + ka);
        int kb = ka + 1;
        while (kb < k_end && (long long)__ldg(offs + kb) - base <= SPAN) ++kb;
        return kb;
    };

    if (producer) {
        // window stores: thread = (sample pair a_j of the chunk, rows a_r + 32 i); a warp stores 4 rows x 8 pairs
        const int a_j = tid & 7, a_r = tid >> 3;
        const int a_dst = (a_j >> 1) * ALBO + (a_j & 1) * 8;
        auto produce = [&](int w, int c, int ka, int kb) {
            const int slot = w & 1;
            if (w >= 2 && ok) ok = wait_bar(&wempty[slot], (uint32_t)(((w >> 1) - 1) & 1));
            const int W = (int)((long long)__ldg(offs + kb - 1) - __ldg(offs + ka)) + BT;
            const int p0 = pmod(th0 + pmod(__ldg(offs + ka), n_az), n_az);
            uint8_t *ws = wbase + slot * WSLOT + a_dst;
            const float2 *col = X + c * MC + 2 * a_j;
            // all of this thread's rows (at most WROUNDS) loaded before any is converted: one memory round trip
            float4 v[WROUNDS];
#pragma unroll
            for (int j = 0; j < WROUNDS; ++j) {
                const int i = a_r + j * (PRODUCERS / 8);
                v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < W) {
                    int pulse = p0 + i;
                    if (pulse >= n_az) pulse %= n_az;
                    v[j] = __ldg(reinterpret_cast<const float4 *>(col + (size_t)pulse * L));
                }
            }
#pragma unroll
            for (int j = 0; j < WROUNDS; ++j) {
                const int i = a_r + j * (PRODUCERS / 8);
                if (i < W) {
                    uint2 hi, lo;
                    split2(v[j].x, v[j].y, hi.x, lo.x);
                    split2(v[j].z, v[j].w, hi.y, lo.y);
                    *reinterpret_cast<uint2 *>(ws + 16 * i) = hi;
                    *reinterpret_cast<uint2 *>(ws + APLANE + 16 * i) = lo;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&wfull[slot])) : "memory");
        };
        auto fold = [&]() {                   // Y (+)= X, this warp's 32 lanes x 64 columns
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float xv[16], yv[16];
                ld16(x_ta + 16 * c, xv);
                if (have_y) {
                    ld16(y_ta + 16 * c, yv);
#pragma unroll
                    for (int j = 0; j < 16; ++j) xv[j] += yv[j];
                }
                st16(y_ta + 16 * c, xv);
            }
            have_y = true;
        };
        if (stages > 0) {
            // windows are staged one ahead: window w + 1 is written (after window w - 1's MMAs released its slot)
            // before the folds that fall inside window w's stages
            int c_cur = 0, ka_cur = k_lo, kb_cur = seg_end(k_lo);
            produce(0, 0, ka_cur, kb_cur);
            int s = 0;
            for (int w = 0;; ++w) {
                int c_n = c_cur, ka_n = kb_cur, kb_n = 0;
                if (ka_n == k_end) {
                    ka_n = k_lo;
                    ++c_n;
                }
                if (c_n < chunks) {
                    kb_n = seg_end(ka_n);
                    produce(w + 1, c_n, ka_n, kb_n);
                }
                const int s_end = s + (kb_cur - ka_cur);
                // period ends inside this window: s + 1 a multiple of PERIOD, not the last stage
                for (int se = ((s + PERIOD) / PERIOD) * PERIOD - 1; se < s_end && se + 1 < stages; se += PERIOD) {
                    if (ok) ok = wait_bar(acc_bar, (uint32_t)((se / PERIOD) & 1));
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (ok) fold();
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(fold_bar)) : "memory");
                }
                s = s_end;
                if (c_n >= chunks) break;
                c_cur = c_n;
                ka_cur = ka_n;
                kb_cur = kb_n;
            }
            if (ok) ok = wait_bar(acc_bar, (uint32_t)(((stages - 1) / PERIOD) & 1));
        }
    } else if (warp == PRODUCERS / 32) {
        if (lane == 0) {                      // the MMA issuer
            int s = 0, w = 0;
            for (int c = 0; c < chunks && ok; ++c) {
                for (int ka = k_lo; ka < k_end && ok;) {
                    const int kb = seg_end(ka);
                    const int slot = w & 1;
                    ok = wait_bar(&wfull[slot], (uint32_t)((w >> 1) & 1));
                    if (!ok) break;
                    const long long base = __ldg(offs + ka);
                    const uint32_t wa = saddr(wbase + slot * WSLOT);
                    for (int k = ka; k < kb; ++k, ++s) {
                        const int b = s % NS;
                        ok = wait_bar(&full[b], (uint32_t)((s / NS) & 1));
                        if (ok && s % PERIOD == 0 && s > 0) ok = wait_bar(fold_bar, (uint32_t)((s / PERIOD - 1) & 1));
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a_hi = wa + (uint32_t)(((long long)__ldg(offs + k) - base) * 16),
                                       a_lo = a_hi + APLANE;
                        const uint32_t b_hi = saddr(bstage + b * BTILE), b_lo = b_hi + TILE;
#pragma unroll
                        for (int ks = 0; ks < KR / 16; ++ks) {
                            const uint32_t ka2 = ks * 2 * ALBO, kb2 = ks * 2 * LBO;
                            mma(tmem, descA(a_hi + ka2), desc(b_hi + kb2), (s % PERIOD != 0 || ks > 0) ? 1u : 0u);
                            mma(tmem, descA(a_hi + ka2), desc(b_lo + kb2), 1u);
                            mma(tmem, descA(a_lo + ka2), desc(b_hi + kb2), 1u);
                        }
                        commit(&empty[b]);
                        if ((s + 1) % PERIOD == 0 || s + 1 == stages) commit(acc_bar);
                    }
                    if (!ok) break;
                    if (c + 1 < chunks || kb < k_end) commit(&wempty[slot]);   // (the last window's slot is not reused)
                    ++w;
                    ka = kb;
                }
            }
        }
    } else if (lane == 0) {                   // the B copies: stage s = (chunk, tap) in the issuer's order
        int s = 0;
        for (int c = 0; c < chunks && ok; ++c) {
            for (int k = k_lo; k < k_end; ++k, ++s) {
                const int b = s % NS;
                if (s >= NS) ok = wait_bar(&empty[b], (uint32_t)(((s / NS) - 1) & 1));
                if (!ok) break;
                const uint8_t *src = Bt + (((size_t)rb * K + k) * chunks + c) * BTILE;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&full[b])),
                             "r"(BTILE) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(saddr(bstage + b * BTILE)), "l"(src), "r"(BTILE), "r"(saddr(&full[b])) : "memory");
            }
        }
        // the copies of the last (up to NS) issued stages may still be in flight if a wait gave up: their
        // completion is the only arrival their phase needs (bounded waits)
        for (int s2 = max(0, s - NS); s2 < s; ++s2) wait_bar(&full[s2 % NS], (uint32_t)((s2 / NS) & 1));
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const int th = 32 * q + lane;
    float v[64];
    if (producer) {
        if (ok && stages > 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                ld16(x_ta + 16 * c, v + 16 * c);
                if (have_y) {
                    float yv[16];
                    ld16(y_ta + 16 * c, yv);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[16 * c + j] += yv[j];
                }
            }
        } else {
            const float f = ok ? 0.f : __int_as_float(0x7fc00000);   // no taps: zero; a wait that gave up: NaN
#pragma unroll
            for (int j = 0; j < 64; ++j) v[j] = f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));

    const int G = gridDim.z;
    bool writer = producer;
    if (G > 1) {                              // partial tiles parked in the stage buffers, rank 0 adds in rank order
        float *red = reinterpret_cast<float *>(smem);            // [128 columns][128 pixels] = 64 KB
        cg::cluster_group cluster = cg::this_cluster();
        if (producer) {
#pragma unroll
            for (int j = 0; j < 64; ++j) red[(64 * h + j) * BT + th] = v[j];
        }
        cluster.sync();
        if (producer && cluster.block_rank() == 0) {
            for (int rk = 1; rk < G; ++rk) {
                const float *rem = cluster.map_shared_rank(red, rk);
#pragma unroll
                for (int j = 0; j < 64; ++j) v[j] += rem[(64 * h + j) * BT + th];
            }
        }
        cluster.sync();
        writer = producer && cluster.block_rank() == 0;
    }
    const int tcol = th0 + th;
    if (writer && tcol < n_az) {
#pragma unroll
        for (int j = 0; j < 64; j += 2) {
            const int r = r0 + (64 * h + j) / 2;
            if (r < p.n_rng) out[(size_t)r * n_az + tcol] = make_float2(v[j], v[j + 1]);
        }
    }
}

// ------------------------------------------------------------ generated-B tensor-core form (sliding A window) --
// td_tcw_kernel's pipeline without a plan: the producer warps generate each stage's B tile (coefficient x fast-
// time phasor of 64 rows x 16 samples: the phase in half-turns reduced exactly by whole turns, then the hardware
// sine and cosine) into a 3-deep ring, and stage the raw-pulse windows as in td_tcw_kernel with the fast-time
// window applied to A as it is staged (it depends on the sample only).  A tenth warp sorts the CTA's taps by
// offset once and fills, two tap groups ahead, the per-(row, tap) table (coefficient, two-way phase, fast-time
// phase in FP64 -> float hi/lo) that the B tiles are made from.  Taps run in groups of at most TG sorted taps within SPAN pulses; stage order = group, chunk,
// tap.  The window of group g and chunk c + 1 is staged after the producers have generated the first NS stages
// of chunk c (by then the MMAs of the window before have finished, so its slot is free).
namespace tcgn {
using namespace tcg;
constexpr int NS = 3;                              // B stage buffers
constexpr int TG = 8;                              // taps per group (table entries per row)
constexpr int WMAX = 176;                          // window rows
constexpr int SPAN = WMAX - BT;
constexpr int ALBO = WMAX * 16 + 32;               // as td_tcw_kernel (+32 B: conflict-free window stores)
constexpr int ASBO = 128;
constexpr int APLANE = 4 * ALBO;
constexpr int WSLOT = 2 * APLANE;
constexpr int WROUNDS = (WMAX + PRODUCERS / 8 - 1) / (PRODUCERS / 8);
constexpr int BSTAGE = 2 * TILE;                   // B hi, B lo
constexpr int TAPS_MAX = 512;                      // taps per CTA (the sorted list in shared memory)
constexpr int TABLE = TG * BR * 16;                // one table slot: [TG][64 rows] float4
constexpr int OFF_WIN = NS * BSTAGE;
constexpr int OFF_TAB = OFF_WIN + 2 * WSLOT;
constexpr int OFF_SORT = OFF_TAB + 2 * TABLE;
constexpr int OFF_BAR = OFF_SORT + 2 * TAPS_MAX * 4;
constexpr int N_BARS = 2 * NS + 2 * 4 + 2;         // full, empty, wfull, wempty, tfull, tempty, fold, acc
constexpr int SMEM = OFF_BAR + 256;                // the barriers, then the TMEM address slot
static_assert(N_BARS * 8 + 4 <= 256, "barriers and the TMEM slot fit their area");
constexpr int THREADS = PRODUCERS + 64;            // warps 0-7 producers, 8 MMA issuer, 9 sort and tables
static_assert(SMEM <= 233472 / 2 - 1024, "two CTAs per SM");
static_assert(BT * NN * 4 <= OFF_TAB, "the cluster reduction parks a tile in the stage and window buffers");
__device__ __forceinline__ uint64_t descA(uint32_t a) {
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)(ALBO >> 4) << 16) | ((uint64_t)(ASBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}
}  // namespace tcgn

// exp(-j*pi*phi*x) for phi = hi + lo, reduced as in phasor_term, with the hardware sine and cosine of the reduced
// argument (|arg| <= about 1 half-turn; absolute error about 1e-6, below the bf16 split's 2^-16 relative)
__device__ __forceinline__ float2 phasor_unit_fast(float hi, float lo, float x) {
    const float prod = hi * x;
    const float err = fmaf(hi, x, -prod);
    const float red = prod - 2.f * rintf(0.5f * prod);
    const float arg = red + fmaf(lo, x, err);
    float sn, cs;
    __sincosf(3.14159265358979f * arg, &sn, &cs);
    return make_float2(cs, -sn);
}

template <bool BPA>
__global__ void __launch_bounds__(tcgn::THREADS, 2)
td_tcg_kernel(const float2 *__restrict__ X, const float *__restrict__ win, const float2 *__restrict__ w,
              const int32_t *__restrict__ o, TdParams p, int K, int k_per, float2 *__restrict__ out) {
    using namespace tcgn;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *bstage = smem;                                          // [NS][B hi, B lo]
    uint8_t *wbase = smem + OFF_WIN;                                 // [2][hi, lo][4 groups][ALBO]
    float4 *tab = reinterpret_cast<float4 *>(smem + OFF_TAB);        // [2][TG][BR]
    int *soff = reinterpret_cast<int *>(smem + OFF_SORT);            // sorted offsets of this CTA's taps
    int *stap = soff + TAPS_MAX;                                     // and their taps
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
    uint64_t *full = bars, *empty = bars + NS, *wfull = bars + 2 * NS, *wempty = wfull + 2, *tfull = wempty + 2,
             *tempty = tfull + 2, *fold_bar = tempty + 2, *acc_bar = fold_bar + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_bar + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool producer = warp < PRODUCERS / 32;
    const int th0 = blockIdx.x * BT, r0 = blockIdx.y * BR;
    const int n_az = p.n_az, L = p.L;
    const int chunks = L / MC;
    const int k_lo = blockIdx.z * k_per;
    const int nk = max(0, min(K, k_lo + k_per) - k_lo);
    const int stages = nk * chunks;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&full[i])), "r"(PRODUCERS / 32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&empty[i])), "r"(1));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&wfull[i])), "r"(PRODUCERS / 32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&wempty[i])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&tfull[i])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&tempty[i])), "r"(PRODUCERS / 32));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(fold_bar)), "r"(PRODUCERS / 32));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(acc_bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == PRODUCERS / 32 + 1) {         // the CTA's taps in ascending offset order (ties by tap)
        for (int i = lane; i < nk; i += 32) {
            const int k = k_lo + i;
            const int v = BPA ? k - K / 2 : __ldg(o + k);
            int rank = i;
            if (!BPA) {
                rank = 0;
                for (int j = 0; j < nk; ++j) {
                    const int u = __ldg(o + k_lo + j);
                    rank += (u < v) || (u == v && j < i);
                }
            }
            soff[rank] = v;
            stap[rank] = k;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int q = warp & 3, h = (warp >> 2) & 1;
    const uint32_t x_ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h);
    const uint32_t y_ta = x_ta + (uint32_t)NN;
    bool have_y = false;
    bool ok = true;

    // group of sorted taps starting at ga: at most TG taps within SPAN of soff[ga]
    auto group_end = [&](int ga) {
        const long long base = soff[ga];
        int gb = ga + 1;
        while (gb < nk && gb - ga < TG && (long long)soff[gb] - base <= SPAN) ++gb;
        return gb;
    };

    if (producer) {
        const int a_j = tid & 7, a_r = tid >> 3;
        const int a_dst = (a_j >> 1) * ALBO + (a_j & 1) * 8;
        auto produce = [&](int wi, int c, int ga, int gb) {           // window wi = (group [ga, gb), chunk c)
            const int slot = wi & 1;
            if (wi >= 2 && ok) ok = wait_bar(&wempty[slot], (uint32_t)(((wi >> 1) - 1) & 1));
            const int W = (int)((long long)soff[gb - 1] - soff[ga]) + BT;
            const int p0 = pmod(th0 + pmod(soff[ga], n_az), n_az);
            uint8_t *ws = wbase + slot * WSLOT + a_dst;
            const float2 *col = X + c * MC + 2 * a_j;
            // the fast-time window multiplies A here, once per staged sample, instead of every B entry
            const float w0 = win ? __ldg(win + c * MC + 2 * a_j) : 1.f;
            const float w1 = win ? __ldg(win + c * MC + 2 * a_j + 1) : 1.f;
            float4 v[WROUNDS];
#pragma unroll
            for (int j = 0; j < WROUNDS; ++j) {
                const int i = a_r + j * (PRODUCERS / 8);
                v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < W) {
                    int pulse = p0 + i;
                    if (pulse >= n_az) pulse %= n_az;
                    v[j] = __ldg(reinterpret_cast<const float4 *>(col + (size_t)pulse * L));
                }
            }
#pragma unroll
            for (int j = 0; j < WROUNDS; ++j) {
                const int i = a_r + j * (PRODUCERS / 8);
                if (i < W) {
                    uint2 hi, lo;
                    split2(v[j].x * w0, v[j].y * w0, hi.x, lo.x);
                    split2(v[j].z * w1, v[j].w * w1, hi.y, lo.y);
                    *reinterpret_cast<uint2 *>(ws + 16 * i) = hi;
                    *reinterpret_cast<uint2 *>(ws + APLANE + 16 * i) = lo;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&wfull[slot])) : "memory");
        };
        auto fold = [&]() {
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float xv[16], yv[16];
                ld16(x_ta + 16 * c, xv);
                if (have_y) {
                    ld16(y_ta + 16 * c, yv);
#pragma unroll
                    for (int j = 0; j < 16; ++j) xv[j] += yv[j];
                }
                st16(y_ta + 16 * c, xv);
            }
            have_y = true;
        };
        // B: thread = (row b_r = 8 warp + (lane & 7), samples 4 (lane >> 3) ..); lanes with b_r & 4 write the im
        // row first, so each 8-lane phase of a 16-byte store hits 8 distinct rows
        const int b_r = 8 * warp + (lane & 7), b_c = lane >> 3;
        const bool b_swap = (b_r & 4) != 0;
        const int b_re = off(2 * b_r, 8 * b_c), b_im = off(2 * b_r + 1, 8 * b_c);
        const int b_first = b_swap ? b_im : b_re, b_second = b_swap ? b_re : b_im;
        const uint32_t sel_first = b_swap ? 0x1032u : 0x7654u, sel_second = b_swap ? 0x7654u : 0x1032u;
        if (stages > 0) {
            int s = 0, wi = 0, g = 0;
            int ga = 0, gb = group_end(0);
            produce(0, 0, ga, gb);
            for (; ga < nk; ga = gb, gb = gb < nk ? group_end(gb) : gb, ++g) {
                const int tslot = g & 1;
                if (ok) ok = wait_bar(&tfull[tslot], (uint32_t)((g >> 1) & 1));
                const float4 *tg = tab + tslot * (TG * BR);
                for (int c = 0; c < chunks; ++c, ++wi) {
                    const int n_w = gb - ga;
                    const int j_next = min(NS, n_w) - 1;                 // stage after which window wi + 1 is staged
                    for (int kk = 0; kk < n_w; ++kk, ++s) {
                        const int b = s % NS;
                        if (s >= NS && ok) ok = wait_bar(&empty[b], (uint32_t)(((s / NS) - 1) & 1));
                        uint8_t *st = bstage + b * BSTAGE;
                        const float4 t4 = tg[kk * BR + b_r];
                        const int mb = c * MC + 4 * b_c;
                        // coefficient x phasor at the thread's first sample (phasor taken directly), the next three
                        // by the one-sample step (three products: about 3e-7 more error)
                        float2 v = cmul(make_float2(t4.x, t4.y), phasor_unit_fast(t4.z, t4.w, (float)mb - p.m_ref));
                        const float2 step = phasor_unit_fast(t4.z, t4.w, 1.f);
                        uint32_t f_hi[4], f_lo[4], s_hi[4], s_lo[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if (i > 0) v = cmul(v, step);
                            uint32_t hi, lo;
                            split2(v.x, v.y, hi, lo);
                            // row (re) = the pair with the high half's sign flipped (bytes 4-7 of the selector
                            // pair), row (im) = the pair with its halves swapped (bytes 2, 3, 0, 1): the first
                            // store of a lane takes the im row where b_swap
                            const uint32_t hs = hi ^ 0x80000000u, ls = lo ^ 0x80000000u;
                            f_hi[i] = __byte_perm(hi, hs, sel_first);
                            f_lo[i] = __byte_perm(lo, ls, sel_first);
                            s_hi[i] = __byte_perm(hi, hs, sel_second);
                            s_lo[i] = __byte_perm(lo, ls, sel_second);
                        }
                        *reinterpret_cast<uint4 *>(st + b_first) = make_uint4(f_hi[0], f_hi[1], f_hi[2], f_hi[3]);
                        *reinterpret_cast<uint4 *>(st + TILE + b_first) = make_uint4(f_lo[0], f_lo[1], f_lo[2], f_lo[3]);
                        *reinterpret_cast<uint4 *>(st + b_second) = make_uint4(s_hi[0], s_hi[1], s_hi[2], s_hi[3]);
                        *reinterpret_cast<uint4 *>(st + TILE + b_second) = make_uint4(s_lo[0], s_lo[1], s_lo[2], s_lo[3]);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&full[b])) : "memory");
                        if (kk == j_next) {                                // stage the next window
                            if (c + 1 < chunks) produce(wi + 1, c + 1, ga, gb);
                            else if (gb < nk) produce(wi + 1, 0, gb, group_end(gb));
                        }
                        if ((s + 1) % PERIOD == 0 && s + 1 < stages) {     // period end: fold X into Y
                            if (ok) ok = wait_bar(acc_bar, (uint32_t)((s / PERIOD) & 1));
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            if (ok) fold();
                            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                            __syncwarp();
                            if (lane == 0)
                                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(fold_bar)) : "memory");
                        }
                    }
                }
                __syncwarp();                                              // the group's table is no longer read
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&tempty[tslot])) : "memory");
            }
            if (ok) ok = wait_bar(acc_bar, (uint32_t)(((stages - 1) / PERIOD) & 1));
        }
    } else if (warp == PRODUCERS / 32) {
        if (lane == 0) {                      // the MMA issuer
            int s = 0, wi = 0;
            for (int ga = 0, gb = 0; ga < nk && ok; ga = gb) {
                gb = group_end(ga);
                for (int c = 0; c < chunks && ok; ++c, ++wi) {
                    const int slot = wi & 1;
                    ok = wait_bar(&wfull[slot], (uint32_t)((wi >> 1) & 1));
                    if (!ok) break;
                    const long long base = soff[ga];
                    const uint32_t wa = saddr(wbase + slot * WSLOT);
                    for (int k = ga; k < gb; ++k, ++s) {
                        const int b = s % NS;
                        ok = wait_bar(&full[b], (uint32_t)((s / NS) & 1));
                        if (ok && s % PERIOD == 0 && s > 0) ok = wait_bar(fold_bar, (uint32_t)((s / PERIOD - 1) & 1));
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a_hi = wa + (uint32_t)(((long long)soff[k] - base) * 16), a_lo = a_hi + APLANE;
                        const uint32_t b_hi = saddr(bstage + b * BSTAGE), b_lo = b_hi + TILE;
#pragma unroll
                        for (int ks = 0; ks < KR / 16; ++ks) {
                            const uint32_t ka2 = ks * 2 * ALBO, kb2 = ks * 2 * LBO;
                            mma(tmem, descA(a_hi + ka2), desc(b_hi + kb2), (s % PERIOD != 0 || ks > 0) ? 1u : 0u);
                            mma(tmem, descA(a_hi + ka2), desc(b_lo + kb2), 1u);
                            mma(tmem, descA(a_lo + ka2), desc(b_hi + kb2), 1u);
                        }
                        commit(&empty[b]);
                        if ((s + 1) % PERIOD == 0 || s + 1 == stages) commit(acc_bar);
                    }
                    if (!ok) break;
                    if (c + 1 < chunks || gb < nk) commit(&wempty[slot]);
                }
            }
        }
    } else {                                  // warp 9: the per-(row, tap) tables, two groups ahead
        int g = 0;
        for (int ga = 0, gb = 0; ga < nk && ok; ga = gb, ++g) {
            gb = group_end(ga);
            const int slot = g & 1;
            if (g >= 2) ok = wait_bar(&tempty[slot], (uint32_t)(((g >> 1) - 1) & 1));
            if (!ok) break;
            float4 *tg = tab + slot * (TG * BR);
            for (int e = lane; e < (gb - ga) * BR; e += 32) {
                const int kk = e / BR, j = e - kk * BR;
                const int r = r0 + j;
                float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r < p.n_rng) {
                    t = tap_entry<BPA>(p, r, pmod(soff[ga + kk], n_az));
                    if (!BPA) {
                        const float2 cw = __ldg(w + (size_t)r * K + stap[ga + kk]);
                        t.x = cw.x;
                        t.y = cw.y;
                    }
                }
                tg[kk * BR + j] = t;
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&tfull[slot])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const int th = 32 * q + lane;
    float v[64];
    if (producer) {
        if (ok && stages > 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                ld16(x_ta + 16 * c, v + 16 * c);
                if (have_y) {
                    float yv[16];
                    ld16(y_ta + 16 * c, yv);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[16 * c + j] += yv[j];
                }
            }
        } else {
            const float f = ok ? 0.f : __int_as_float(0x7fc00000);   // no taps: zero; a wait that gave up: NaN
#pragma unroll
            for (int j = 0; j < 64; ++j) v[j] = f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));

    const int G = gridDim.z;
    bool writer = producer;
    if (G > 1) {                              // partial tiles parked in the stage buffers, rank 0 adds in rank order
        float *red = reinterpret_cast<float *>(smem);            // [128 columns][128 pixels] = 64 KB
        cg::cluster_group cluster = cg::this_cluster();
        if (producer) {
#pragma unroll
            for (int j = 0; j < 64; ++j) red[(64 * h + j) * BT + th] = v[j];
        }
        cluster.sync();
        if (producer && cluster.block_rank() == 0) {
            for (int rk = 1; rk < G; ++rk) {
                const float *rem = cluster.map_shared_rank(red, rk);
#pragma unroll
                for (int j = 0; j < 64; ++j) v[j] += rem[(64 * h + j) * BT + th];
            }
        }
        cluster.sync();
        writer = producer && cluster.block_rank() == 0;
    }
    const int tcol = th0 + th;
    if (writer && tcol < n_az) {
#pragma unroll
        for (int j = 0; j < 64; j += 2) {
            const int r = r0 + (64 * h + j) / 2;
            if (r < p.n_rng) out[(size_t)r * n_az + tcol] = make_float2(v[j], v[j + 1]);
        }
    }
}

// Taps in ascending offset order (ties by tap index): offs[i] the i-th smallest offset as given (BPA: k - K/2,
// already ascending), perm[i] its tap.  One CTA; a tap's position is the number of taps before it in that order.
__global__ void __launch_bounds__(256)
td_sort_taps_kernel(const int32_t *__restrict__ o, int K, int bpa, int32_t *__restrict__ offs, int32_t *__restrict__ perm) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int v = bpa ? k - K / 2 : __ldg(o + k);
        int rank = k;
        if (!bpa) {
            rank = 0;
            for (int j = 0; j < K; ++j) {
                const int u = __ldg(o + j);
                rank += (u < v) || (u == v && j < k);
            }
        }
        offs[rank] = v;
        perm[rank] = k;
    }
}

// The B operand tiled as td_tcw_kernel reads it: block (row block rb, sorted tap i, chunk c) holds the B hi tile
// then the B lo tile of rows rb*64 .. rb*64+63 and samples 16c .. 16c+15 (coefficient x window x phasor, each
// sample's phasor taken directly; rows (r, re) = [v.re, -v.im], (r, im) = [v.im, v.re]; rows past n_rng zero).
// Grid (chunks, K, row blocks), 256 threads = 64 rows x 4 groups of 4 samples.
template <bool BPA>
__global__ void __launch_bounds__(256)
td_btile_kernel(const float *__restrict__ win, const float2 *__restrict__ w, const int32_t *__restrict__ offs,
                const int32_t *__restrict__ perm, TdParams p, int K, uint8_t *__restrict__ Bt) {
    using namespace tcg;
    __shared__ float4 tab[BR];
    const int c = blockIdx.x, i = blockIdx.y, rb = blockIdx.z;
    const int chunks = p.L / MC;
    const int k = __ldg(perm + i);
    const int o_n = pmod(__ldg(offs + i), p.n_az);
    if (threadIdx.x < BR) {
        const int r = rb * BR + threadIdx.x;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < p.n_rng) {
            t = tap_entry<BPA>(p, r, o_n);
            if (!BPA) {
                const float2 cw = __ldg(w + (size_t)r * K + k);
                t.x = cw.x;
                t.y = cw.y;
            }
        }
        tab[threadIdx.x] = t;
    }
    __syncthreads();
    const int b_r = threadIdx.x & (BR - 1), b_c = threadIdx.x / BR;
    uint32_t re_hi[4], re_lo[4], im_hi[4], im_lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = c * MC + 4 * b_c + j;
        float2 val = make_float2(0.f, 0.f);
        if (rb * BR + b_r < p.n_rng) val = phasor_term(tab[b_r], win ? __ldg(win + m) : 1.f, (float)m - p.m_ref);
        uint32_t hi, lo;
        split2(val.x, val.y, hi, lo);
        re_hi[j] = hi ^ 0x80000000u;
        re_lo[j] = lo ^ 0x80000000u;
        im_hi[j] = __byte_perm(hi, 0, 0x1032);
        im_lo[j] = __byte_perm(lo, 0, 0x1032);
    }
    uint8_t *blk = Bt + (((size_t)rb * K + i) * chunks + c) * tcw::BTILE;
    *reinterpret_cast<uint4 *>(blk + off(2 * b_r, 8 * b_c)) = make_uint4(re_hi[0], re_hi[1], re_hi[2], re_hi[3]);
    *reinterpret_cast<uint4 *>(blk + TILE + off(2 * b_r, 8 * b_c)) = make_uint4(re_lo[0], re_lo[1], re_lo[2], re_lo[3]);
    *reinterpret_cast<uint4 *>(blk + off(2 * b_r + 1, 8 * b_c)) = make_uint4(im_hi[0], im_hi[1], im_hi[2], im_hi[3]);
    *reinterpret_cast<uint4 *>(blk + TILE + off(2 * b_r + 1, 8 * b_c)) = make_uint4(im_lo[0], im_lo[1], im_lo[2], im_lo[3]);
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

// Cluster size for the tap split: the G (1 .. 8, at most K/4) whose clusters fill the co-resident cluster slots
// in the most nearly whole number of waves (occupancy of the tensor-core kernel: its shared memory and threads).
// Cluster size G (taps split over G CTAs, 1 <= G <= TD_MAX_CLUSTER, at least 4 taps each) that fills the GPU
// in the most nearly whole number of waves (occupancy of the kernel: its shared memory and threads).
int pick_cluster(const void *kernel, int threads, int smem, int tiles, int K) {
    struct Entry { const void *kernel; int dev, tiles, K, G; };
    static Entry cache[8] = {};
    static int next = 0;
    static std::mutex mu;                     // host threads may launch concurrently
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry &e : cache)
            if (e.kernel == kernel && e.dev == dev && e.tiles == tiles && e.K == K) return e.G;
    }
    int best_G = 1;
    double best = -1.0;
    for (int G = 1; G <= TD_MAX_CLUSTER; ++G) {
        if (G > 1 && (K < 4 * G)) break;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3(1, 1, G);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = G;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess || clusters < 1) {
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
    {
        std::lock_guard<std::mutex> lock(mu);
        cache[next] = Entry{kernel, dev, tiles, K, best_G};
        next = (next + 1) % 8;
    }
    return best_G;
}

template <bool BPA>
rosar_status launch_tc(const float2 *raw, const float *win, const float2 *w, const int32_t *o, const TdParams &p, int K,
                       float2 *out, cudaStream_t s) {
    static int done[kMaxDevices] = {};
    rosar_status st = ensure_smem((const void *)td_tc_kernel<BPA>, tcg::SMEM, done, BPA ? "bpa_time" : "sas_time");
    if (st != ROSAR_OK) return st;
    const int gx = (p.n_az + tcg::BT - 1) / tcg::BT, gy = (p.n_rng + tcg::BR - 1) / tcg::BR;
    const int G = pick_cluster((const void *)td_tc_kernel<BPA>, tcg::THREADS, tcg::SMEM, gx * gy, K);
    const int k_per = (K + G - 1) / G;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(gx, gy, G);
    cfg.blockDim = dim3(tcg::THREADS);
    cfg.dynamicSmemBytes = tcg::SMEM;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = G;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, td_tc_kernel<BPA>, raw, win, w, o, p, K, k_per, out);
    if (e != cudaSuccess)
        return set_error(ROSAR_ERR_CUDA, "%s: launch failed: %s", BPA ? "bpa_time" : "sas_time", cudaGetErrorString(e));
    return check_launch(BPA ? "bpa_time" : "sas_time");
}

template <bool BPA>
rosar_status launch_tcg(const float2 *raw, const float *win, const float2 *w, const int32_t *o, const TdParams &p, int K,
                        float2 *out, cudaStream_t s, bool *used) {
    *used = false;
    static int done[kMaxDevices] = {};
    const char *what = BPA ? "bpa_time" : "sas_time";
    rosar_status st = ensure_smem((const void *)td_tcg_kernel<BPA>, tcgn::SMEM, done, what);
    if (st != ROSAR_OK) return st;
    const int gx = (p.n_az + tcg::BT - 1) / tcg::BT, gy = (p.n_rng + tcg::BR - 1) / tcg::BR;
    const int G = pick_cluster((const void *)td_tcg_kernel<BPA>, tcgn::THREADS, tcgn::SMEM, gx * gy, K);
    const int k_per = (K + G - 1) / G;
    if (k_per > tcgn::TAPS_MAX) return ROSAR_OK;             // the caller runs td_tc_kernel instead
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(gx, gy, G);
    cfg.blockDim = dim3(tcgn::THREADS);
    cfg.dynamicSmemBytes = tcgn::SMEM;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = G;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, td_tcg_kernel<BPA>, raw, win, w, o, p, K, k_per, out);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
    *used = true;
    return check_launch(what);
}

template <bool BPA>
rosar_status launch_tcw(const float2 *raw, const uint8_t *Bt, const int32_t *offs, const TdParams &p, int K, float2 *out,
                        cudaStream_t s) {
    static int done[kMaxDevices] = {};
    const char *what = BPA ? "bpa_time_planned" : "sas_time_planned";
    rosar_status st = ensure_smem((const void *)td_tcw_kernel<BPA>, tcw::SMEM, done, what);
    if (st != ROSAR_OK) return st;
    const int gx = (p.n_az + tcg::BT - 1) / tcg::BT, gy = (p.n_rng + tcg::BR - 1) / tcg::BR;
    const int G = pick_cluster((const void *)td_tcw_kernel<BPA>, tcw::THREADS, tcw::SMEM, gx * gy, K);
    const int k_per = (K + G - 1) / G;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(gx, gy, G);
    cfg.blockDim = dim3(tcw::THREADS);
    cfg.dynamicSmemBytes = tcw::SMEM;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = G;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, td_tcw_kernel<BPA>, raw, Bt, offs, p, K, k_per, out);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
    return check_launch(what);
}

}  // namespace

int time_domain_sample_multiple() { return TD_MC; }

namespace {
size_t td_tile_bytes(int n_rng, int L, int K) {
    return (size_t)((n_rng + tcg::BR - 1) / tcg::BR) * (size_t)K * (size_t)(L / TD_MC) * (size_t)tcw::BTILE;
}
}  // namespace

// [row blocks][sorted taps][chunks] B blocks of 16 KB, then the sorted offsets and their taps (int32 each)
size_t time_domain_plan_bytes(int n_rng, int L, int K) {
    return td_tile_bytes(n_rng, L, K) + (((size_t)8 * (size_t)K + 15) & ~(size_t)15);
}

rosar_status launch_time_domain_plan(const float *win, const float2 *w, const int32_t *o, const TdParams &p, int K,
                                     bool bpa, void *plan, cudaStream_t s) {
    if (p.L % TD_MC != 0) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain plan: L=%d is not a multiple of %d", p.L, TD_MC);
    const int rbs = (p.n_rng + tcg::BR - 1) / tcg::BR;
    if (rbs > 65535 || K > 65535)
        return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain plan: n_rng=%d or K=%d too large", p.n_rng, K);
    uint8_t *Bt = static_cast<uint8_t *>(plan);
    int32_t *offs = reinterpret_cast<int32_t *>(Bt + td_tile_bytes(p.n_rng, p.L, K));
    int32_t *perm = offs + K;
    td_sort_taps_kernel<<<1, 256, 0, s>>>(o, K, bpa ? 1 : 0, offs, perm);
    rosar_status st = check_launch(bpa ? "bpa_time_plan" : "sas_time_plan");
    if (st != ROSAR_OK) return st;
    dim3 grid(p.L / TD_MC, K, rbs);
    if (bpa) td_btile_kernel<true><<<grid, 256, 0, s>>>(win, w, offs, perm, p, K, Bt);
    else td_btile_kernel<false><<<grid, 256, 0, s>>>(win, w, offs, perm, p, K, Bt);
    return check_launch(bpa ? "bpa_time_plan" : "sas_time_plan");
}

rosar_status launch_time_domain_planned(const float2 *raw, const TdParams &p, int K, bool bpa, const void *plan,
                                        float2 *out, cudaStream_t s) {
    if (p.L % TD_MC != 0) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: L=%d is not a multiple of %d", p.L, TD_MC);
    if ((p.n_rng + tcg::BR - 1) / tcg::BR > 65535)
        return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: n_rng=%d too large", p.n_rng);
    const uint8_t *Bt = static_cast<const uint8_t *>(plan);
    const int32_t *offs = reinterpret_cast<const int32_t *>(Bt + td_tile_bytes(p.n_rng, p.L, K));
    return bpa ? launch_tcw<true>(raw, Bt, offs, p, K, out, s) : launch_tcw<false>(raw, Bt, offs, p, K, out, s);
}

rosar_status launch_time_domain(const float2 *raw, const float *win, const float2 *w, const int32_t *o,
                                int o_row_stride, const TdParams &p, int K, bool bpa, float2 *out, cudaStream_t s) {
    if (p.L % TD_MC != 0) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: L=%d is not a multiple of %d", p.L, TD_MC);
    if (bpa || o_row_stride == 0) {
        if ((p.n_rng + tcg::BR - 1) / tcg::BR > 65535)
            return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: n_rng=%d too large", p.n_rng);
        bool used = false;
        rosar_status st = bpa ? launch_tcg<true>(raw, win, w, o, p, K, out, s, &used)
                              : launch_tcg<false>(raw, win, w, o, p, K, out, s, &used);
        if (st != ROSAR_OK || used) return st;
        return bpa ? launch_tc<true>(raw, win, w, o, p, K, out, s) : launch_tc<false>(raw, win, w, o, p, K, out, s);
    }
    if (p.n_rng > 65535) return set_error(ROSAR_ERR_UNSUPPORTED, "time-domain: n_rng=%d too large", p.n_rng);
    dim3 grid((p.n_az + TR_BT - 1) / TR_BT, p.n_rng);
    td_row_kernel<<<grid, TR_THREADS, 0, s>>>(raw, win, w, o, o_row_stride, p, K, out);
    return check_launch("sas_time");
}

}  // namespace rosar
