// K1: range compression of every pulse (arXiv 2309.08038, Sec. III-D, Eq. (38)).
//
//   S[l][n] = c_l * sum_m win[m] * raw[n][m] * exp(-j*2*pi*l*m/L),  c_l = exp(+j*pi*l*(L-1)/L)
//
// One CTA transforms P consecutive pulses.  Each pulse uses T = L/16 threads that
// hold 16 complex samples each in registers; the FFT is a Stockham auto-sort
// sequence of radix-16 passes (plus one radix-2/4/8 pass when log2(L) is not a
// multiple of 4), each an in-register DFT followed by an exchange through shared
// memory.  The window is applied as samples are loaded from HBM; the centring
// phase c_l is applied in the last pass, which writes the tile transposed
// ([l][p]) so that the store to the range-major S[l][n0..n0+P) is coalesced
// along azimuth.  Twiddles come from a two-level per-CTA table of exp(-j*pi*q/L)
// (32 + 2L/32 entries, built with sincospif), one lookup per butterfly raised to
// powers.  (fft_tile.cuh holds the tile itself.)
//
// Memory-bound: 16 algorithmic bytes per sample (8 read, 8 written).

#include "fft_tile.cuh"

namespace rosar {
namespace {

// Pulses per CTA for the standalone kernel: small tiles give enough CTAs to cover
// the memory latency at the scan sizes of interest.
template <int L>
struct Plan : fft::Tile<L, (L <= 16 ? 32 : L <= 64 ? 16 : L <= 256 ? 8 : L <= 1024 ? 4 : 2)> {};

template <int L>
__global__ void __launch_bounds__(Plan<L>::THREADS)
range_compress_kernel(const float2 *__restrict__ raw, const float *__restrict__ win, int n_az, int centred,
                      float2 *__restrict__ S, int vec_store) {
    extern __shared__ float2 smem[];
    const size_t scan = (size_t)blockIdx.y * n_az * L;      // grid.y: scans of a stack
    fft::range_tile<L, Plan<L>::P>(raw + scan, win, n_az, centred != 0, S + scan, blockIdx.x * Plan<L>::P, smem, true,
                                   vec_store != 0);
}

template <int L>
__global__ void __launch_bounds__(Plan<L>::THREADS)
range_adjoint_kernel(const float2 *__restrict__ g, const float *__restrict__ win, int n_az, int centred,
                     float2 *__restrict__ grad_raw) {
    extern __shared__ float2 smem[];
    const size_t scan = (size_t)blockIdx.y * n_az * L;      // grid.y: scans of a stack
    fft::range_adjoint_tile<L, Plan<L>::P>(g + scan, win, n_az, centred != 0, grad_raw + scan, blockIdx.x * Plan<L>::P,
                                           smem);
}

template <int L>
rosar_status launch_adjoint_L(const float2 *g, const float *win, int n_az, int centred, float2 *grad_raw,
                              cudaStream_t s, int n_scans) {
    using PL = Plan<L>;
    if (PL::SMEM > 48 * 1024) {
        static int done[kMaxDevices] = {};
        rosar_status st = ensure_smem((const void *)range_adjoint_kernel<L>, PL::SMEM, done, "range_compress_adjoint");
        if (st != ROSAR_OK) return st;
    }
    const dim3 grid((n_az + PL::P - 1) / PL::P, n_scans);
    range_adjoint_kernel<L><<<grid, PL::THREADS, PL::SMEM, s>>>(g, win, n_az, centred, grad_raw);
    return check_launch("range_compress_adjoint");
}

template <int L>
rosar_status launch_L(const float2 *raw, const float *win, int n_az, int centred, float2 *S, cudaStream_t s,
                      int n_scans) {
    using PL = Plan<L>;
    static_assert(PL::SMEM <= 227 * 1024, "range-compress tile exceeds shared memory");
    if (PL::SMEM > 48 * 1024) {
        static int done[kMaxDevices] = {};
        rosar_status st = ensure_smem((const void *)range_compress_kernel<L>, PL::SMEM, done, "range_compress");
        if (st != ROSAR_OK) return st;
    }
    const dim3 grid((n_az + PL::P - 1) / PL::P, n_scans);
    const int vec = ((n_az % 2) == 0) && ((reinterpret_cast<uintptr_t>(S) & 15) == 0);
    range_compress_kernel<L><<<grid, PL::THREADS, PL::SMEM, s>>>(raw, win, n_az, centred, S, vec);
    return check_launch("range_compress");
}

}  // namespace

rosar_status launch_range_compress(const float2 *raw, const float *win, int n_az, int L, int centred, float2 *S,
                                   cudaStream_t s, int n_scans) {
    if (n_scans < 1 || n_scans > 65535)
        return set_error(ROSAR_ERR_UNSUPPORTED, "range_compress: n_scans=%d not in [1, 65535]", n_scans);
    switch (L) {
        case 8: return launch_L<8>(raw, win, n_az, centred, S, s, n_scans);
        case 16: return launch_L<16>(raw, win, n_az, centred, S, s, n_scans);
        case 32: return launch_L<32>(raw, win, n_az, centred, S, s, n_scans);
        case 64: return launch_L<64>(raw, win, n_az, centred, S, s, n_scans);
        case 128: return launch_L<128>(raw, win, n_az, centred, S, s, n_scans);
        case 256: return launch_L<256>(raw, win, n_az, centred, S, s, n_scans);
        case 512: return launch_L<512>(raw, win, n_az, centred, S, s, n_scans);
        case 1024: return launch_L<1024>(raw, win, n_az, centred, S, s, n_scans);
        case 2048: return launch_L<2048>(raw, win, n_az, centred, S, s, n_scans);
        case 4096: return launch_L<4096>(raw, win, n_az, centred, S, s, n_scans);
        default: return set_error(ROSAR_ERR_UNSUPPORTED, "range_compress: L=%d is not a power of two in [8, 4096]", L);
    }
}

rosar_status launch_range_compress_adjoint(const float2 *g, const float *win, int n_az, int L, int centred,
                                           float2 *grad_raw, cudaStream_t s, int n_scans) {
    if (n_scans < 1 || n_scans > 65535)
        return set_error(ROSAR_ERR_UNSUPPORTED, "range_compress_adjoint: n_scans=%d not in [1, 65535]", n_scans);
    switch (L) {
        case 8: return launch_adjoint_L<8>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 16: return launch_adjoint_L<16>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 32: return launch_adjoint_L<32>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 64: return launch_adjoint_L<64>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 128: return launch_adjoint_L<128>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 256: return launch_adjoint_L<256>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 512: return launch_adjoint_L<512>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 1024: return launch_adjoint_L<1024>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 2048: return launch_adjoint_L<2048>(g, win, n_az, centred, grad_raw, s, n_scans);
        case 4096: return launch_adjoint_L<4096>(g, win, n_az, centred, grad_raw, s, n_scans);
        default:
            return set_error(ROSAR_ERR_UNSUPPORTED, "range_compress_adjoint: L=%d is not a power of two in [8, 4096]", L);
    }
}

}  // namespace rosar
