// Image loss of the differentiable form and its gradient: the squared L2 distance between a stack of images
// (Eq. (43) outputs, arXiv 2309.08038 Sec. III-D) and a reference stack, e.g. back-projection images:
//
//   loss    = sum_i |out[i] - ref[i]|^2
//   grad[i] = 2 g (out[i] - ref[i])        (torch's conjugate-Wirtinger gradient for the upstream scalar g)
//
// One pass each way over the two stacks instead of the separate difference, square, reduction and backward
// kernels of a composed expression.  The reduction is deterministic: the elements are cut into
// kLossBlocks contiguous chunks fixed by n alone, each chunk is summed by one CTA in a fixed order (per-thread
// float sums, then a double tree), and a second one-CTA kernel adds the chunk sums in chunk order.

#include "rosar_internal.cuh"

namespace rosar {
namespace {

constexpr int kLossThreads = 256;
constexpr int kLossBlocks = 1216;            // 8 per SM of a 152-SM GB300; fixed so the sum order depends on n only

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLossThreads / 32; ++w) t += red[w];
    return t;
}

__global__ void __launch_bounds__(kLossThreads)
loss_partial_kernel(const float2 *__restrict__ out, const float2 *__restrict__ ref, long long n, long long chunk,
                    double *__restrict__ partial) {
    __shared__ double red[kLossThreads / 32];
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = min(n, lo + chunk);
    float acc = 0.f;
    for (long long i = lo + threadIdx.x; i < hi; i += kLossThreads) {
        const float2 a = __ldcs(out + i), b = __ldcs(ref + i);
        const float dx = a.x - b.x, dy = a.y - b.y;
        acc = fmaf(dx, dx, acc);
        acc = fmaf(dy, dy, acc);
    }
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kLossThreads)
loss_final_kernel(const double *__restrict__ partial, int nb, float *__restrict__ loss) {
    __shared__ double red[kLossThreads / 32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += kLossThreads) acc += partial[b];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) *loss = (float)s;
}

__global__ void __launch_bounds__(kLossThreads)
loss_grad_kernel(const float2 *__restrict__ out, const float2 *__restrict__ ref, long long n,
                 const float *__restrict__ g, float2 *__restrict__ grad) {
    const float s = 2.f * __ldg(g);
    for (long long i = (long long)blockIdx.x * kLossThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kLossThreads) {
        const float2 a = __ldcs(out + i), b = __ldcs(ref + i);
        __stcs(grad + i, make_float2(s * (a.x - b.x), s * (a.y - b.y)));
    }
}

}  // namespace

int image_loss_partials() { return kLossBlocks; }

rosar_status launch_image_l2_loss(const float2 *out, const float2 *ref, long long n, double *partial, float *loss,
                                  cudaStream_t s) {
    const int nb = n < kLossBlocks ? (int)n : kLossBlocks;
    const long long chunk = (n + nb - 1) / nb;
    loss_partial_kernel<<<nb, kLossThreads, 0, s>>>(out, ref, n, chunk, partial);
    rosar_status st = check_launch("image_l2_loss");
    if (st != ROSAR_OK) return st;
    loss_final_kernel<<<1, kLossThreads, 0, s>>>(partial, nb, loss);
    return check_launch("image_l2_loss");
}

rosar_status launch_image_l2_loss_grad(const float2 *out, const float2 *ref, long long n, const float *g,
                                       float2 *grad, cudaStream_t s) {
    const long long want = (n + kLossThreads - 1) / kLossThreads;
    const long long blocks = want < 152LL * 16 ? want : 152LL * 16;
    loss_grad_kernel<<<(unsigned)blocks, kLossThreads, 0, s>>>(out, ref, n, g, grad);
    return check_launch("image_l2_loss_grad");
}

}  // namespace rosar
