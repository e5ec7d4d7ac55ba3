// Imaging a sequence of scans with the frequency-domain filter, software-pipelined across scans
// (arXiv 2309.08038, Sec. III-D: Eq. (38) range compression, then Eq. (43) per range row).
//
// For one scan the two stages are strictly ordered (every azimuth row needs every pulse's range
// transform), so a single image leaves the GPU half idle at each hand-over: the range kernel is one
// short wave whose loads and stores cannot overlap, and the azimuth kernel has one row per CTA for
// 256 rows on 152 SMs.  Across scans they are independent, so stage i of the pipeline runs, in ONE
// launch, the azimuth rows of scan i-1 (CTAs 0 .. L-1, longest work first) and the range tiles of
// scan i (the CTAs after them).  Two workspaces alternate: scan i's range tiles write ws[i & 1] while
// scan i-1's rows read ws[(i-1) & 1].
//
// Stages are chained with programmatic dependent launch: every CTA lets the next stage start at once,
// the azimuth rows wait for the previous stage (their S) before their first read of S, and the range
// tiles wait before storing (the previous stage's rows read the buffer they overwrite; the raw cube
// was written before the first stage, which is launched without overlap).  The arithmetic of both
// parts is that of rosar_range_compress and rosar_sparse_azimuth_fft, so every image equals a
// rosar_image_fft call bit for bit.

#include "row_fft.cuh"

namespace rosar {
namespace {

constexpr int kStageThreads = 256;

template <int L>
constexpr int stage_pulses() { return 4096 / L; }     // 16 threads per pulse of 256 samples, 256 threads

template <int L, int N, int... R>
constexpr size_t stage_smem() {
    constexpr size_t a = rowfft::filter_row_smem<N>();
    constexpr size_t b = fft::Tile<L, stage_pulses<L>()>::SMEM;
    return a > b ? a : b;
}

// Stage kernel: blocks [0, L) filter the rows of the previous scan (S_prev -> out_prev); blocks
// [L, L + ceil(n_az / P)) range-compress the pulses of the current scan (raw_cur -> S_cur).  Either
// part may be absent (the first and last stages).
template <int L, int N, int... R>
__global__ void __launch_bounds__(kStageThreads, 3)
image_stage_kernel(const float2 *__restrict__ S_prev, const float2 *__restrict__ H, float2 *__restrict__ out_prev,
                   int n_rows, const float2 *__restrict__ raw_cur, const float *__restrict__ win,
                   float2 *__restrict__ S_cur, int vec_store) {
    extern __shared__ float2 sm[];
    griddep_launch_dependents();
    const int b = blockIdx.x;
    if (b < n_rows) {
        rowfft::filter_row_cta<kStageThreads, N, true, R...>(S_prev + (size_t)b * N, H + (size_t)b * N, false,
                                                       out_prev + (size_t)b * N, sm);
    } else {
        constexpr int P = stage_pulses<L>();
        fft::range_tile<L, P>(raw_cur, win, N, true, S_cur, (b - n_rows) * P, sm, true, vec_store != 0, true);
    }
}

using StageFn = void (*)(const float2 *, const float2 *, float2 *, int, const float2 *, const float *, float2 *, int);

struct StagePlan {
    int L, N;
    StageFn fn;
    size_t smem;
    int pulses;
    int *smem_done;        // per-kernel record of the shared-memory limit set on each device
};

template <int L, int N, int... R>
StagePlan stage_plan() {
    static int done[kMaxDevices] = {};
    return StagePlan{L, N, image_stage_kernel<L, N, R...>, stage_smem<L, N, R...>(), stage_pulses<L>(), done};
}

// The (L, n_az) pairs with a pipelined stage kernel; the azimuth radices must be those the run-time
// planner picks for n_az (H is in that order): checked before use.
const StagePlan *find_stage(int L, int n_az) {
    static const StagePlan plans[] = {
        stage_plan<64, 360, 8, 3, 15>(),     stage_plan<128, 1800, 8, 15, 15>(), stage_plan<256, 1800, 8, 15, 15>(),
        stage_plan<128, 3600, 16, 15, 15>(), stage_plan<256, 3600, 16, 15, 15>(), stage_plan<512, 3600, 16, 15, 15>(),
    };
    static const int rad360[] = {8, 3, 15}, rad1800[] = {8, 15, 15}, rad3600[] = {16, 15, 15};
    for (const StagePlan &p : plans) {
        if (p.L != L || p.N != n_az) continue;
        rowfft::RowPlan pl;
        if (!rowfft::make_plan(n_az, &pl) || rowfft::threads_for(n_az) != kStageThreads) return nullptr;
        const int *rad = n_az == 360 ? rad360 : n_az == 1800 ? rad1800 : rad3600;
        if (pl.npass != 3 || pl.rad[0] != rad[0] || pl.rad[1] != rad[1] || pl.rad[2] != rad[2]) return nullptr;
        return &p;
    }
    return nullptr;
}

rosar_status launch_stage(const StagePlan &p, bool overlap, const float2 *S_prev, const float2 *H, float2 *out_prev,
                          const float2 *raw_cur, const float *win, float2 *S_cur, cudaStream_t s) {
    rosar_status st = ensure_smem((const void *)p.fn, p.smem, p.smem_done, "image_fft_scans");
    if (st != ROSAR_OK) return st;
    const int rows = S_prev ? p.L : 0;
    const int tiles = raw_cur ? (p.N + p.pulses - 1) / p.pulses : 0;
    const int vec = (p.N % 2 == 0) && S_cur && ((reinterpret_cast<uintptr_t>(S_cur) & 15) == 0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(rows + tiles);
    cfg.blockDim = dim3(kStageThreads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = overlap ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, p.fn, S_prev, H, out_prev, rows, raw_cur, win, S_cur, vec);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "image_fft_scans: launch failed: %s", cudaGetErrorString(e));
    return check_launch("image_fft_scans");
}

}  // namespace

int image_pipeline_supported(int L, int n_az) { return find_stage(L, n_az) ? 1 : 0; }

rosar_status launch_image_pipeline(const float2 *raw, const float *win, const float2 *H, int n_scans, int n_az, int L,
                                   float2 *workspace, float2 *out, cudaStream_t s) {
    const StagePlan *p = find_stage(L, n_az);
    if (!p) return set_error(ROSAR_ERR_UNSUPPORTED, "image_fft_scans: no pipelined plan for L=%d n_az=%d", L, n_az);
    const size_t cube = (size_t)n_az * L;
    float2 *ws[2] = {workspace, workspace + cube};
    // stage 0: range tiles of scan 0 only, ordered after everything before it in the stream
    rosar_status st = launch_stage(*p, false, nullptr, H, nullptr, raw, win, ws[0], s);
    for (int i = 1; st == ROSAR_OK && i <= n_scans; ++i) {
        const bool has_cur = i < n_scans;
        st = launch_stage(*p, true, ws[(i - 1) & 1], H, out + (size_t)(i - 1) * cube, has_cur ? raw + (size_t)i * cube : nullptr,
                          win, has_cur ? ws[i & 1] : nullptr, s);
    }
    return st;
}

}  // namespace rosar
