// Batched form: many uneven scans, one persistent launch inside a CUDA graph.
//
// Work is a list of tiles in ticket order.  A range tile runs the range-FFT tile
// (fft_tile.cuh) on P = 4096/L pulses of one scan with the CTA's 256 threads; an
// azimuth tile runs the gather-MAC tile (azimuth_tile.cuh) on 256*J outputs of one
// row of one scan, or, for a scan given its frequency-domain plan H, the whole row
// through the row FFT (row_fft.cuh): forward transform, product with H, inverse.
// Tickets are handed out by an atomic counter, range tiles of a scan always before
// its azimuth tiles; the scan's done-counter is bumped (release) after each range
// tile, and an azimuth tile's thread 0 polls it (acquire) before the CTA reads S
// through L2.  The poll is bounded; on expiry the kernel raises an error word that
// every CTA checks before taking its next ticket.
//
// Keeping S in L2: with interleave d >= 2 the range tiles of scan s+d-1 and the
// azimuth tiles of scan s alternate in `mix` chunks each, so a scan's S is read
// back while it is still in L2, and with DISCARD_S whole-row FFT tiles drop each
// S row from L2 once read, so S, a scratch buffer, is not written back to memory
// while it stays cached.  A CTA takes its next ticket when it starts a tile.

#include <stdlib.h>
#include <string.h>

#include <new>

#include "azimuth_tile.cuh"
#include "fft_tile.cuh"
#include "row_fft.cuh"

namespace rosar {
namespace {

constexpr int BT_THREADS = 256;

struct ScanDev {
    const float2 *raw;
    const float *win;
    const float2 *w;
    const int32_t *o;
    float2 *S;
    float2 *out;
    const float2 *H;          // frequency-domain plan [L][n_az], or null: gather tiles
    int o_row_stride, n_az, L, K;
    int range_tiles, az_tiles_per_row, P, vec_store;
    int fixed;                // compile-time plan of the row FFT (1: 1800, 2: 3600, 3: 7200 pulses), 0: run-time plan
    rowfft::RowPlan plan;
};

struct Segment {
    int first;   // first ticket
    int scan;
    int kind;    // 0 range tiles, 1 azimuth tiles
    int count;
    int start;   // tile index (within the scan's tiles of this kind) of the segment's first ticket
};

constexpr int MIX_MAX = 32;              // chunks per scan and kind
constexpr int SEGS_PER_SCAN = 2 * MIX_MAX;

// counters[0] ticket head, [1] error flag, [2] scan that timed out, [3] unused, [4 + s] range tiles done of scan s
constexpr int CNT_HEAD = 0, CNT_ERR = 1, CNT_ERR_SCAN = 2, CNT_DONE = 4;

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int L>
__device__ __forceinline__ void run_range(const ScanDev &sc, int n0, char *sm, bool build) {
    fft::range_tile<L, 4096 / L>(sc.raw, sc.win, sc.n_az, true, sc.S, n0, reinterpret_cast<float2 *>(sm), build,
                                 sc.vec_store != 0);
}
// Range lengths outside 128..1024 out of line, like fft_row_runtime below: they are rare, and inlined their
// register needs cost the common paths spills.
template <int L>
__device__ __noinline__ void run_range_rare(const ScanDev &sc, int n0, char *sm, bool build) {
    run_range<L>(sc, n0, sm, build);
}

// The rows without a compile-time plan (run-time radices), kept out of line: inlined, their register needs
// made the whole kernel spill.
__device__ __noinline__ void fft_row_runtime(const ScanDev &sc, const float2 *Srow, size_t row, float2 *x,
                                             const float2 *tc, const float2 *tf) {
    const int N = sc.n_az;
    for (int n0 = threadIdx.x; n0 < N; n0 += 8 * BT_THREADS) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int n = n0 + u * BT_THREADS;
            v[u] = n < N ? __ldcg(Srow + n) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int n = n0 + u * BT_THREADS;
            if (n < N) x[rowfft::rpad(n, sc.plan.pad_shift)] = v[u];
        }
    }
    __syncthreads();
    rowfft::row_dif(x, N, sc.plan, tc, tf);
    for (int n = threadIdx.x; n < N; n += BT_THREADS) {
        const float2 y = cmul(__ldg(sc.H + row + n), x[rowfft::rpad(n, sc.plan.pad_shift)]);
        x[rowfft::rpad(n, sc.plan.pad_shift)] = make_float2(y.x, -y.y);
    }
    __syncthreads();
    rowfft::row_dit(x, N, sc.plan, tc, tf);
    for (int n = threadIdx.x; n < N; n += BT_THREADS) {
        const float2 y = x[rowfft::rpad(n, sc.plan.pad_shift)];
        sc.out[row + n] = make_float2(y.x, -y.y);
    }
    __syncthreads();
}

// One range row of a scan through the frequency-domain azimuth filter (same arithmetic as
// rosar_sparse_azimuth_fft).  S was written by this kernel's range tiles: read through L2 (ld.cg).  The row
// lengths with a compile-time plan run the fused filter (first and last passes on global memory, H read from
// global in the fused middle step); the others load the row, eight loads in flight per thread, and run the
// run-time plan.
// build_tw = false: the previous tile of this CTA was a row of the same length and left its twiddle table in
// place (the rows write only their buffer in front of it).
__device__ __forceinline__ void fft_row_tile(const ScanDev &sc, int r, char *smem, bool discard, bool build_tw) {
    const int N = sc.n_az;
    float2 *x = reinterpret_cast<float2 *>(smem);
    float2 *tw = x + rowfft::padded_len(N);
    const float2 *tc = tw + 64, *tf = tw;           // the layout build_twiddles(N, false, ...) writes
    if (build_tw) rowfft::build_twiddles(N, false, tw, &tc, &tf);
    const size_t row = (size_t)r * N;
    const float2 *Srow = sc.S + row;
    if (sc.fixed) {
        if (build_tw) __syncthreads();        // else the caller's dependency barrier already ordered shared memory
        switch (sc.fixed) {                   // the run-time plan's radices, constant strides
            case 1: rowfft::row_filter_fused<1800, BT_THREADS, false, 8, 15, 15>(Srow, sc.H + row, 1.f, x, sc.out + row, tc, tf, discard); break;
            case 2: rowfft::row_filter_fused<3600, BT_THREADS, false, 16, 15, 15>(Srow, sc.H + row, 1.f, x, sc.out + row, tc, tf, discard); break;
            default: rowfft::row_filter_fused<7200, BT_THREADS, false, 8, 4, 15, 15>(Srow, sc.H + row, 1.f, x, sc.out + row, tc, tf, discard); break;
        }
        __syncthreads();
        return;
    }
    fft_row_runtime(sc, Srow, row, x, tc, tf);
}

__device__ __forceinline__ int find_segment(const Segment *__restrict__ segs, int n_segs, int t) {
    int lo = 0, hi = n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&segs[mid].first) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int J>
__global__ void __launch_bounds__(BT_THREADS, 3)
batch_kernel(const ScanDev *__restrict__ scans, const Segment *__restrict__ segs, int n_segs, int total,
             int *counters, int spin_limit, int debug_scan, int flags) {
    extern __shared__ __align__(16) char sm[];
    __shared__ int red[4 * az::THREADS / 32];
    __shared__ int s_ticket[2], s_abort;
    // the segment and scan of the current and the next ticket, decoded once by the thread that takes the ticket
    __shared__ Segment s_sg[2];
    __shared__ ScanDev s_sc[2];
    int *head = counters + CNT_HEAD, *err = counters + CNT_ERR, *done = counters + CNT_DONE;
    const bool discard = (flags & ROSAR_BATCH_DISCARD_S) != 0;
    int tab_L = 0;   // L of the twiddle table left in shared memory by the previous range tile
    int tab_N = 0;   // n_az of the row twiddle table left by the previous azimuth FFT tile

    // a CTA holds two tickets: the tile it runs and the next one, taken when the current tile starts (the
    // smallest unfinished ticket is always some CTA's current tile, and its dependencies have smaller tickets,
    // so every wait ends)
    constexpr int GRAB = 32;   // the thread that takes tickets (warp 1: thread 0 does the dependency waits)
    auto decode = [&](int slot, int tk) {     // the ticket's segment and scan into shared memory (GRAB only)
        s_ticket[slot] = tk;
        if (tk < total) {
            const Segment g = segs[find_segment(segs, n_segs, tk)];
            s_sg[slot] = g;
            s_sc[slot] = scans[g.scan];
        }
    };
    if (threadIdx.x == GRAB) decode(0, atomicAdd(head, 1));
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const int t = s_ticket[cur];
        if (t >= total) break;
        const Segment sg = s_sg[cur];
        const ScanDev &sc = s_sc[cur];
        const int local = t - sg.first + sg.start;
        if (threadIdx.x == 0) s_abort = 0;
        if (threadIdx.x == GRAB) {
            int nt = atomicAdd(head, 1);
            if (nt < total && ld_relaxed(err) != 0) nt = total;
            decode(cur ^ 1, nt);
        }
        if (sg.kind == 0) {
            const bool build = tab_L != sc.L;
            const int n0 = local * sc.P;
            switch (sc.L) {
                case 16: run_range_rare<16>(sc, n0, sm, build); break;
                case 32: run_range_rare<32>(sc, n0, sm, build); break;
                case 64: run_range_rare<64>(sc, n0, sm, build); break;
                case 128: run_range<128>(sc, n0, sm, build); break;
                case 256: run_range<256>(sc, n0, sm, build); break;
                case 512: run_range<512>(sc, n0, sm, build); break;
                case 1024: run_range<1024>(sc, n0, sm, build); break;
                default: run_range_rare<2048>(sc, n0, sm, build); break;
            }
            tab_L = sc.L;
            tab_N = 0;             // the range tile overwrites the row table
            __threadfence();       // this thread's S stores are visible device-wide ...
            __syncthreads();       // ... for every thread of the tile ...
            if (threadIdx.x == 0) atomicAdd(done + sg.scan, 1);   // ... before the tile is counted
        } else {
            tab_L = 0;             // the azimuth tile overwrites the table
            if (threadIdx.x == 0) {
                const int need = sc.range_tiles + (sg.scan == debug_scan ? 1 : 0);
                int polls = 0;
                while (ld_acquire(done + sg.scan) < need) {
                    if (++polls > spin_limit || ((polls & 255) == 0 && ld_relaxed(err) != 0)) {
                        if (atomicExch(err, 1) == 0) atomicExch(counters + CNT_ERR_SCAN, sg.scan);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __syncthreads();
            if (s_abort) break;
            if (sc.H) {
                fft_row_tile(sc, local, sm, discard, tab_N != sc.n_az);
                tab_N = sc.n_az;
            } else {
                tab_N = 0;         // the gather tile overwrites the row table
                const int r = local / sc.az_tiles_per_row;
                const int th0 = (local - r * sc.az_tiles_per_row) * az::Geo<J>::TW;
                az::azimuth_tile<J, true>(sc.S, sc.w, sc.o, sc.o_row_stride, sc.n_az, sc.K, sc.out, r, th0, sm, red);
            }
        }
        __syncthreads();           // the tile is done with shared memory; the next ticket is visible
    }
}

using KernelFn = void (*)(const ScanDev *, const Segment *, int, int, int *, int, int, int);

KernelFn kernel_for(int J) {
    switch (J) {
        case 1: return batch_kernel<1>;
        case 2: return batch_kernel<2>;
        case 8: return batch_kernel<8>;
        default: return batch_kernel<4>;
    }
}

// The compile-time plans fft_row_tile carries, used only when the run-time planner picks the same radices.
int fixed_plan_code(int n_az, const rowfft::RowPlan &pl) {
    static const int r1800[] = {8, 15, 15}, r3600[] = {16, 15, 15}, r7200[] = {8, 4, 15, 15};
    const int *rad = n_az == 1800 ? r1800 : n_az == 3600 ? r3600 : n_az == 7200 ? r7200 : nullptr;
    const int np = n_az == 7200 ? 4 : 3;
    if (!rad || pl.npass != np || pl.pad_shift != rowfft::pad_shift_for(n_az)) return 0;
    for (int i = 0; i < np; ++i)
        if (pl.rad[i] != rad[i]) return 0;
    return n_az == 1800 ? 1 : n_az == 3600 ? 2 : 3;
}

int g_smem_done[4][kMaxDevices] = {};

int j_index(int J) { return J == 1 ? 0 : J == 2 ? 1 : J == 4 ? 2 : 3; }

int range_smem_bytes(int L) {
    switch (L) {
        case 16: return (int)fft::Tile<16, 256>::SMEM;
        case 32: return (int)fft::Tile<32, 128>::SMEM;
        case 64: return (int)fft::Tile<64, 64>::SMEM;
        case 128: return (int)fft::Tile<128, 32>::SMEM;
        case 256: return (int)fft::Tile<256, 16>::SMEM;
        case 512: return (int)fft::Tile<512, 8>::SMEM;
        case 1024: return (int)fft::Tile<1024, 4>::SMEM;
        default: return (int)fft::Tile<2048, 2>::SMEM;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace rosar

using namespace rosar;

struct rosar_batch {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int *counters;           // device
    int n_scans;
    int range_tiles, az_tiles, ctas, smem;
};

extern "C" {

size_t rosar_batch_workspace_bytes(int n_scans) {
    if (n_scans < 1) return 0;
    return align256(sizeof(ScanDev) * (size_t)n_scans) + align256(sizeof(Segment) * SEGS_PER_SCAN * (size_t)n_scans) +
           align256(sizeof(int) * (CNT_DONE + (size_t)n_scans));
}

rosar_status rosar_batch_create(const rosar_scan *scans, int n_scans, const rosar_batch_tuning *tuning,
                                void *workspace, size_t workspace_bytes, rosar_batch **batch) {
    clear_error();
    if (!scans || !workspace || !batch) return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: null argument");
    *batch = nullptr;
    if (n_scans < 1) return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: n_scans=%d < 1", n_scans);
    if (workspace_bytes < rosar_batch_workspace_bytes(n_scans))
        return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: workspace of %zu bytes < %zu needed", workspace_bytes,
                         rosar_batch_workspace_bytes(n_scans));
    if (reinterpret_cast<uintptr_t>(workspace) % 256)
        return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: workspace must be 256-byte aligned");
    rosar_batch_tuning tn = {1024, 0, 0, 1 << 24, -1, 1, 0};
    if (tuning) tn = *tuning;
    if (tn.az_tile == 0) tn.az_tile = 1024;
    if (tn.spin_limit <= 0) tn.spin_limit = 1 << 24;
    if (tn.mix <= 0) tn.mix = 1;
    if (tn.interleave < 0 || tn.interleave > 8)
        return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: interleave=%d not in [0, 8]", tn.interleave);
    if (tn.mix > MIX_MAX)
        return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: mix=%d not in [1, %d]", tn.mix, MIX_MAX);
    if (tn.flags & ~ROSAR_BATCH_DISCARD_S)
        return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: unknown flags 0x%x", tn.flags);
    const int J = tn.az_tile / az::THREADS;
    if (tn.az_tile % az::THREADS || (J != 1 && J != 2 && J != 4 && J != 8))
        return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: az_tile=%d not in {256, 512, 1024, 2048}", tn.az_tile);

    ScanDev *hs = static_cast<ScanDev *>(calloc((size_t)n_scans, sizeof(ScanDev)));
    Segment *hg = static_cast<Segment *>(calloc(SEGS_PER_SCAN * (size_t)n_scans, sizeof(Segment)));
    if (!hs || !hg) {
        free(hs);
        free(hg);
        return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: host allocation failed");
    }
    int smem = az::Geo<8>::SMEM_BYTES;
    switch (J) {
        case 1: smem = az::Geo<1>::SMEM_BYTES; break;
        case 2: smem = az::Geo<2>::SMEM_BYTES; break;
        case 4: smem = az::Geo<4>::SMEM_BYTES; break;
        default: break;
    }
    long long total_range = 0, total_az = 0;
    rosar_status st = ROSAR_OK;
    for (int s = 0; s < n_scans && st == ROSAR_OK; ++s) {
        const rosar_scan &q = scans[s];
        if (!q.raw || !q.w || !q.o || !q.S || !q.out)
            st = set_error(ROSAR_ERR_INVALID_ARG, "batch_create: scan %d has a null pointer", s);
        else if (q.n_az < 1 || q.K < 1 || (q.o_row_stride != 0 && q.o_row_stride < q.K))
            st = set_error(ROSAR_ERR_INVALID_ARG, "batch_create: scan %d: n_az=%d K=%d o_row_stride=%d", s, q.n_az,
                           q.K, q.o_row_stride);
        else if (!is_pow2(q.L) || q.L < 16 || q.L > 2048)
            st = set_error(ROSAR_ERR_UNSUPPORTED, "batch_create: scan %d: L=%d not a power of two in [16, 2048]", s,
                           q.L);
        else if ((long long)q.L * q.n_az > (1LL << 31) - 1)
            st = set_error(ROSAR_ERR_UNSUPPORTED, "batch_create: scan %d too large", s);
        if (st != ROSAR_OK) break;
        ScanDev &d = hs[s];
        d.raw = reinterpret_cast<const float2 *>(q.raw);
        d.win = q.win;
        d.w = reinterpret_cast<const float2 *>(q.w);
        d.o = q.o;
        d.S = reinterpret_cast<float2 *>(q.S);
        d.out = reinterpret_cast<float2 *>(q.out);
        d.H = reinterpret_cast<const float2 *>(q.H);
        if (q.H && !rowfft::make_plan(q.n_az, &d.plan)) {
            st = set_error(ROSAR_ERR_UNSUPPORTED, "batch_create: scan %d: n_az=%d has no frequency-domain plan", s,
                           q.n_az);
            break;
        }
        d.fixed = q.H ? fixed_plan_code(q.n_az, d.plan) : 0;
        d.o_row_stride = q.o_row_stride;
        d.n_az = q.n_az;
        d.L = q.L;
        d.K = q.K;
        d.P = 4096 / q.L;
        d.range_tiles = (q.n_az + d.P - 1) / d.P;
        d.az_tiles_per_row = q.H ? 1 : (q.n_az + tn.az_tile - 1) / tn.az_tile;
        d.vec_store = (q.n_az % 2 == 0) && (reinterpret_cast<uintptr_t>(q.S) % 16 == 0);
        smem = smem > range_smem_bytes(q.L) ? smem : range_smem_bytes(q.L);
        if (q.H) {
            const int rs = (int)(sizeof(float2) * (size_t)(rowfft::padded_len(q.n_az) + 64 + rowfft::coarse_len(q.n_az)));
            smem = smem > rs ? smem : rs;
        }
        total_range += d.range_tiles;
        total_az += (long long)d.az_tiles_per_row * q.L;
    }
    if (st == ROSAR_OK && total_range + total_az > (1LL << 31) - 1)
        st = set_error(ROSAR_ERR_UNSUPPORTED, "batch_create: %lld tiles exceed 2^31", total_range + total_az);
    if (st != ROSAR_OK) {
        free(hs);
        free(hg);
        return st;
    }
    // ticket order.  Azimuth tiles of a scan always come after all of its range tiles, so every range tile an
    // azimuth tile waits for has been handed to a running CTA (which waits on nothing) before it.
    int first = 0, ns = 0;
    auto push = [&](int s, int kind, int start, int count) {
        if (count > 0) {
            hg[ns++] = {first, s, kind, count, start};
            first += count;
        }
    };
    auto n_range = [&](int s) { return hs[s].range_tiles; };
    auto n_az = [&](int s) { return hs[s].az_tiles_per_row * hs[s].L; };
    if (tn.interleave >= 1) {
        // range tiles run (interleave - 1) scans ahead of the azimuth tiles: 1 = scan by scan, 2 = the next
        // scan's range tiles alongside this scan's azimuth tiles (its S is produced while this one is
        // filtered).  With mix = m the two lists alternate in m chunks each (range chunk first).
        const int ahead = tn.interleave - 1;
        for (int s = 0; s < n_scans && s < ahead; ++s) push(s, 0, 0, n_range(s));
        for (int s = 0; s < n_scans; ++s) {
            const int rs = s + ahead;
            const int nr = (rs < n_scans && ahead > 0) ? n_range(rs) : 0, na = n_az(s);
            if (ahead == 0) push(s, 0, 0, n_range(s));
            const int m = ahead > 0 ? tn.mix : 1;
            for (int c = 0; c < m; ++c) {
                const int r0 = (int)((long long)nr * c / m), r1 = (int)((long long)nr * (c + 1) / m);
                const int a0 = (int)((long long)na * c / m), a1 = (int)((long long)na * (c + 1) / m);
                push(rs, 0, r0, r1 - r0);
                push(s, 1, a0, a1 - a0);
            }
        }
    } else {
        for (int s = 0; s < n_scans; ++s) push(s, 0, 0, n_range(s));
        for (int s = 0; s < n_scans; ++s) push(s, 1, 0, n_az(s));
    }
    const int total = first;

    char *ws = static_cast<char *>(workspace);
    ScanDev *d_scans = reinterpret_cast<ScanDev *>(ws);
    Segment *d_segs = reinterpret_cast<Segment *>(ws + align256(sizeof(ScanDev) * (size_t)n_scans));
    int *d_cnt = reinterpret_cast<int *>(ws + align256(sizeof(ScanDev) * (size_t)n_scans) +
                                         align256(sizeof(Segment) * SEGS_PER_SCAN * (size_t)n_scans));
    cudaError_t e = cudaMemcpy(d_scans, hs, sizeof(ScanDev) * (size_t)n_scans, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_segs, hg, sizeof(Segment) * (size_t)ns, cudaMemcpyHostToDevice);
    free(hs);
    free(hg);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "batch_create: descriptor copy: %s", cudaGetErrorString(e));

    KernelFn fn = kernel_for(J);
    st = ensure_smem((const void *)fn, (size_t)smem, g_smem_done[j_index(J)], "batch_create");
    if (st != ROSAR_OK) return st;
    int dev = 0, n_sm = 0, occ = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BT_THREADS, (size_t)smem);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "batch_create: occupancy query: %s", cudaGetErrorString(e));
    if (occ < 1) return set_error(ROSAR_ERR_UNSUPPORTED, "batch_create: %d B of shared memory per CTA does not fit", smem);
    const int per_sm = (tn.ctas_per_sm > 0 && tn.ctas_per_sm < occ) ? tn.ctas_per_sm : occ;
    int grid = per_sm * n_sm;
    if (grid > total) grid = total;

    rosar_batch *b = new (std::nothrow) rosar_batch();
    if (!b) return set_error(ROSAR_ERR_INVALID_ARG, "batch_create: host allocation failed");
    b->counters = d_cnt;
    b->n_scans = n_scans;
    b->range_tiles = (int)total_range;
    b->az_tiles = (int)total_az;
    b->ctas = grid;
    b->smem = smem;
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(d_cnt, 0, sizeof(int) * (CNT_DONE + (size_t)n_scans), cs);
        fn<<<grid, BT_THREADS, smem, cs>>>(d_scans, d_segs, ns, total, d_cnt, tn.spin_limit, tn.debug_unmet_scan,
                                           tn.flags);
        e = cudaStreamEndCapture(cs, &b->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        delete b;
        return set_error(ROSAR_ERR_CUDA, "batch_create: graph capture: %s", cudaGetErrorString(e));
    }
    *batch = b;
    return ROSAR_OK;
}

rosar_status rosar_batch_launch(rosar_batch *batch, void *stream) {
    clear_error();
    if (!batch) return set_error(ROSAR_ERR_INVALID_ARG, "batch_launch: null batch");
    const cudaError_t e = cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "batch_launch: %s", cudaGetErrorString(e));
    return ROSAR_OK;
}

rosar_status rosar_batch_status(rosar_batch *batch, void *stream) {
    clear_error();
    if (!batch) return set_error(ROSAR_ERR_INVALID_ARG, "batch_status: null batch");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    int flags[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(flags, batch->counters, sizeof(flags), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_error(ROSAR_ERR_CUDA, "batch_status: %s", cudaGetErrorString(e));
    if (flags[CNT_ERR])
        return set_error(ROSAR_ERR_TIMEOUT, "batch: an azimuth tile of scan %d gave up waiting for its range tiles",
                         flags[CNT_ERR_SCAN]);
    return ROSAR_OK;
}

rosar_status rosar_batch_info(const rosar_batch *batch, int *range_tiles, int *azimuth_tiles, int *ctas,
                              int *smem_bytes) {
    clear_error();
    if (!batch) return set_error(ROSAR_ERR_INVALID_ARG, "batch_info: null batch");
    if (range_tiles) *range_tiles = batch->range_tiles;
    if (azimuth_tiles) *azimuth_tiles = batch->az_tiles;
    if (ctas) *ctas = batch->ctas;
    if (smem_bytes) *smem_bytes = batch->smem;
    return ROSAR_OK;
}

rosar_status rosar_batch_destroy(rosar_batch *batch) {
    clear_error();
    if (!batch) return ROSAR_OK;
    cudaError_t e1 = cudaGraphExecDestroy(batch->exec);
    cudaError_t e2 = cudaGraphDestroy(batch->graph);
    delete batch;
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return set_error(ROSAR_ERR_CUDA, "batch_destroy: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return ROSAR_OK;
}

}  // extern "C"
