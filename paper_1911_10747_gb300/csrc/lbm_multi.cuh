// Multi-run kernels: one launch advances every run of a batch by one step
// of one kernel kind, over a work list of (run, tile).  The runs' descriptors
// (constants, buffers of both step parities, tile counts and the first tile
// of each run in the launch) sit in a device array sorted by first tile;
// each block takes a contiguous share of the list, finds the runs it touches
// by binary search, copies each one's constants to shared memory and runs
// the single-run kernels' persistent bodies over its tiles of that run
// (the flow kernel's and the paired heat kernel's, with their next-tile
// prefetch), and the diagnostics take one block per run.  A run stepped through a launch of its own with these
// kernels (the "multi" launch-shape variants) gives bit for bit what it
// gives inside any batch: the per-site arithmetic is the same, and the mass
// and vapour-count partials are written per tile, so their sums do not
// depend on how tiles were shared among blocks.
#pragma once
#include <type_traits>

#include "lbm_fast.cuh"

namespace lbmgb {

// flow tiles: 32 x 16 sites, 256 threads of 2 sites
constexpr int MR_FBX = 32, MR_FBY = 8, MR_FRY = 2, MR_FTX = MR_FBX, MR_FTY = MR_FBY * MR_FRY;
// heat tiles: the paired-column tiles, 64 x 48 cells with a 4-cell halo (56 x 40 outputs), 384 threads
constexpr int MR_HBY = 12, MR_HR = 4, MR_HTXO = 64 - 8, MR_HTYO = MR_HR * MR_HBY - 8;

struct MultiRun {
    FParams p;             // the run's constants
    StepBuffers b[2];      // its buffers, by the parity of its state
    int parity;            // parity of its state at phase 0 of the launch sequence
    int flow_tiles_x, flow_ntiles, flow_tile0;
    int heat_tiles_x, heat_ntiles, heat_tile0;
    int nblk;              // per-block partials its diagnostics sum (= flow tiles)
    unsigned magic;        // MULTI_MAGIC: set by fill_multi, checked by every block
    double inv_nx, inv_nfl;
};
constexpr unsigned MULTI_MAGIC = 0x4c424d52u;

// A block whose descriptor is not a filled one, or whose tile is not one of
// its run's, touches nothing: it sets ERRW_DESC in the launch's error word
// (the host reports LBM_E_STATE) and returns.
__device__ __forceinline__ bool multi_desc_ok(const MultiRun *r, int run, int nruns, int local, int ntiles) {
    return run >= 0 && run < nruns && r->magic == MULTI_MAGIC && local >= 0 && local < ntiles;
}

// index of the run whose tiles [tile0, tile0 + ntiles) hold `tile`
template <int KIND>
__device__ __forceinline__ int find_run(const MultiRun *__restrict__ runs, int nruns, int tile) {
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int t0 = KIND == 0 ? runs[mid].flow_tile0 : runs[mid].heat_tile0;
        if (t0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the run's constants into shared memory (all threads of the block)
__device__ __forceinline__ void copy_params(FParams &dst, const FParams &src, int tid, int nthreads) {
    const int *s = reinterpret_cast<const int *>(&src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int k = tid; k < (int)(sizeof(FParams) / sizeof(int)); k += nthreads) d[k] = s[k];
}

// Each block takes a contiguous share of the launch's (run, tile) list,
// [b T / G, (b + 1) T / G) for block b of G over T tiles, and runs the
// persistent single-run body over each run's part of it, prefetching the
// next tile of the same run while it computes the current one.
struct TileShare {
    int begin, end;
};
__device__ __forceinline__ TileShare tile_share(int total) {
    const long long g = gridDim.x, b = blockIdx.x;
    return {(int)(b * total / g), (int)((b + 1) * total / g)};
}

// Walk the block's share run by run: for each run it touches, check its
// descriptor, copy its constants to shared memory and call body(run, p,
// local_begin, local_end).  KIND 0: flow tiles, 1: heat tiles.
template <int KIND, class Body>
__device__ __forceinline__ void for_each_run_segment(const MultiRun *__restrict__ runs, int nruns, int total,
                                                     unsigned *__restrict__ errw, FParams &sp, int *s_run,
                                                     Body &&body) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const TileShare share = tile_share(total);
    int t = share.begin;
    while (t < share.end) {
        __syncthreads();  // the previous segment is done with sp and s_run
        if (tid == 0) {
            const int r = find_run<KIND>(runs, nruns, t);
            const MultiRun *q = runs + r;
            const int t0 = KIND == 0 ? q->flow_tile0 : q->heat_tile0, nt = KIND == 0 ? q->flow_ntiles : q->heat_ntiles;
            const bool ok = multi_desc_ok(q, r, nruns, t - t0, nt);
            s_run[0] = ok ? r : -1;
            s_run[1] = ok ? (share.end < t0 + nt ? share.end : t0 + nt) - t0 : 0;  // local end of the segment
            s_run[2] = ok ? t - t0 : 0;
            if (!ok) atomicOr(errw, (unsigned)ERRW_DESC);
        }
        __syncthreads();
        const int r = s_run[0];
        if (r < 0) return;  // (uniform: every thread read the same s_run)
        copy_params(sp, runs[r].p, tid, nth);
        const int lend = s_run[1], lbegin = s_run[2];
        __syncthreads();
        body(runs + r, sp, lbegin, lend);
        t = (KIND == 0 ? runs[r].flow_tile0 : runs[r].heat_tile0) + lend;
    }
}

// ---- flow: Eq. 1-15 and streaming over 32 x 16 tiles -------------------------
template <class P>
__global__ void __launch_bounds__(MR_FBX * MR_FBY, 2)
k_flow_multi(const MultiRun *__restrict__ runs, int nruns, int total, int phase, unsigned *__restrict__ errw) {
    using S = typename P::fst;
    __shared__ FParams sp;
    __shared__ int s_run[3];
    for_each_run_segment<0>(runs, nruns, total, errw, sp, s_run, [&](const MultiRun *run, const FParams &p, int lb, int le) {
        const StepBuffers &B = run->b[(run->parity + phase) & 1];
        flow_pers_body<P, MR_FBX, MR_FBY, MR_FRY, false, true>(
            p, run->flow_tiles_x, le, lb, 1, (const S *)B.f_in, (S *)B.f_out, (const typename P::tst *)B.T_in,
            (float *)B.rho, (float *)B.ux, (float *)B.uy, B.cw, B.part, B.err, B.step, 0);
    });
}

// ---- heat: one RK4 step over the paired-column tiles -------------------------
template <class P>
__global__ void __launch_bounds__(32 * MR_HBY, 1)
k_heat_multi(const MultiRun *__restrict__ runs, int nruns, int total, int phase, unsigned *__restrict__ errw) {
    __shared__ FParams sp;
    __shared__ int s_run[3];
    for_each_run_segment<1>(runs, nruns, total, errw, sp, s_run, [&](const MultiRun *run, const FParams &p, int lb, int le) {
        const StepBuffers &B = run->b[(run->parity + phase) & 1];
        // the general column wrap serves runs of any width (computed once per tile)
        heat_pair_body<P, MR_HBY, MR_HR, false>(p, run->heat_tiles_x, le, lb, 1, (const typename P::tst *)B.T_in,
                                                (typename P::tst *)B.T_out, (const float *)B.rho, (const float *)B.ux,
                                                (const float *)B.uy, B.step, B.err);
    });
}

// ---- diagnostics: one block per run ----------------------------------------
template <class P>
__global__ void __launch_bounds__(1024)
k_diag_multi(const MultiRun *__restrict__ runs, int phase, unsigned *__restrict__ errw) {
    const MultiRun *run = runs + blockIdx.x;
    if (run->magic != MULTI_MAGIC) {
        if (threadIdx.x == 0) atomicOr(errw, (unsigned)ERRW_DESC);
        return;
    }
    const int par = (run->parity + phase) & 1;
    const StepBuffers &B = run->b[par];
    diag_flat_body<P, 1024>(run->p, (const float *)B.T_out, (const float *)B.rho, B.part, run->nblk, B.q_top, B.series,
                            B.series_cap, B.last, B.step, run->inv_nx, run->inv_nfl);
}

// ---- host side ---------------------------------------------------------------
inline int multi_flow_tiles_x(const DevParams &p) { return (p.nx + MR_FTX - 1) / MR_FTX; }
inline int multi_flow_tiles(const DevParams &p) { return multi_flow_tiles_x(p) * ((p.nf + MR_FTY - 1) / MR_FTY); }
inline int multi_heat_tiles_x(const DevParams &p) { return (p.nx + MR_HTXO - 1) / MR_HTXO; }
inline int multi_heat_tiles(const DevParams &p) { return multi_heat_tiles_x(p) * ((p.nt + MR_HTYO - 1) / MR_HTYO); }

// Descriptor of a run whose first flow / heat tiles in the launch are
// flow_tile0 / heat_tile0; b0, b1: its buffers for state parity 0 and 1.
inline void fill_multi(const DevParams &p, const StepBuffers &b0, const StepBuffers &b1, int parity, int flow_tile0,
                       int heat_tile0, void *out) {
    MultiRun m{};
    m.p = make_fparams(p);
    m.b[0] = b0;
    m.b[1] = b1;
    m.parity = parity;
    m.flow_tiles_x = multi_flow_tiles_x(p);
    m.flow_ntiles = multi_flow_tiles(p);
    m.flow_tile0 = flow_tile0;
    m.heat_tiles_x = multi_heat_tiles_x(p);
    m.heat_ntiles = multi_heat_tiles(p);
    m.heat_tile0 = heat_tile0;
    m.nblk = m.flow_ntiles;
    m.magic = MULTI_MAGIC;
    m.inv_nx = 1.0 / (double)p.nx;
    m.inv_nfl = 1.0 / ((double)p.nx * (double)p.nf);
    *static_cast<MultiRun *>(out) = m;
}

template <class P>
struct MultiKernels {
    static int flow_grid, heat_grid;  // resident blocks on the device
    static cudaError_t prepare() {
        int dev = 0, sms = 0, pf = 0, ph = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, k_flow_multi<P>, MR_FBX * MR_FBY, 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ph, k_heat_multi<P>, 32 * MR_HBY, 0);
        if (e != cudaSuccess) return e;
        flow_grid = sms * (pf > 0 ? pf : 1);
        heat_grid = sms * (ph > 0 ? ph : 1);
        return cudaSuccess;
    }
    // kind 0 flow, 1 heat, 2 diagnostics; tiles = all runs' tiles of that
    // kind; errw: the launch's error word (ERRW_DESC)
    static cudaError_t launch(int kind, const void *desc, int nruns, int tiles, int phase, unsigned *errw,
                              cudaStream_t s) {
        const MultiRun *d = static_cast<const MultiRun *>(desc);
        if (kind == 0) {
            const int g = tiles < flow_grid ? tiles : flow_grid;
            k_flow_multi<P><<<g, dim3(MR_FBX, MR_FBY), 0, s>>>(d, nruns, tiles, phase, errw);
        } else if (kind == 1) {
            const int g = tiles < heat_grid ? tiles : heat_grid;
            k_heat_multi<P><<<g, dim3(32, MR_HBY), 0, s>>>(d, nruns, tiles, phase, errw);
        } else {
            k_diag_multi<P><<<nruns, 1024, 0, s>>>(d, phase, errw);
        }
        return cudaGetLastError();
    }
    // the same kernels as launch-shape variants of a single run (its own
    // descriptor, for the parity of its current state, is b.mdesc)
    static int flow_blocks(const DevParams &p) { return multi_flow_tiles(p); }
    static cudaError_t flow(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        return launch(0, b.mdesc, 1, multi_flow_tiles(p), 0, b.err, s);
    }
    static cudaError_t heat(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        return launch(1, b.mdesc, 1, multi_heat_tiles(p), 0, b.err, s);
    }
};
template <class P>
int MultiKernels<P>::flow_grid = 304;
template <class P>
int MultiKernels<P>::heat_grid = 152;

}  // namespace lbmgb
