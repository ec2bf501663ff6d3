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
#include <cstring>
#include <type_traits>

#include "lbm_fast.cuh"
#include "lbm_flowwave.cuh"

namespace lbmgb {

// Runs whose columns come in strips of 64 (FP32 storage, at least 128
// columns) take the row-wavefront flow kernel instead of the tiles: their
// work items are strips of 64 columns x MR_WSEG rows (units), the top
// MR_WTAIL rows in segments of MR_WSEG2 rows, each unit swept by one warp,
// with the unit's mass and vapour count as its partials.
constexpr int MR_WSEG = 16, MR_WSEG2 = 4, MR_WTAIL = 48, MR_WWPB = 4, MR_WMINB = 4;
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
    int nblk;              // partials its diagnostics sum (flow tiles, or units in wavefront mode)
    unsigned magic;        // MULTI_MAGIC: set by fill_multi, checked by every block
    double inv_nx, inv_nfl;
    // wavefront mode (wave_ok): 64-column strips x MR_WSEG-row units below
    // row wave_y2 (wave_nmain of them) and MR_WSEG2-row units above, the
    // first of them wave_unit0 in a launch that takes each run's units in
    // turn; packed constants; tensor maps of f, T and the wrapped halo boxes
    // for each state parity
    int wave_ok, wave_nstrips, wave_nunits, wave_unit0, wave_nmain, wave_y2;
    FlowWaveConsts K;
    CUtensorMap wave_map[2][4];
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
// ROWS: every run stages whole rows of the next tile (nx a multiple of 4 and
// at least 64; if periodic in y, at least one tile of rows): a single
// column wrap.  Otherwise the general column wrap serves runs of any width
// (computed once per tile).  Both give the same results.
template <class P, bool ROWS>
__global__ void __launch_bounds__(32 * MR_HBY, 1)
k_heat_multi(const MultiRun *__restrict__ runs, int nruns, int total, int phase, unsigned *__restrict__ errw) {
    __shared__ FParams sp;
    __shared__ int s_run[3];
    for_each_run_segment<1>(runs, nruns, total, errw, sp, s_run, [&](const MultiRun *run, const FParams &p, int lb, int le) {
        const StepBuffers &B = run->b[(run->parity + phase) & 1];
        heat_pair_body<P, MR_HBY, MR_HR, ROWS, ROWS>(p, run->heat_tiles_x, le, lb, 1, (const typename P::tst *)B.T_in,
                                                     (typename P::tst *)B.T_out, (const float *)B.rho,
                                                     (const float *)B.ux, (const float *)B.uy, B.step, B.err);
    });
}
inline bool multi_heat_rows(const DevParams &p) {
    return p.nx % 4 == 0 && p.nx >= 64 && (!(p.flags & FLAG_PERIODIC_Y) || p.nt >= MR_HR * MR_HBY);
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

// ---- flow, wavefront mode: one warp per unit (strip x segment of rows) ------
// Warps take units from the launch's counter (wq, zero between launches):
// first every run's MR_WSEG-row units, run by run, then every run's
// MR_WSEG2-row units of its top rows, so that the units taken last, while
// the other warps run out of work, are short.  A warp finds the run by
// binary search over the runs' first units in either phase, copies its
// constants to the warp's shared memory when the run changes, and sweeps
// the unit with the single-run wavefront kernel's body; the unit's mass and
// vapour count go to its own partial slot (the run's unit numbering, the
// same in every launch).  Launches of more than MR_WTAB runs take each
// run's units in turn (wave_unit0).
constexpr int MR_WTAB = 256;
// index of the last run whose first unit (u0) is at most u
__device__ __forceinline__ int find_run_wave(const MultiRun *__restrict__ runs, const int *s_u0, int nruns, int u) {
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int u0 = s_u0 ? s_u0[mid] : runs[mid].wave_unit0;
        if (u0 <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
template <int WPB, int MINB>
__global__ void __launch_bounds__(32 * WPB, MINB)
k_flow_wave_multi(const MultiRun *__restrict__ runs, int nruns, int total, int phase, unsigned *__restrict__ errw,
                  unsigned *__restrict__ wq) {
    extern __shared__ float4 fw_raw[];  // the warps' rings (+128 bytes of slack)
    __shared__ __align__(8) uint64_t fw_bar[WPB][FW_RS];
    __shared__ FParams s_p[WPB];
    __shared__ FlowWaveConsts s_k[WPB];
    __shared__ int s_u0[MR_WTAB], s_u1[MR_WTAB], s_ta;  // first units of the runs in either phase
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool phased = nruns <= MR_WTAB;
    if (phased && warp == 0) {
        // exclusive prefix sums of the runs' long and short unit counts
        int ca = 0, cb = 0;
        for (int base = 0; base < nruns; base += 32) {
            const int r = base + lane;
            const int a = r < nruns ? runs[r].wave_nmain : 0, c = r < nruns ? runs[r].wave_nunits - a : 0;
            int ia = a, ic = c;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int ta = __shfl_up_sync(FULL, ia, o), tc = __shfl_up_sync(FULL, ic, o);
                if (lane >= o) {
                    ia += ta;
                    ic += tc;
                }
            }
            if (r < nruns) {
                s_u0[r] = ca + ia - a;
                s_u1[r] = cb + ic - c;
            }
            ca += __shfl_sync(FULL, ia, 31);
            cb += __shfl_sync(FULL, ic, 31);
        }
        if (lane == 0) s_ta = ca;
    }
    __syncthreads();
    float *const ring = reinterpret_cast<float *>(fw_raw) + ((128u - (smem_u32(fw_raw) & 127u)) & 127u) / 4u +
                        warp * (FW_RS * FW_SLOT);
    FParams &p = s_p[warp];
    FlowWaveConsts &K = s_k[warp];
    WaveRing w;
    wave_ring_init(w, ring, fw_bar[warp], lane);
    int cur = -1;  // run whose constants are in p and K
    for (;;) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(wq, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= total) break;
        int r, lu;
        if (!phased) {
            r = find_run_wave(runs, nullptr, nruns, u);
            lu = u - runs[r].wave_unit0;
        } else if (u < s_ta) {
            r = find_run_wave(runs, s_u0, nruns, u);
            lu = u - s_u0[r];
        } else {
            r = find_run_wave(runs, s_u1, nruns, u - s_ta);
            lu = runs[r].wave_nmain + (u - s_ta - s_u1[r]);
        }
        const MultiRun *q = runs + r;
        if (!(r >= 0 && r < nruns && q->magic == MULTI_MAGIC && q->wave_ok && lu >= 0 && lu < q->wave_nunits)) {
            if (lane == 0) atomicOr(errw, (unsigned)ERRW_DESC);
            continue;
        }
        if (r != cur) {
            __syncwarp();  // the previous run's constants are no longer read
            const int *sp = reinterpret_cast<const int *>(&q->p);
            int *dp = reinterpret_cast<int *>(&p);
            for (int k = lane; k < (int)(sizeof(FParams) / sizeof(int)); k += 32) dp[k] = sp[k];
            const int *sk = reinterpret_cast<const int *>(&q->K);
            int *dk = reinterpret_cast<int *>(&K);
            for (int k = lane; k < (int)(sizeof(FlowWaveConsts) / sizeof(int)); k += 32) dk[k] = sk[k];
            __syncwarp();
            cur = r;
        }
        const int par = (q->parity + phase) & 1;
        const StepBuffers &B = q->b[par];
        const size_t plane = (size_t)p.nf * p.nx;
        float *op[9];
        #pragma unroll
        for (int i = 0; i < 9; i++) op[i] = (float *)B.f_out + i * plane;
        WaveUnits wu;
        wu.nstrips = q->wave_nstrips;
        wu.seg = MR_WSEG;
        wu.nmain = q->wave_nmain;
        wu.y2 = q->wave_y2;
        wu.seg2 = MR_WSEG2;
        wu.nunits = q->wave_nunits;
        int strip, ys, ye;
        wu.unit(lu, p.nf, strip, ys, ye);
        float mass = 0.0f, nvap = 0.0f;
        unsigned errbits = 0;
        wave_unit(p, K, &q->wave_map[par][0], &q->wave_map[par][1], &q->wave_map[par][2], &q->wave_map[par][3],
                  strip * FW_W, ys, ye, op, (float *)B.rho, (float *)B.ux, (float *)B.uy, B.cw, w, lane, mass, nvap,
                  errbits);
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mass += __shfl_down_sync(FULL, mass, o);
            nvap += __shfl_down_sync(FULL, nvap, o);
        }
        if (lane == 0) {
            B.part[2 * lu] = (double)mass;
            B.part[2 * lu + 1] = (double)nvap;
        }
        if (w.failed) errbits |= ERRW_TIMEOUT;
        if (errbits) atomicOr(B.err, errbits);
        if (w.failed) break;
    }
    if (w.failed) wave_ring_drain(w);
    if (lane == 0) {
        // the last warp of the launch to finish leaves the counter at zero
        __threadfence();
        const unsigned done = atomicAdd(wq + 1, 1u);
        if (done == gridDim.x * WPB - 1) {
            wq[0] = 0u;
            wq[1] = 0u;
        }
    }
}

// ---- host side ---------------------------------------------------------------
inline int multi_flow_tiles_x(const DevParams &p) { return (p.nx + MR_FTX - 1) / MR_FTX; }
inline int multi_flow_tiles(const DevParams &p) { return multi_flow_tiles_x(p) * ((p.nf + MR_FTY - 1) / MR_FTY); }
inline int multi_heat_tiles_x(const DevParams &p) { return (p.nx + MR_HTXO - 1) / MR_HTXO; }
inline int multi_heat_tiles(const DevParams &p) { return multi_heat_tiles_x(p) * ((p.nt + MR_HTYO - 1) / MR_HTYO); }

// wavefront mode: FP32 storage and whole 64-column strips (at least two)
template <class P>
inline int multi_wave_ok(const DevParams &p) {
    return sizeof(typename P::fst) == 4 && p.nx % FW_W == 0 && p.nx >= 2 * FW_W && !(p.flags & FLAG_FROZEN_FLOW) &&
           tensor_map_encoder() != nullptr;
}
inline int multi_wave_y2(const DevParams &p) { return p.nf > MR_WTAIL ? p.nf - MR_WTAIL : 0; }
inline int multi_wave_nmain(const DevParams &p) { return (p.nx / FW_W) * ((multi_wave_y2(p) + MR_WSEG - 1) / MR_WSEG); }
inline int multi_wave_units(const DevParams &p) {
    return multi_wave_nmain(p) + (p.nx / FW_W) * ((p.nf - multi_wave_y2(p) + MR_WSEG2 - 1) / MR_WSEG2);
}
// flow work items of a run: tiles, or wavefront units (mode bit 0)
template <class P>
inline int multi_flow_items(const DevParams &p, int mode) {
    return (mode & 1) && multi_wave_ok<P>(p) ? multi_wave_units(p) : multi_flow_tiles(p);
}
// the run's launch mode: bit 0 wavefront flow, bit 1 whole-row heat staging
template <class P>
inline int multi_mode(const DevParams &p) {
    return (multi_wave_ok<P>(p) ? 1 : 0) | (multi_heat_rows(p) ? 2 : 0);
}

// the tensor maps of the wavefront flow (see FlowWaveShape::launch)
inline bool wave_maps(const DevParams &p, const StepBuffers &b, CUtensorMap *m) {
    const cuuint64_t nxu = (cuuint64_t)p.nx, nfu = (cuuint64_t)p.nf, ntu = (cuuint64_t)p.nt;
    const cuuint64_t gd_f[3] = {nxu, nfu, 9}, gs_f[2] = {nxu * 4, nxu * nfu * 4};
    const cuuint64_t gd_t[2] = {nxu, ntu}, gs_t[1] = {nxu * 4};
    const cuuint32_t bx_f[3] = {(cuuint32_t)FW_SC, 1, 9}, bx_t[2] = {(cuuint32_t)FW_SC, 1};
    const cuuint32_t bs_f[3] = {(cuuint32_t)FW_H, 1, 9}, bs_t[2] = {(cuuint32_t)FW_H, 1}, one[3] = {1, 1, 1};
    auto enc = tensor_map_encoder();
    auto make = [&](CUtensorMap *t, int rank, const void *base, const cuuint64_t *gd, const cuuint64_t *gs,
                    const cuuint32_t *bx) {
        return enc(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void *>(base), gd, gs, bx, one,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    return make(&m[0], 3, b.f_in, gd_f, gs_f, bx_f) && make(&m[1], 2, b.T_in, gd_t, gs_t, bx_t) &&
           make(&m[2], 3, b.f_in, gd_f, gs_f, bs_f) && make(&m[3], 2, b.T_in, gd_t, gs_t, bs_t);
}

// Descriptor of a run whose first flow items (tiles, or units in mode 1) and
// heat tiles in the launch are flow0 / heat_tile0; b0, b1: its buffers for
// state parity 0 and 1.  The wavefront fields are filled whenever the run
// can take that mode, so that a run's own descriptor serves both
// single-run multi variants.
template <class P>
inline void fill_multi(const DevParams &p, const StepBuffers &b0, const StepBuffers &b1, int parity, int mode,
                       int flow0, int heat_tile0, void *out) {
    // built in an aligned local and copied: `out` (a byte buffer) need not
    // have the descriptor's 64-byte alignment
    MultiRun md{};
    MultiRun *m = &md;
    m->p = make_fparams(p);
    m->b[0] = b0;
    m->b[1] = b1;
    m->parity = parity;
    m->flow_tiles_x = multi_flow_tiles_x(p);
    m->flow_ntiles = multi_flow_tiles(p);
    m->heat_tiles_x = multi_heat_tiles_x(p);
    m->heat_ntiles = multi_heat_tiles(p);
    m->heat_tile0 = heat_tile0;
    m->wave_ok = multi_wave_ok<P>(p);
    if (m->wave_ok) {
        m->wave_nstrips = p.nx / FW_W;
        m->wave_nunits = multi_wave_units(p);
        m->wave_nmain = multi_wave_nmain(p);
        m->wave_y2 = multi_wave_y2(p);
        m->K = make_flowwave_consts(m->p);
        // the copies read the state parity's input buffers: f_in of b0 is the
        // input of a run whose state is in parity 0
        if (!wave_maps(p, b0, m->wave_map[0]) || !wave_maps(p, b1, m->wave_map[1])) m->wave_ok = 0;
    }
    const bool wave = (mode & 1) && m->wave_ok;
    m->flow_tile0 = wave ? 0 : flow0;
    m->wave_unit0 = wave ? flow0 : 0;
    m->nblk = wave ? m->wave_nunits : m->flow_ntiles;
    m->magic = MULTI_MAGIC;
    m->inv_nx = 1.0 / (double)p.nx;
    m->inv_nfl = 1.0 / ((double)p.nx * (double)p.nf);
    std::memcpy(out, &md, sizeof md);
}

template <class P>
struct MultiKernels {
    static int flow_grid, heat_grid, wave_grid;  // resident blocks on the device
    static constexpr size_t wave_smem = (size_t)MR_WWPB * FW_RS * FW_SLOT * sizeof(float) + 128;
    static cudaError_t prepare() {
        int dev = 0, sms = 0, pf = 0, ph = 0, pw = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, k_flow_multi<P>, MR_FBX * MR_FBY, 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ph, k_heat_multi<P, false>, 32 * MR_HBY, 0);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_flow_wave_multi<MR_WWPB, MR_WMINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)wave_smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pw, k_flow_wave_multi<MR_WWPB, MR_WMINB>, 32 * MR_WWPB,
                                                              wave_smem);
        if (e != cudaSuccess) return e;
        flow_grid = sms * (pf > 0 ? pf : 1);
        heat_grid = sms * (ph > 0 ? ph : 1);
        wave_grid = sms * (pw > 0 ? pw : 1);
        return cudaSuccess;
    }
    // kind 0 flow (tiles), 1 heat, 2 diagnostics, 3 flow (wavefront units),
    // 4 heat (whole-row staging);
    // items = all runs' work items of that kind; errw: the launch's error
    // word (ERRW_DESC); wq: the wavefront launches' work counter
    static cudaError_t launch(int kind, const void *desc, int nruns, int tiles, int phase, unsigned *errw,
                              unsigned *wq, cudaStream_t s) {
        const MultiRun *d = static_cast<const MultiRun *>(desc);
        if (kind == 3) {
            const int need = (tiles + MR_WWPB - 1) / MR_WWPB;
            const int g = need < wave_grid ? need : wave_grid;
            k_flow_wave_multi<MR_WWPB, MR_WMINB><<<g, 32 * MR_WWPB, wave_smem, s>>>(d, nruns, tiles, phase, errw, wq);
        } else if (kind == 0) {
            const int g = tiles < flow_grid ? tiles : flow_grid;
            k_flow_multi<P><<<g, dim3(MR_FBX, MR_FBY), 0, s>>>(d, nruns, tiles, phase, errw);
        } else if (kind == 1 || kind == 4) {
            const int g = tiles < heat_grid ? tiles : heat_grid;
            auto k = kind == 4 ? k_heat_multi<P, true> : k_heat_multi<P, false>;
            k<<<g, dim3(32, MR_HBY), 0, s>>>(d, nruns, tiles, phase, errw);
        } else {
            k_diag_multi<P><<<nruns, 1024, 0, s>>>(d, phase, errw);
        }
        return cudaGetLastError();
    }
    // the same kernels as launch-shape variants of a single run (its own
    // descriptor, for the parity of its current state, is b.mdesc)
    static int flow_blocks(const DevParams &p) { return multi_flow_tiles(p); }
    static cudaError_t flow(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        return launch(0, b.mdesc, 1, multi_flow_tiles(p), 0, b.err, b.wq, s);
    }
    static cudaError_t heat(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        return launch(multi_heat_rows(p) ? 4 : 1, b.mdesc, 1, multi_heat_tiles(p), 0, b.err, b.wq, s);
    }
    // the wavefront flow, for runs that can take it (else the tiles)
    static int wave_blocks(const DevParams &p) { return multi_flow_items<P>(p, 1); }
    static cudaError_t wave(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        if (!multi_wave_ok<P>(p)) return flow(p, b, s);
        return launch(3, b.mdesc, 1, multi_wave_units(p), 0, b.err, b.wq, s);
    }
};
template <class P>
int MultiKernels<P>::flow_grid = 304;
template <class P>
int MultiKernels<P>::heat_grid = 152;
template <class P>
int MultiKernels<P>::wave_grid = 456;

}  // namespace lbmgb
