// Flow kernel, FP32, with the tile and its halo staged in shared memory by
// the Blackwell tensor-memory-accelerator (TMA).  Same step as k_flow_pers
// (Eq. 3-15, push streaming with halfway bounce-back); only the way the
// populations reach the SM differs.
//
// A persistent CTA loops over 64 x TY tiles.  One thread stages the next
// tile -- rows y0-1 .. y0+TY, columns x0-4 .. x0+67 -- with two tensor copies
// (cp.async.bulk.tensor: one 3-D box over the nine population planes, one
// 2-D box of T), completion counted in bytes on an mbarrier, into the other
// of two shared-memory stages while all warps compute the current tile from
// theirs.  Rows outside the fluid arrive as zeros (never read: psi is 0
// there); at the periodic x edges the four wrapped halo columns are loaded
// by the threads after the copy lands.  Every thread then reads its sites
// and the psi halo ring from shared memory at constant offsets: no per-load
// address arithmetic and no prefetch registers.
//
// Requirements (checked by the launcher, which otherwise runs k_flow_pers):
// FP32 storage, nx a multiple of 64 (16-byte aligned box origins, tiles
// cover the columns exactly), walls at the bottom and top (not periodic in y).
//
// Waits are bounded (100 ms): a stage that does not complete in time sets
// ERRW_TIMEOUT, the block stops issuing copies, waits (again bounded) for the
// copy it has in flight, and leaves; the host then reports LBM_E_TIMEOUT.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm_fast.cuh"

namespace lbmgb {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// arrive, adding `bytes` to the transaction count this phase waits for
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for phase `parity`: false once 100 ms (or 2^20 polls) have
// passed without it
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;  // the usual case: no timer read
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 20); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > 100000000ull) break;
    }
    return false;
}
// global -> shared tensor copies of one box (origin in elements, x first)
__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(float *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

constexpr int TMA_TX = 64;                    // tile columns
constexpr int TMA_HX = 4;                     // staged halo columns on each side (16 bytes)
constexpr int TMA_SC = TMA_TX + 2 * TMA_HX;   // staged columns per row
constexpr int TMA_ARR = 10;                   // nine population planes and T

// Stage layout (floats): the population box [9][SR][SC] at 0, the T box
// [SR][SC] at a 128-byte aligned offset (TMA destinations need it), the
// stage padded to 128 bytes.
__host__ __device__ constexpr int tma_round32(int n) { return (n + 31) / 32 * 32; }
template <int BY, int RY>
__host__ __device__ constexpr int tma_t_offset() { return tma_round32(9 * (BY * RY + 2) * TMA_SC); }
template <int BY, int RY>
__host__ __device__ constexpr int tma_stage_floats() { return tma_round32(tma_t_offset<BY, RY>() + (BY * RY + 2) * TMA_SC); }

template <int BY, int RY, int MINB>
__global__ void __launch_bounds__(TMA_TX * BY, MINB)
k_flow_tma(const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_t, const FParams p,
           int tiles_x, int ntiles, const float *__restrict__ fin, float *__restrict__ fout,
           const float *__restrict__ Tin, float *__restrict__ rho_o, float *__restrict__ ux_o,
           float *__restrict__ uy_o, const double *__restrict__ cw, double *__restrict__ part,
           unsigned *__restrict__ err) {
    constexpr int BX = TMA_TX, TY = BY * RY, SR = TY + 2, SW = BX + 2, NT = BX * BY, SC = TMA_SC;
    constexpr int STAGE = tma_stage_floats<BY, RY>(), TOFF = tma_t_offset<BY, RY>();
    constexpr uint32_t BYTES = 10u * SR * SC * 4u;  // both boxes, out-of-range elements included
    constexpr int RING = 2 * SW + 2 * TY;
    static_assert(RING <= NT, "one ring site per thread");
    extern __shared__ __align__(128) float stg_raw[];  // two stages (+128 bytes of slack)
    float *const stg = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(stg_raw) + 127) & ~uintptr_t(127));
    __shared__ float s_psi[SR * SW];
    __shared__ float s_red[2][NT / 32];
    __shared__ __align__(8) uint64_t bar[2];

    const int nx = p.nx, nf = p.nf;
    const size_t plane = (size_t)nf * nx;
    float *oplane[9];
    #pragma unroll
    for (int i = 0; i < 9; i++) oplane[i] = fout + i * plane;
    const float *Tfl = Tin + (size_t)p.ns * nx;  // first fluid row of T
    constexpr bool py = false;  // the launcher takes walled domains only
    const bool frozen = (p.flags & FLAG_FROZEN_FLOW) != 0;
    const bool outflow = p.top_mode == TOP_OUTFLOW;
    const int tid = threadIdx.y * BX + threadIdx.x;
    const float rho0 = p.rho_shift;
    const float tsat = p.T_sat;
    unsigned errbits = 0;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();  // the initialised barriers are visible to the copy engine
    }
    __syncthreads();

    // Thread 0: stage tile (txt, tyt) into stage s (two tensor copies).
    auto stage_tile = [&](int txt, int tyt, int s) {
        float *dst = stg + s * STAGE;
        fence_proxy_async();  // this block's earlier reads of stage s come first
        mbar_arrive_expect_tx(&bar[s], BYTES + p.tx_pad);
        tma_load_3d(dst, &map_f, txt * BX - TMA_HX, tyt * TY - 1, 0, &bar[s]);
        tma_load_2d(dst + TOFF, &map_t, txt * BX - TMA_HX, p.ns + tyt * TY - 1, &bar[s]);
    };
    // All threads: the four wrapped halo columns of an edge tile, from the
    // far end of each row (the box read zeros there)
    auto wrap_columns = [&](float *st, int x0, int y0) {
        const bool left = x0 == 0, right = x0 + BX == nx;
        if (!left && !right) return;
        for (int q = tid; q < 2 * TMA_HX * SR * TMA_ARR; q += NT) {
            const int side = q / (TMA_HX * SR * TMA_ARR), r = q - side * (TMA_HX * SR * TMA_ARR);
            if (side == 0 ? !left : !right) continue;
            const int c = r % TMA_HX, hy = (r / TMA_HX) % SR, a = r / (TMA_HX * SR);
            const int y = y0 - 1 + hy;
            if (y < 0 || y >= nf) continue;
            const int xs = side == 0 ? nx - TMA_HX + c : c;
            const float v = (a < 9 ? fin + a * plane : Tfl)[(size_t)y * nx + xs];
            const int col = side == 0 ? c : TMA_HX + BX + c;
            (a < 9 ? st + (a * SR + hy) * SC : st + TOFF + hy * SC)[col] = v;
        }
        __syncthreads();
    };

    float g[RY][9];
    float dd[RY];
    float mass = 0.0f, nvap = 0.0f;
    const int gdx = (int)gridDim.x % tiles_x, gdy = (int)gridDim.x / tiles_x;
    int cxt = (int)blockIdx.x % tiles_x, cyt = (int)blockIdx.x / tiles_x;
    uint32_t phase = 0;  // bit s: parity of stage s's next completion
    int pending = -1;    // stage with copies in flight that nobody waited for
    int stalled = -1;    // stage whose wait ran out
    if (tid == 0 && (int)blockIdx.x < ntiles) stage_tile(cxt, cyt, 0);
    if ((int)blockIdx.x < ntiles) pending = 0;
    int k = 0;  // tiles done by this block
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, k++) {
        const int s = k & 1;
        const int x0 = cxt * BX, y0 = cyt * TY;
        int nxt = cxt + gdx, nyt = cyt + gdy;
        if (nxt >= tiles_x) { nxt -= tiles_x; nyt += 1; }
        const bool more = tile + (int)gridDim.x < ntiles;
        // the other stage was last read by the previous tile (its barrier passed)
        if (tid == 0 && more) stage_tile(nxt, nyt, s ^ 1);
        const bool ok = mbar_wait(&bar[s], (phase >> s) & 1u);
        phase ^= 1u << s;
        pending = more ? (s ^ 1) : -1;
        float *st = stg + s * STAGE;
        wrap_columns(st, x0, y0);  // every thread: its barrier must be uniform

        // ---- own sites: populations from the stage, density, psi ----
        #pragma unroll
        for (int r = 0; r < RY; r++) {
            const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
            const bool has = py || y0 + ly < nf;
            const float *q = st + (ly + 1) * SC + lx + TMA_HX;
            float psi = 0.0f;
            dd[r] = 0.0f;
            if (has) {
                #pragma unroll
                for (int i = 0; i < 9; i++) g[r][i] = q[i * SR * SC];
                const float d = ((g[r][0] + g[r][1]) + (g[r][2] + g[r][3])) + ((g[r][4] + g[r][5]) + (g[r][6] + g[r][7])) + g[r][8];
                dd[r] = d;
                if (!frozen) psi = psi_fast(p, d + rho0, st[TOFF + (ly + 1) * SC + lx + TMA_HX] + tsat, errbits);
            }
            s_psi[(ly + 1) * SW + lx + 1] = psi;
        }
        // ---- the psi halo ring, one site per thread ----
        if (!frozen && tid < RING) {
            int hx, hy;
            if (tid < SW) { hx = tid; hy = 0; }
            else if (tid < 2 * SW) { hx = tid - SW; hy = SR - 1; }
            else if (tid < 2 * SW + TY) { hx = 0; hy = 1 + (tid - 2 * SW); }
            else { hx = SW - 1; hy = 1 + (tid - 2 * SW - TY); }
            const int y = y0 - 1 + hy;
            float psi = 0.0f;
            if (py || (y >= 0 && y < nf)) {
                const float *q = st + hy * SC + hx + TMA_HX - 1;
                float f9[9];
                #pragma unroll
                for (int i = 0; i < 9; i++) f9[i] = q[i * SR * SC];
                const float d = ((f9[0] + f9[1]) + (f9[2] + f9[3])) + ((f9[4] + f9[5]) + (f9[6] + f9[7])) + f9[8];
                psi = psi_fast(p, d + rho0, st[TOFF + hy * SC + hx + TMA_HX - 1] + tsat, errbits);
            }
            s_psi[hy * SW + hx] = psi;
        }
        if (__syncthreads_or(!ok)) {  // a stage never completed: stop cleanly
            errbits |= ERRW_TIMEOUT;
            stalled = s;
            break;
        }

        // ---- collide and push (tiles that touch no boundary skip the wall terms) ----
        auto collide = [&](auto edge_tag) {
            constexpr bool E = decltype(edge_tag)::value;
            #pragma unroll
            for (int r = 0; r < RY; r++) {
                const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
                const int x = x0 + lx, y = y0 + ly;
                if (E && y >= nf) continue;
                const int ks = y * nx + x;
                PopDither dz{1u};
                const float d = dd[r];
                const float rho = d + rho0;
                if (!(fabsf(rho) < 1e30f)) errbits |= ERRW_NONFINITE_RHO;
                mass += rho;
                nvap += (rho < p.vap_threshold) ? 1.0f : 0.0f;
                if (frozen) {
                    #pragma unroll
                    for (int i = 0; i < 9; i++) oplane[i][ks] = g[r][i];
                    rho_o[ks] = rho;
                    ux_o[ks] = 0.0f;
                    uy_o[ks] = 0.0f;
                    continue;
                }
                flow_site<float, E>(p, g[r], d, rho, s_psi + (ly + 1) * SW + (lx + 1), SW, x, y, ks, py, outflow, cw,
                                    oplane, rho_o, ux_o, uy_o, dz);
            }
        };
        if (x0 == 0 || x0 + BX >= nx || y0 == 0 || y0 + TY >= nf) collide(std::true_type{});
        else collide(std::false_type{});
        __syncthreads();  // s_psi and this stage are rewritten
        cxt = nxt; cyt = nyt;
    }
    if (tid == 0) {
        // only after a timeout: let the copies into the other stage, and any
        // still owed to the stage whose wait ran out, land before the block's
        // shared memory is released (each wait bounded; the stalled stage's
        // parity bit was already flipped at its wait)
        if (pending >= 0) mbar_wait(&bar[pending], (phase >> pending) & 1u);
        if (stalled >= 0) mbar_wait(&bar[stalled], ((phase >> stalled) & 1u) ^ 1u);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mass += __shfl_down_sync(0xffffffffu, mass, o);
        nvap += __shfl_down_sync(0xffffffffu, nvap, o);
    }
    if ((tid & 31) == 0) { s_red[0][tid >> 5] = mass; s_red[1][tid >> 5] = nvap; }
    __syncthreads();
    if (tid == 0) {
        double m = 0.0, v = 0.0;
        #pragma unroll
        for (int w = 0; w < NT / 32; w++) { m += (double)s_red[0][w]; v += (double)s_red[1][w]; }
        part[2 * blockIdx.x] = m;
        part[2 * blockIdx.x + 1] = v;
    }
    if (errbits) atomicOr(err, errbits);
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link-time
// dependency on the driver library).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// Launch shape of k_flow_tma; shapes it cannot take (FP16 storage, nx not a
// multiple of 64, periodic in y) run the register-prefetch kernel of the
// same tile instead.
template <class P, int BY, int RY, int MINB>
struct FlowTmaShape {
    using Fallback = FlowPersShape<P, TMA_TX, BY, RY, (MINB < 2 ? MINB : 2)>;  // its registers need <= 2 blocks / SM
    static constexpr int SR = BY * RY + 2;
    static constexpr size_t smem_bytes = 2 * sizeof(float) * (size_t)tma_stage_floats<BY, RY>() + 128;
    static int grid_blocks;
    static bool eligible(const DevParams &p) {
        return sizeof(typename P::fst) == 4 && p.nx % TMA_TX == 0 && !(p.flags & FLAG_PERIODIC_Y) &&
               tensor_map_encoder() != nullptr;
    }
    static cudaError_t prepare() {
        cudaError_t e = Fallback::prepare();
        if (e != cudaSuccess || sizeof(typename P::fst) != 4) return e;
        int dev = 0, sms = 0, per = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_flow_tma<BY, RY, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_flow_tma<BY, RY, MINB>, TMA_TX * BY, smem_bytes);
        if (e != cudaSuccess) return e;
        grid_blocks = sms * (per > 0 ? per : 1);
        return cudaSuccess;
    }
    static int tiles(const DevParams &p) { return (p.nx / TMA_TX) * ((p.nf + BY * RY - 1) / (BY * RY)); }
    static int blocks(const DevParams &p) {
        if (!eligible(p)) return Fallback::blocks(p);
        const int t = tiles(p);
        return t < grid_blocks ? t : grid_blocks;
    }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        if (!eligible(p)) return Fallback::launch(p, b, s);
        // boxes: 72 columns x SR rows x 9 planes of the populations, 72 x SR of T
        // (all T rows, heater included: the tile's rows sit at ns + y)
        CUtensorMap mf, mt;
        const cuuint64_t nx = (cuuint64_t)p.nx, nf = (cuuint64_t)p.nf, nt = (cuuint64_t)p.nt;
        const cuuint64_t gd_f[3] = {nx, nf, 9}, gs_f[2] = {nx * 4, nx * nf * 4};
        const cuuint32_t bx_f[3] = {(cuuint32_t)TMA_SC, (cuuint32_t)SR, 9}, one[3] = {1, 1, 1};
        const cuuint64_t gd_t[2] = {nx, nt}, gs_t[1] = {nx * 4};
        const cuuint32_t bx_t[2] = {(cuuint32_t)TMA_SC, (cuuint32_t)SR};
        auto enc = tensor_map_encoder();
        CUresult r = enc(&mf, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(b.f_in), gd_f, gs_f, bx_f, one,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = enc(&mt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(b.T_in), gd_t, gs_t, bx_t, one,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        k_flow_tma<BY, RY, MINB><<<blocks(p), dim3(TMA_TX, BY), smem_bytes, s>>>(
            mf, mt, make_fparams(p), p.nx / TMA_TX, tiles(p), (const float *)b.f_in, (float *)b.f_out,
            (const float *)b.T_in, (float *)b.rho, (float *)b.ux, (float *)b.uy, b.cw, b.part, b.err);
        return cudaGetLastError();
    }
};
template <class P, int BY, int RY, int MINB>
int FlowTmaShape<P, BY, RY, MINB>::grid_blocks = 152;

}  // namespace lbmgb
