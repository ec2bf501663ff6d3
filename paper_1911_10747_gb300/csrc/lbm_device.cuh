// Device kernels of one boiling time step (arXiv:1911.10747), templated on
// the precision policy.  Included by lbm_fp64.cu (compiled without FMA
// contraction, so the FP64 path rounds like a plain evaluation of the
// formulas) and lbm_fp32.cu (FP32 arithmetic, FP32 or FP16 population
// storage).
//
// Data layout in HBM (all row-major, x fastest, no padding):
//   populations  f[9][nf][nx]   two buffers (read f_in, push-write f_out)
//   temperature  T[nt][nx]      two buffers, rows 0..ns-1 heater, ns.. fluid
//   moments      rho, ux, uy [nf][nx] of the current step (read by the heat kernel)
// Shifted policies store g_i = f_i - w_i rho0 and theta = T - T_sat.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbm_launch.h"

namespace lbmgb {

// ---- D2Q9 velocity set (Eq. 2) and weights --------------------------------
__host__ __device__ constexpr int cx(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int cy(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }
// lattice weights (equilibrium, Eq. 27-28)
template <class R> __host__ __device__ constexpr R wl(int i) { return i == 0 ? R(4.0 / 9.0) : (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0)); }
// pseudopotential weights w(1) = 1/3, w(2) = 1/12 (Eq. 11)
template <class R> __host__ __device__ constexpr R wf(int i) { return i <= 4 ? R(1.0 / 3.0) : R(1.0 / 12.0); }

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp axis");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp diag");

// ---- precision policies ----------------------------------------------------
struct PolicyF64 { using real = double; using fst = double; using tst = double; static constexpr bool shifted = false; };
struct PolicyF32 { using real = float; using fst = float; using tst = float; static constexpr bool shifted = true; };
struct PolicyF16 { using real = float; using fst = __half; using tst = float; static constexpr bool shifted = true; };

template <class R, class S> __device__ __forceinline__ R ld_as(const S *p) { return R(__ldg(p)); }
template <> __device__ __forceinline__ float ld_as<float, __half>(const __half *p) { return __half2float(__ldg(p)); }
template <class S, class R> __device__ __forceinline__ void st_as(S *p, R v) { *p = S(v); }
template <> __device__ __forceinline__ void st_as<__half, float>(__half *p, float v) { *p = __float2half_rn(v); }

__device__ __forceinline__ double rsq(double v) { return sqrt(v); }
__device__ __forceinline__ float rsq(float v) { return sqrtf(v); }

__device__ __forceinline__ int wrapi(int v, int n) { v %= n; return v < 0 ? v + n : v; }
// v in [-n, 2n)
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// ---- counter-based uniform draw --------------------------------------------
// splitmix64 finaliser (Steele, Lea, Flood 2014) folded over the counters
// (seed, tag, step, index); U in [0, 1) from the top 53 bits.
__host__ __device__ __forceinline__ uint64_t smix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double draw_u01(uint64_t seed, uint64_t tag, uint64_t step, uint64_t idx) {
    const uint64_t gam = 0x9E3779B97F4A7C15ULL;
    uint64_t h = smix(seed + gam);
    h = smix((h ^ tag) + gam);
    h = smix((h ^ step) + gam);
    h = smix((h ^ idx) + gam);
    return double(h >> 11) * (1.0 / 9007199254740992.0);
}

// Bottom temperature of column x at step n (Sec. 3.2 and 4.1), FP64.
__device__ __forceinline__ double bottom_temperature(const DevParams &p, int x, long long n) {
    if (p.bc_mode == BCM_NOISE) {
        double U = draw_u01(p.seed, TAG_BOTTOM_NOISE, (uint64_t)n, (uint64_t)x);
        return p.T_b * (1.0 + p.bc_noise * (2.0 * U - 1.0));
    }
    if (p.bc_mode == BCM_SINE && n > p.sine_t0 && n < p.sine_t1) {
        double wl_ = p.sine_wl;
        double arg = (2.0 * 3.14159265358979323846) * ((double)x - wl_ / 4.0) / wl_;
        return p.T_b + p.sine_amp * sin(arg);
    }
    return p.T_b;
}

// ---- Peng-Robinson EOS (Eq. 13) and pseudopotential (Eq. 12) ---------------
template <class R>
__device__ __forceinline__ R eos_pressure(const DevParams &p, R rho, R T) {
    const R one = R(1.0), two = R(2.0);
    R t1 = rsq(T / R(p.Tc));
    R t2 = one + R(p.kappa) * (one - t1);
    R phi = t2 * t2;
    R br = R(p.b) * rho;
    R p1 = (rho * R(p.R) * T) / (one - br);
    R den = one + two * br - br * br;
    R p2 = (R(p.a) * phi * rho * rho) / den;
    return p1 - p2;
}

template <class R>
__device__ __forceinline__ R pseudo_psi(const DevParams &p, R rho, R T, unsigned &errbits) {
    R pr = eos_pressure<R>(p, rho, T);
    R arg = (R(2.0) * (pr - rho / R(3.0))) / R(p.G);
    if (!(arg >= R(0))) {
        errbits |= ERRW_PSI;
        return R(0);
    }
    return rsq(arg);
}

// ---- MRT collision with the improved forcing (Eq. 6, 7, 9, 10) -------------
// Unshifted form: f holds populations, d = rho.  Shifted form: f holds
// g_i = f_i - w_i rho0, d = rho - rho0; the moments of g differ from those of
// f only in m0, m1, m2 by rho0 (1, -2, 1), which the equilibrium absorbs.
template <class P>
__device__ __forceinline__ void mrt_collide(const DevParams &p, const typename P::real (&f)[9],
                                            typename P::real d, typename P::real rho,
                                            typename P::real psi, typename P::real Fx,
                                            typename P::real Fy, typename P::real Fmx,
                                            typename P::real Fmy, typename P::real &ux,
                                            typename P::real &uy, typename P::real (&fo)[9]) {
    using R = typename P::real;
    // m = M f (Eq. 6), columns summed in increasing order
    const R m0 = d;
    const R m1 = R(-4.0) * f[0] - f[1] - f[2] - f[3] - f[4] + R(2.0) * f[5] + R(2.0) * f[6] + R(2.0) * f[7] + R(2.0) * f[8];
    const R m2 = R(4.0) * f[0] - R(2.0) * f[1] - R(2.0) * f[2] - R(2.0) * f[3] - R(2.0) * f[4] + f[5] + f[6] + f[7] + f[8];
    const R m3 = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const R m4 = R(-2.0) * f[1] + R(2.0) * f[3] + f[5] - f[6] - f[7] + f[8];
    const R m5 = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    const R m6 = R(-2.0) * f[2] + R(2.0) * f[4] + f[5] + f[6] - f[7] - f[8];
    const R m7 = f[1] - f[2] + f[3] - f[4];
    const R m8 = f[5] - f[6] + f[7] - f[8];
    // Eq. 10: rho v = sum e f + F / 2
    ux = (m3 + R(0.5) * Fx) / rho;
    uy = (m5 + R(0.5) * Fy) / rho;
    // Eq. 5 then Eq. 4
    const R tau = R(p.tau_V) + ((rho - R(p.rho_V)) / R(p.drho_LV)) * R(p.dtau_LV);
    const R s78 = R(1.0) / tau;
    const R usq = ux * ux + uy * uy;
    R q0, q1, q2;  // first three equilibrium moments in the stored frame
    if constexpr (P::shifted) {
        q0 = d;
        q1 = R(-2.0) * d + R(3.0) * (rho * usq);
        q2 = d - R(3.0) * (rho * usq);
    } else {
        q0 = rho;
        q1 = rho * (R(-2.0) + R(3.0) * usq);
        q2 = rho * (R(1.0) - R(3.0) * usq);
    }
    const R q3 = rho * ux, q4 = -(rho * ux), q5 = rho * uy, q6 = -(rho * uy);
    const R q7 = rho * (ux * ux - uy * uy), q8 = rho * (ux * uy);
    // S-bar of Eq. 9 (entry 8 read as ux Fy + uy Fx; sign_eps on entry 2)
    const R uF = ux * Fx + uy * Fy;
    const R num = R(p.varpi12) * (Fmx * Fmx + Fmy * Fmy);
    const R psi2 = psi * psi;
    const R S1 = R(6.0) * uF + num / (psi2 * R(p.tau_e_m));
    const R S2 = R(-6.0) * uF + R(p.sign_eps) * (num / (psi2 * R(p.tau_s_m)));
    const R S3 = Fx, S4 = -Fx, S5 = Fy, S6 = -Fy;
    const R S7 = R(2.0) * (ux * Fx - uy * Fy);
    const R S8 = ux * Fy + uy * Fx;
    // Eq. 7: m* = m - s (m - m_eq) + (1 - s/2) S
    const R z0 = (m0 - R(p.s[0]) * (m0 - q0)) + R(p.hs[0]) * R(0.0);
    const R z1 = (m1 - R(p.s[1]) * (m1 - q1)) + R(p.hs[1]) * S1;
    const R z2 = (m2 - R(p.s[2]) * (m2 - q2)) + R(p.hs[2]) * S2;
    const R z3 = (m3 - R(p.s[3]) * (m3 - q3)) + R(p.hs[3]) * S3;
    const R z4 = (m4 - R(p.s[4]) * (m4 - q4)) + R(p.hs[4]) * S4;
    const R z5 = (m5 - R(p.s[5]) * (m5 - q5)) + R(p.hs[5]) * S5;
    const R z6 = (m6 - R(p.s[6]) * (m6 - q6)) + R(p.hs[6]) * S6;
    const R h78 = R(1.0) - R(0.5) * s78;
    const R z7 = (m7 - s78 * (m7 - q7)) + h78 * S7;
    const R z8 = (m8 - s78 * (m8 - q8)) + h78 * S8;
    // f* = M^T diag(1/|row k|^2) m*
    const R d0 = z0 * R(1.0 / 9.0), d1 = z1 * R(1.0 / 36.0), d2 = z2 * R(1.0 / 36.0);
    const R d3 = z3 * R(1.0 / 6.0), d4 = z4 * R(1.0 / 12.0), d5 = z5 * R(1.0 / 6.0);
    const R d6 = z6 * R(1.0 / 12.0), d7 = z7 * R(1.0 / 4.0), d8 = z8 * R(1.0 / 4.0);
    fo[0] = d0 - R(4.0) * d1 + R(4.0) * d2;
    fo[1] = d0 - d1 - R(2.0) * d2 + d3 - R(2.0) * d4 + d7;
    fo[2] = d0 - d1 - R(2.0) * d2 + d5 - R(2.0) * d6 - d7;
    fo[3] = d0 - d1 - R(2.0) * d2 - d3 + R(2.0) * d4 + d7;
    fo[4] = d0 - d1 - R(2.0) * d2 - d5 + R(2.0) * d6 - d7;
    fo[5] = d0 + R(2.0) * d1 + d2 + d3 + d4 + d5 + d6 + d8;
    fo[6] = d0 + R(2.0) * d1 + d2 - d3 - d4 + d5 + d6 - d8;
    fo[7] = d0 + R(2.0) * d1 + d2 - d3 - d4 - d5 - d6 + d8;
    fo[8] = d0 + R(2.0) * d1 + d2 + d3 + d4 - d5 - d6 - d8;
}

// Block-wide sum of two doubles (fixed order: deterministic for a given
// launch shape).  Result valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*sh)[NT / 32]) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int w = tid >> 5, l = tid & 31;
    if (l == 0) { sh[0][w] = a; sh[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        a = (l < NT / 32) ? sh[0][l] : 0.0;
        b = (l < NT / 32) ? sh[1][l] : 0.0;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// ============================================================================
// Flow kernel: one fused pass per step.
//   phase A: each thread pulls nothing -- populations are stored post-stream,
//            so the RY sites of a thread are read locally (coalesced along
//            x), summed to rho, and psi(rho, T) goes to shared memory; the
//            one-site halo ring of the tile is recomputed from its own
//            populations (they sit in L2: the neighbouring tiles read them
//            in the same wave).
//   phase B: forces from the psi tile (Eq. 11, 14, 15), velocity (Eq. 10),
//            MRT collision (Eq. 7), push-streaming (Eq. 8) with halfway
//            bounce-back into f_out, moments for the heat kernel, per-block
//            mass / vapour partial sums.
// Tile: TX = BX columns x TY = BY * RY rows; thread (tx, ty) owns rows
// ty, ty + BY, ... so each warp row reads 32 consecutive x.
// ============================================================================
template <class P, int BX, int BY, int RY>
__global__ void __launch_bounds__(BX *BY)
k_flow(const DevParams p, const typename P::fst *__restrict__ fin, typename P::fst *__restrict__ fout,
       const typename P::tst *__restrict__ Tin, typename P::real *__restrict__ rho_o,
       typename P::real *__restrict__ ux_o, typename P::real *__restrict__ uy_o,
       const double *__restrict__ cw, double *__restrict__ part, unsigned *__restrict__ err) {
    using R = typename P::real;
    using S = typename P::fst;
    constexpr int TX = BX, TY = BY * RY, SW = TX + 2, SH = TY + 2, NT = BX * BY;
    __shared__ R s_psi[SH * SW];
    __shared__ double s_red[2][NT / 32];

    const int nx = p.nx, nf = p.nf;
    const size_t plane = (size_t)nf * nx;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool frozen = (p.flags & FLAG_FROZEN_FLOW) != 0;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * BX + threadIdx.x;
    const R rho0 = P::shifted ? R(p.rho_shift) : R(0);
    const R tsat = P::shifted ? R(p.T_sat) : R(0);
    unsigned errbits = 0;

    R fl[RY][9];
    R dd[RY];
    R psv[RY];

    // ---- phase A: own sites ----
    #pragma unroll
    for (int r = 0; r < RY; r++) {
        const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
        const int x = wrapi(x0 + lx, nx);
        int y = y0 + ly;
        const bool has = py || y < nf;
        if (py) y = wrapi(y, nf);
        R psi = R(0);
        dd[r] = R(0);
        if (has) {
            const size_t k = (size_t)y * nx + x;
            #pragma unroll
            for (int i = 0; i < 9; i++) fl[r][i] = ld_as<R>(fin + i * plane + k);
            R d = fl[r][0];
            #pragma unroll
            for (int i = 1; i < 9; i++) d += fl[r][i];
            dd[r] = d;
            const R T = ld_as<R>(Tin + (size_t)(p.ns + y) * nx + x) + tsat;
            if (!frozen) psi = pseudo_psi<R>(p, d + rho0, T, errbits);
        } else {
            #pragma unroll
            for (int i = 0; i < 9; i++) fl[r][i] = R(0);
        }
        psv[r] = psi;
        s_psi[(ly + 1) * SW + lx + 1] = psi;
    }
    // ---- phase A: halo ring of the psi tile ----
    if (!frozen) {
        for (int k = tid; k < 2 * SW + 2 * TY; k += NT) {
            int hx, hy;
            if (k < SW) { hx = k; hy = 0; }
            else if (k < 2 * SW) { hx = k - SW; hy = SH - 1; }
            else if (k < 2 * SW + TY) { hx = 0; hy = 1 + (k - 2 * SW); }
            else { hx = SW - 1; hy = 1 + (k - 2 * SW - TY); }
            const int x = wrapi(x0 + hx - 1, nx);
            int y = y0 + hy - 1;
            bool valid = py || (y >= 0 && y < nf);
            if (py) y = wrapi(y, nf);
            R psi = R(0);
            if (valid) {
                const size_t kk = (size_t)y * nx + x;
                R d = ld_as<R>(fin + kk);
                #pragma unroll
                for (int i = 1; i < 9; i++) d += ld_as<R>(fin + i * plane + kk);
                const R T = ld_as<R>(Tin + (size_t)(p.ns + y) * nx + x) + tsat;
                psi = pseudo_psi<R>(p, d + rho0, T, errbits);
            }
            s_psi[hy * SW + hx] = psi;
        }
    }
    __syncthreads();

    // ---- phase B ----
    double mass = 0.0, nvap = 0.0;
    #pragma unroll
    for (int r = 0; r < RY; r++) {
        const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
        const int x = x0 + lx, y = y0 + ly;
        if (x >= nx || y >= nf) continue;
        const size_t k = (size_t)y * nx + x;
        const R d = dd[r];
        const R rho = d + rho0;
        if (!(rho == rho) || rho > R(1e30) || rho < R(-1e30)) errbits |= ERRW_NONFINITE_RHO;
        mass += (double)rho;
        nvap += ((double)rho < p.vap_threshold) ? 1.0 : 0.0;
        if (frozen) {
            #pragma unroll
            for (int i = 0; i < 9; i++) st_as(fout + i * plane + k, fl[r][i]);
            rho_o[k] = rho;
            ux_o[k] = R(0);
            uy_o[k] = R(0);
            continue;
        }
        const R psi = psv[r];
        // Eq. 11 over fluid neighbours; Eq. 14 (solid-neighbour reading) with
        // c_w of the wall site; top wall uses c_w_top.
        R sx = R(0), sy = R(0), ax = R(0), ay = R(0);
        #pragma unroll
        for (int i = 1; i < 9; i++) {
            const int yn = y + cy(i);
            if (py || (yn >= 0 && yn < nf)) {
                const R t = wf<R>(i) * s_psi[(ly + 1 + cy(i)) * SW + (lx + 1 + cx(i))];
                if (cx(i) > 0) sx = sx + t; else if (cx(i) < 0) sx = sx - t;
                if (cy(i) > 0) sy = sy + t; else if (cy(i) < 0) sy = sy - t;
            } else if (yn >= nf && p.top_mode == TOP_OUTFLOW) {
                // open top: psi continued with zero normal gradient (same row)
                const R t = wf<R>(i) * s_psi[(ly + 1) * SW + (lx + 1 + cx(i))];
                if (cx(i) > 0) sx = sx + t; else if (cx(i) < 0) sx = sx - t;
                if (cy(i) > 0) sy = sy + t; else if (cy(i) < 0) sy = sy - t;
            } else {
                const R c = (yn < 0) ? R(cw[wrap1(x + cx(i), nx)]) : R(p.c_w_top);
                const R t = wf<R>(i) * c;
                if (cx(i) > 0) ax = ax + t; else if (cx(i) < 0) ax = ax - t;
                if (cy(i) > 0) ay = ay + t; else if (cy(i) < 0) ay = ay - t;
            }
        }
        const R pre = R(-p.G) * psi;
        const R Fmx = pre * sx, Fmy = pre * sy;
        const R Fax = (-psi) * ax, Fay = (-psi) * ay;
        const R Fgy = -((rho - R(p.rho_mean)) * R(p.g));
        const R Fx = Fmx + Fax;
        const R Fy = (Fmy + Fay) + Fgy;
        R ux, uy, fo[9];
        mrt_collide<P>(p, fl[r], d, rho, psi, Fx, Fy, Fmx, Fmy, ux, uy, fo);
        rho_o[k] = rho;
        ux_o[k] = ux;
        uy_o[k] = uy;
        // Eq. 8 (push) with halfway bounce-back at the heater surface and
        // the top wall; OUTFLOW drops upward populations at the top row and
        // copies the downward ones into the top row (zero gradient).
        #pragma unroll
        for (int i = 0; i < 9; i++) {
            const int xd = wrap1(x + cx(i), nx);
            int yd = y + cy(i);
            if (py) {
                st_as(fout + i * plane + (size_t)wrap1(yd, nf) * nx + xd, fo[i]);
            } else if (yd >= 0 && yd < nf) {
                st_as(fout + i * plane + (size_t)yd * nx + xd, fo[i]);
                if (cy(i) < 0 && y == nf - 1 && p.top_mode == TOP_OUTFLOW)
                    st_as(fout + i * plane + (size_t)y * nx + xd, fo[i]);
            } else if (yd < 0 || p.top_mode == TOP_WALL) {
                st_as(fout + opp(i) * plane + k, fo[i]);
            }
        }
    }
    block_sum2<NT>(mass, nvap, s_red);
    if (tid == 0) {
        const int b = blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * b] = mass;
        part[2 * b + 1] = nvap;
    }
    if (errbits) atomicOr(err, errbits);
}

// ============================================================================
// Heat kernel: one RK4 step (Eq. 25-26) of Eq. 24 on a TX x TY tile, all
// four stages in shared memory.  The tile is loaded with a 4-cell halo (one
// cell per stage); stage k is evaluated on the tile grown by 3 - k cells, so
// the halo cells repeat the neighbours' arithmetic exactly.  rho and u are
// the moments of this step, frozen over the stages.
// Cell kinds: 0 outside, 1 solid (evolved), 2 fluid (evolved), 3 fixed
// (bottom Dirichlet row or top ghost row).
// ============================================================================
template <class R>
struct FdSmem {
    R *Tn, *A, *B, *acc, *lE, *lN, *lNE, *lNW, *ux, *uy, *div, *rcv, *d1, *pa, *den;
    unsigned char *kind;
};

template <int TX, int TY>
__host__ __device__ constexpr size_t fd_cells() { return (size_t)(TX + 8) * (TY + 8); }

template <class R, int TX, int TY>
__host__ __device__ constexpr size_t fd_smem_bytes() {
    return fd_cells<TX, TY>() * (14 * sizeof(R) + 1) + (size_t)TX * TY * sizeof(R) + 64;
}

template <class P, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_heat(const DevParams p, const typename P::tst *__restrict__ Tin, typename P::tst *__restrict__ Tout,
       const typename P::real *__restrict__ rho_i, const typename P::real *__restrict__ ux_i,
       const typename P::real *__restrict__ uy_i, const long long *__restrict__ stepp,
       unsigned *__restrict__ err) {
    using R = typename P::real;
    constexpr int H = 4, SW = TX + 2 * H, SH = TY + 2 * H, NC = SW * SH;
    extern __shared__ __align__(16) unsigned char smraw[];
    R *base = reinterpret_cast<R *>(smraw);
    R *sTn = base, *sA = base + NC, *sB = base + 2 * NC;
    R *lE = base + 3 * NC, *lN = base + 4 * NC, *lNE = base + 5 * NC, *lNW = base + 6 * NC;
    R *sUx = base + 7 * NC, *sUy = base + 8 * NC, *sDiv = base + 9 * NC, *sRcv = base + 10 * NC;
    R *sD1 = base + 11 * NC, *sPa = base + 12 * NC, *sDen = base + 13 * NC;
    R *sLam = sD1;  // lambda shares the d1 array until the links are built
    R *sAcc = base + 14 * NC;
    unsigned char *kind = reinterpret_cast<unsigned char *>(sAcc + TX * TY);

    const int nx = p.nx, nt = p.nt, ns = p.ns, nf = p.nf;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool iso = (p.flags & FLAG_ISOTHERMAL) != 0;
    const int x0 = blockIdx.x * TX, r0 = blockIdx.y * TY;
    const int tid = threadIdx.x;
    const long long n = *stepp;
    const R tsat = P::shifted ? R(p.T_sat) : R(0);
    unsigned errbits = 0;

    // ---- load: T, lambda, u, rho-dependent factors; cell kinds ----
    for (int c = tid; c < NC; c += NT) {
        const int hx = c % SW, hy = c / SW;
        const int x = wrapi(x0 + hx - H, nx);
        int row = r0 + hy - H;
        unsigned char kd;
        if (py) { row = wrapi(row, nt); kd = 2; }
        else if (row < 0 || row > nt) kd = 0;
        else if (row == 0 || row == nt) kd = 3;
        else kd = (row < ns) ? 1 : 2;
        R T = R(0), lam = R(0), ux = R(0), uy = R(0), rcv = R(1), rho = R(0);
        if (kd == 1) {
            T = ld_as<R>(Tin + (size_t)row * nx + x);
            lam = R(p.lambda_s);
            rcv = R(p.rho_c_s);
        } else if (kd == 2) {
            const size_t kf = (size_t)(row - ns) * nx + x;
            T = ld_as<R>(Tin + (size_t)row * nx + x);
            rho = rho_i[kf];
            ux = ux_i[kf];
            uy = uy_i[kf];
            lam = R(p.cv_chi) * rho;
            rcv = rho * R(p.c_v);
        } else if (kd == 3) {
            if (row == 0) {
                T = R(bottom_temperature(p, x, n) - (P::shifted ? p.T_sat : 0.0));
                // Model A: the wall row conducts like the first fluid row
                lam = (p.flags & FLAG_MODEL_A) ? R(p.cv_chi) * rho_i[x] : R(p.lambda_s);
            } else {
                T = P::shifted ? R(0) : R(p.T_sat);
                lam = R(p.cv_chi) * rho_i[(size_t)(nf - 1) * nx + x];
            }
        }
        sTn[c] = T; sA[c] = T; sB[c] = T;
        sLam[c] = lam; sUx[c] = ux; sUy[c] = uy; sRcv[c] = rcv;
        sDen[c] = rho;  // rho parked here until the factors are built
        kind[c] = kd;
    }
    __syncthreads();
    // ---- links (harmonic mean conductances), divergence, EOS factors ----
    for (int c = tid; c < NC; c += NT) {
        const int hx = c % SW, hy = c / SW;
        const R l0 = sLam[c];
        auto hm = [&](R la) -> R {
            const R s = l0 + la;
            return (s == R(0)) ? R(0) : (R(2.0) * (l0 * la)) / s;
        };
        lE[c] = (hx + 1 < SW) ? hm(sLam[c + 1]) : R(0);
        lN[c] = (hy + 1 < SH) ? hm(sLam[c + SW]) : R(0);
        lNE[c] = (hx + 1 < SW && hy + 1 < SH) ? hm(sLam[c + SW + 1]) : R(0);
        lNW[c] = (hx >= 1 && hy + 1 < SH) ? hm(sLam[c + SW - 1]) : R(0);
    }
    __syncthreads();
    for (int c = tid; c < NC; c += NT) {
        const int hx = c % SW, hy = c / SW;
        R dv = R(0), d1 = R(0), pa = R(0), den = R(1);
        if (kind[c] == 2 && hx >= 1 && hx < SW - 1 && hy >= 1 && hy < SH - 1) {
            // Eq. 27 on the frozen velocity: div u = 3 sum w e.u
            const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
            R dx = w1 * sUx[c + 1];
            dx = dx - w1 * sUx[c - 1];
            dx = dx + w2 * sUx[c + SW + 1];
            dx = dx - w2 * sUx[c + SW - 1];
            dx = dx - w2 * sUx[c - SW - 1];
            dx = dx + w2 * sUx[c - SW + 1];
            R dy = w1 * sUy[c + SW];
            dy = dy - w1 * sUy[c - SW];
            dy = dy + w2 * sUy[c + SW + 1];
            dy = dy + w2 * sUy[c + SW - 1];
            dy = dy - w2 * sUy[c - SW - 1];
            dy = dy - w2 * sUy[c - SW + 1];
            dv = R(3.0) * dx + R(3.0) * dy;
            // rho-only factors of (dp/dT)_rho (Eq. 13 differentiated)
            const R rho = sDen[c];
            const R br = R(p.b) * rho;
            den = R(1.0) + R(2.0) * br - br * br;
            d1 = (rho * R(p.R)) / (R(1.0) - br);
            pa = R(p.a) * R(p.kappa) * rho * rho;
        }
        sDiv[c] = dv;
        sD1[c] = d1;  // overwrites lambda: the links were built in the previous pass
        sPa[c] = pa;
        sDen[c] = den;
    }
    __syncthreads();

    // ---- four RK stages on shrinking regions ----
    if (!iso) {
        #pragma unroll 1
        for (int st = 0; st < 4; st++) {
            const int m = 1 + st;
            const int RW = SW - 2 * m, RH = SH - 2 * m;
            const R *Tk = (st == 0) ? sTn : ((st == 2) ? sB : sA);
            R *To = (st == 1) ? sB : sA;
            for (int q = tid; q < RW * RH; q += NT) {
                const int hx = m + q % RW, hy = m + q / RW;
                const int c = hy * SW + hx;
                const unsigned char kd = kind[c];
                if (kd != 1 && kd != 2) continue;
                const R T0 = Tk[c];
                const R T1 = Tk[c + 1], T2 = Tk[c + SW], T3 = Tk[c - 1], T4 = Tk[c - SW];
                const R T5 = Tk[c + SW + 1], T6 = Tk[c + SW - 1], T7 = Tk[c - SW - 1], T8 = Tk[c - SW + 1];
                const R w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
                // Eq. 28 with the link conductances
                R sD = w1 * (lE[c] * (T1 - T0));
                sD = sD + w1 * (lN[c] * (T2 - T0));
                sD = sD + w1 * (lE[c - 1] * (T3 - T0));
                sD = sD + w1 * (lN[c - SW] * (T4 - T0));
                sD = sD + w2 * (lNE[c] * (T5 - T0));
                sD = sD + w2 * (lNW[c] * (T6 - T0));
                sD = sD + w2 * (lNE[c - SW - 1] * (T7 - T0));
                sD = sD + w2 * (lNW[c - SW + 1] * (T8 - T0));
                const R D = R(6.0) * sD;
                R h;
                if (kd == 1) {
                    h = D / sRcv[c];
                } else {
                    // Eq. 27 gradient of T
                    R gx = w1 * T1;
                    gx = gx - w1 * T3;
                    gx = gx + w2 * T5;
                    gx = gx - w2 * T6;
                    gx = gx - w2 * T7;
                    gx = gx + w2 * T8;
                    R gy = w1 * T2;
                    gy = gy - w1 * T4;
                    gy = gy + w2 * T5;
                    gy = gy + w2 * T6;
                    gy = gy - w2 * T7;
                    gy = gy - w2 * T8;
                    gx = R(3.0) * gx;
                    gy = R(3.0) * gy;
                    const R rcv = sRcv[c];
                    const R adv = sUx[c] * gx + sUy[c] * gy;
                    const R Ta = T0 + tsat;  // absolute temperature
                    const R t1 = rsq(Ta / R(p.Tc));
                    const R t2 = R(1.0) + R(p.kappa) * (R(1.0) - t1);
                    const R dp = sD1[c] + (sPa[c] * t2) / (rsq(Ta * R(p.Tc)) * sDen[c]);
                    h = (-adv + D / rcv) - (((Ta / rcv) * dp) * sDiv[c]);
                }
                const bool in_tile = hx >= H && hx < H + TX && hy >= H && hy < H + TY;
                const int a = (hy - H) * TX + (hx - H);
                const R Tn = sTn[c];
                if (st == 0) {
                    if (in_tile) sAcc[a] = h;
                    To[c] = Tn + R(0.5) * h;
                } else if (st == 1) {
                    if (in_tile) sAcc[a] = sAcc[a] + R(2.0) * h;
                    To[c] = Tn + R(0.5) * h;
                } else if (st == 2) {
                    if (in_tile) sAcc[a] = sAcc[a] + R(2.0) * h;
                    To[c] = Tn + h;
                } else {
                    sAcc[a] = sAcc[a] + h;
                }
            }
            __syncthreads();
        }
    }
    // ---- write T^{n+1} of the tile (bottom row: the Dirichlet value used) ----
    for (int a = tid; a < TX * TY; a += NT) {
        const int tx = a % TX, ty = a / TX;
        const int x = x0 + tx, row = r0 + ty;
        if (x >= nx || row >= nt) continue;
        const int c = (ty + H) * SW + (tx + H);
        const unsigned char kd = kind[c];
        R v = sTn[c];
        if ((kd == 1 || kd == 2) && !iso) v = sTn[c] + sAcc[a] / R(6.0);
        if (!(v == v) || v > R(1e30) || v < R(-1e30)) errbits |= ERRW_NONFINITE_T;
        st_as(Tout + (size_t)row * nx + x, v);
    }
    if (errbits) atomicOr(err, errbits);
}

// ============================================================================
// Diagnostics kernel (one block): mass and vapour fraction from the flow
// kernel's per-block partials, heater-bottom flux (Eq. 36/39) and the local
// heater/fluid interface flux from T^{n+1}; appends to the series ring and
// advances the device step counter.  Fixed reduction order.
// ============================================================================
template <class P, int NT>
__global__ void __launch_bounds__(NT)
k_diag(const DevParams p, const typename P::tst *__restrict__ T, const typename P::real *__restrict__ rho,
       const double *__restrict__ part, int nblk, double *__restrict__ q_top, double *__restrict__ series,
       int cap, double *__restrict__ last, long long *__restrict__ stepp) {
    __shared__ double sh[2][NT / 32];
    const int nx = p.nx, ns = p.ns;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool model_a = (p.flags & FLAG_MODEL_A) != 0;  // no heater: wall flux for both
    const double toff = P::shifted ? p.T_sat : 0.0;
    double mass = 0.0, nvap = 0.0;
    for (int b = threadIdx.x; b < nblk; b += NT) {
        mass += part[2 * b];
        nvap += part[2 * b + 1];
    }
    block_sum2<NT>(mass, nvap, sh);
    __syncthreads();
    double qb = 0.0, qt = 0.0;
    for (int x = threadIdx.x; x < nx; x += NT) {
        if (ns >= 3 && !model_a && !py) {
            const double T0 = (double)T[x] + toff, T1 = (double)T[nx + x] + toff, T2 = (double)T[2 * nx + x] + toff;
            const double dTdy = ((4.0 * T1 - T2) - 3.0 * T0) / 2.0;
            qb += (-p.lambda_s) * dTdy;
        }
        if (ns >= 1 && !py) {
            const double lf1 = p.cv_chi * (double)rho[x], lf0 = model_a ? p.cv_chi * (double)rho[x] : p.lambda_s;
            const double lf = (2.0 * (lf0 * lf1)) / (lf0 + lf1);
            const double Tu = (double)T[(size_t)ns * nx + x] + toff;
            const double Td = (double)T[(size_t)(ns - 1) * nx + x] + toff;
            const double q = (-lf) * (Tu - Td);
            q_top[x] = q;
            qt += q;
        }
    }
    block_sum2<NT>(qb, qt, sh);
    if (threadIdx.x == 0) {
        const long long n = *stepp;
        const double nfl = (double)nx * (double)p.nf;
        double v[SERIES_WIDTH] = {qb / (double)nx, qt / (double)nx, nvap / nfl, mass};
        if (!(ns >= 3 && !model_a && !py)) v[0] = 0.0;
        if (!(ns >= 1 && !py)) v[1] = 0.0;
        if (model_a) v[0] = v[1];
        const long long slot = n % cap;
        #pragma unroll
        for (int k = 0; k < SERIES_WIDTH; k++) {
            series[slot * SERIES_WIDTH + k] = v[k];
            last[k] = v[k];
        }
        *stepp = n + 1;
    }
}

// ---- initial state (Sec. 3.1) ------------------------------------------------
template <class P>
__global__ void k_init_rho(const DevParams p, typename P::real *__restrict__ rho) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nfl = (size_t)p.nx * p.nf;
    if (k >= nfl) return;
    const int y = (int)(k / p.nx);
    const double base = (y < p.liquid_rows) ? p.rho_L : p.rho_V;
    const double U = draw_u01(p.seed, TAG_INIT_NOISE, 0, (uint64_t)k);
    rho[k] = (typename P::real)(base * (1.0 + p.init_noise * (2.0 * U - 1.0)));
}

// Sum of the initial densities in a fixed order: block b of nblk sums the
// contiguous sites [b chunk, (b + 1) chunk) into out[1 + b]; then one block
// sums out[1 .. nblk] into out[0].  The order depends only on the domain
// size, so the mean is the same on every call; the blocks spread over the
// device instead of one block reading the whole field.
template <class P, int NT>
__global__ void __launch_bounds__(NT) k_sum_rho_part(const DevParams p, const typename P::real *__restrict__ rho,
                                                     double *__restrict__ out, long long chunk) {
    __shared__ double sh[2][NT / 32];
    const long long nfl = (long long)p.nx * p.nf;
    const long long k0 = (long long)blockIdx.x * chunk, k1 = k0 + chunk < nfl ? k0 + chunk : nfl;
    double s = 0.0, z = 0.0;
    for (long long k = k0 + threadIdx.x; k < k1; k += NT) s += (double)rho[k];
    block_sum2<NT>(s, z, sh);
    if (threadIdx.x == 0) out[1 + blockIdx.x] = s;
}
template <int NT>
__global__ void __launch_bounds__(NT) k_sum_rho_final(double *__restrict__ out, int nblk) {
    __shared__ double sh[2][NT / 32];
    double s = 0.0, z = 0.0;
    for (int b = threadIdx.x; b < nblk; b += NT) s += out[1 + b];
    block_sum2<NT>(s, z, sh);
    if (threadIdx.x == 0) out[0] = s;
}

template <class P>
__global__ void k_init_state(const DevParams p, const typename P::real *__restrict__ rho,
                             typename P::fst *__restrict__ f, typename P::tst *__restrict__ T) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nfl = (size_t)p.nx * p.nf, ntl = (size_t)p.nx * p.nt;
    if (k < nfl) {
        const double r = (double)rho[k];
        #pragma unroll
        for (int i = 0; i < 9; i++) {
            const double v = P::shifted ? wl<double>(i) * (r - p.rho_shift) : wl<double>(i) * r;
            st_as(f + i * nfl + k, (typename P::real)v);
        }
    }
    if (k < ntl) st_as(T + k, (typename P::real)(P::shifted ? 0.0 : p.T_sat));
}

// ---- state import / field export (float64 at the ABI; float32 import too) --
// In: the ABI arrays' type (double, or float for lbm_set_state_f32); the
// shift to storage is taken in float64 either way, so a float32 array and
// the same values widened to float64 import to the same storage.
template <class P, class In = double>
__global__ void k_import(const DevParams p, const In *__restrict__ f64, const In *__restrict__ T64,
                         typename P::fst *__restrict__ f, typename P::tst *__restrict__ T) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nfl = (size_t)p.nx * p.nf, ntl = (size_t)p.nx * p.nt;
    if (f64 && k < nfl) {
        #pragma unroll
        for (int i = 0; i < 9; i++) {
            const double v = (double)f64[i * nfl + k];
            st_as(f + i * nfl + k, (typename P::real)(P::shifted ? v - wl<double>(i) * p.rho_shift : v));
        }
    }
    if (T64 && k < ntl) {
        const double v = (double)T64[k];
        st_as(T + k, (typename P::real)(P::shifted ? v - p.T_sat : v));
    }
}

template <class P>
__global__ void k_export(const DevParams p, const typename P::fst *__restrict__ f,
                         const typename P::tst *__restrict__ T, const typename P::real *__restrict__ rho,
                         const typename P::real *__restrict__ ux, const typename P::real *__restrict__ uy,
                         double *__restrict__ rho64, double *__restrict__ ux64, double *__restrict__ uy64,
                         double *__restrict__ T64, double *__restrict__ f64) {
    using R = typename P::real;
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nfl = (size_t)p.nx * p.nf, ntl = (size_t)p.nx * p.nt;
    if (k < nfl) {
        if (rho64) rho64[k] = (double)rho[k];
        if (ux64) ux64[k] = (double)ux[k];
        if (uy64) uy64[k] = (double)uy[k];
        if (f64) {
            #pragma unroll
            for (int i = 0; i < 9; i++) {
                const double v = (double)ld_as<R>(f + i * nfl + k);
                f64[i * nfl + k] = P::shifted ? v + wl<double>(i) * p.rho_shift : v;
            }
        }
    }
    if (T64 && k < ntl) T64[k] = (double)T[k] + (P::shifted ? p.T_sat : 0.0);
}

// ---- launchers -------------------------------------------------------------------
template <class P, int BX, int BY, int RY>
struct FlowShape {
    static dim3 grid(const DevParams &p) { return dim3((p.nx + BX - 1) / BX, (p.nf + BY * RY - 1) / (BY * RY)); }
    static int blocks(const DevParams &p) { dim3 g = grid(p); return (int)(g.x * g.y); }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        using R = typename P::real;
        k_flow<P, BX, BY, RY><<<grid(p), dim3(BX, BY), 0, s>>>(
            p, (const typename P::fst *)b.f_in, (typename P::fst *)b.f_out, (const typename P::tst *)b.T_in,
            (R *)b.rho, (R *)b.ux, (R *)b.uy, b.cw, b.part, b.err);
        return cudaGetLastError();
    }
};

template <class P, int TX, int TY, int NT>
struct HeatShape {
    static constexpr size_t smem = fd_smem_bytes<typename P::real, TX, TY>();
    // Opt in to more than 48 KB of dynamic shared memory (called once per
    // run at creation, outside any stream capture).
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(k_heat<P, TX, TY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        using R = typename P::real;
        dim3 g((p.nx + TX - 1) / TX, (p.nt + TY - 1) / TY);
        k_heat<P, TX, TY, NT><<<g, NT, smem, s>>>(p, (const typename P::tst *)b.T_in, (typename P::tst *)b.T_out,
                                                  (const R *)b.rho, (const R *)b.ux, (const R *)b.uy, b.step, b.err);
        return cudaGetLastError();
    }
};

template <class P, int NT>
cudaError_t launch_diag(const DevParams &p, const StepBuffers &b, int nblk, cudaStream_t s) {
    k_diag<P, NT><<<1, NT, 0, s>>>(p, (const typename P::tst *)b.T_out, (const typename P::real *)b.rho, b.part,
                                   nblk, b.q_top, b.series, b.series_cap, b.last, b.step);
    return cudaGetLastError();
}

template <class P>
cudaError_t launch_init(const DevParams &p, const StepBuffers &b, int phase, cudaStream_t s) {
    using R = typename P::real;
    const size_t nfl = (size_t)p.nx * p.nf, ntl = (size_t)p.nx * p.nt;
    if (phase == 0) {
        k_init_rho<P><<<(unsigned)((nfl + 255) / 256), 256, 0, s>>>(p, (R *)b.rho);
        // partial sums in scratch[1 ..] (the scratch holds 1024 doubles)
        long long chunk = 256 * 16;
        long long nblk = ((long long)nfl + chunk - 1) / chunk;
        if (nblk > 1023) {
            chunk = ((long long)nfl + 1022) / 1023;
            nblk = ((long long)nfl + chunk - 1) / chunk;
        }
        k_sum_rho_part<P, 256><<<(unsigned)nblk, 256, 0, s>>>(p, (const R *)b.rho, b.scratch, chunk);
        k_sum_rho_final<1024><<<1, 1024, 0, s>>>(b.scratch, (int)nblk);
    } else {
        const size_t n = nfl > ntl ? nfl : ntl;
        k_init_state<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, (const R *)b.rho, (typename P::fst *)b.f_out,
                                                                    (typename P::tst *)b.T_out);
        cudaMemsetAsync(b.ux, 0, nfl * sizeof(R), s);
        cudaMemsetAsync(b.uy, 0, nfl * sizeof(R), s);
    }
    return cudaGetLastError();
}

template <class P>
cudaError_t launch_import(const DevParams &p, const double *f, const double *T, const StepBuffers &b, cudaStream_t s) {
    const size_t n = (size_t)p.nx * p.nt;
    k_import<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, f, T, (typename P::fst *)b.f_out, (typename P::tst *)b.T_out);
    return cudaGetLastError();
}
template <class P>
cudaError_t launch_import32(const DevParams &p, const float *f, const float *T, const StepBuffers &b, cudaStream_t s) {
    const size_t n = (size_t)p.nx * p.nt;
    k_import<P, float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, f, T, (typename P::fst *)b.f_out,
                                                                    (typename P::tst *)b.T_out);
    return cudaGetLastError();
}

template <class P>
cudaError_t launch_export(const DevParams &p, const StepBuffers &b, double *rho, double *ux, double *uy, double *T,
                          double *f, cudaStream_t s) {
    using R = typename P::real;
    const size_t n = (size_t)p.nx * p.nt;
    k_export<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        p, (const typename P::fst *)b.f_in, (const typename P::tst *)b.T_in, (const R *)b.rho, (const R *)b.ux,
        (const R *)b.uy, rho, ux, uy, T, f);
    return cudaGetLastError();
}

}  // namespace lbmgb
