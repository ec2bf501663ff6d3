// Throughput kernels of the FP32 path (shifted populations g = f - w rho0,
// theta = T - T_sat, FP32 arithmetic with hardware reciprocal / square-root
// approximations).  Same method and boundary treatment as the FP64 kernels of
// lbm_device.cuh, rearranged for speed:
//   flow: the 9-point force sums and the push targets are written out in
//         closed form; wall-side work happens only on the two boundary rows;
//   heat: per cell, once per step, the conduction link weights (harmonic mean
//         conductance x lattice weight x 6 / (rho c)), the velocity and the
//         phase-change source coefficients are precomputed, so that each RK
//         stage costs ~30 FMA-class operations per cell.  The source
//         -(T / rho C_V) (dp/dT)_rho div u is exactly C1 T + C2 sqrt(T) with
//         C1, C2 functions of rho and div u only (Eq. 13 differentiated:
//         (dp/dT)_rho = A(rho) + B(rho) / sqrt(T)).
#pragma once
#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_dfloat.cuh"

namespace lbmgb {

// Every constant an FP32 kernel needs, converted and combined on the host:
// the kernels then issue no FP64 instruction (GB300 runs FP64 at a small
// fraction of the FP32 rate, so even one FP64 division per thread shows).
struct FParams {
    int nx, nf, ns, nt, flags, top_mode, bc_mode, pad0;
    unsigned long long seed;
    long long sine_t0, sine_t1;
    float rho_shift, T_sat, inv_Tc, kappa, a, b, R, two_over_G, mG;
    float tau_V, rho_V, inv_drho, dtau, rho_mean, g, varpi12G2, inv_tauem, sgn_over_taus;
    float s[9], hs[9];
    float c_w_top, vap_threshold;
    float lambda_s, cv_chi, c_v, rho_c_s;
    float inv_c_v, inv_cv_chi;                     // 1 / c_v, 1 / (C_V chi)
    float a_kappa, kappa_over_Tc, B_coef;          // (dp/dT)_rho pieces: a kappa, kappa / Tc, (1 + kappa) / sqrt(Tc)
    float dTb, Tb_noise, sine_amp, sine_wl;        // bottom: T_b - T_sat, T_b A, amp Tc, wavelength
    unsigned tx_pad;                               // test hook of the staged-copy waits (0)
    // the same constants as double-float pairs (hi, lo) for the heat kernels
    // that evaluate the Eq. 24 source in double-float arithmetic
    float df_tsat[2], df_b[2], df_R[2], df_akappa[2], df_koTc[2], df_Bcoef[2], df_cv[2], df_w1[2], df_w2[2];
};

inline FParams make_fparams(const DevParams &p) {
    FParams q{};
    q.nx = p.nx; q.nf = p.nf; q.ns = p.ns; q.nt = p.nt;
    q.flags = p.flags; q.top_mode = p.top_mode; q.bc_mode = p.bc_mode;
    q.seed = p.seed; q.sine_t0 = p.sine_t0; q.sine_t1 = p.sine_t1;
    q.rho_shift = (float)p.rho_shift; q.T_sat = (float)p.T_sat; q.inv_Tc = (float)(1.0 / p.Tc);
    q.kappa = (float)p.kappa; q.a = (float)p.a; q.b = (float)p.b; q.R = (float)p.R;
    q.two_over_G = (float)(2.0 / p.G); q.mG = (float)(-p.G);
    q.tau_V = (float)p.tau_V; q.rho_V = (float)p.rho_V; q.inv_drho = (float)(1.0 / p.drho_LV);
    q.dtau = (float)p.dtau_LV; q.rho_mean = (float)p.rho_mean; q.g = (float)p.g;
    // |F_m|^2 / psi^2 = G^2 |stencil|^2 (Eq. 10), so eta needs no division by psi^2
    q.varpi12G2 = (float)(p.varpi12 * p.G * p.G); q.inv_tauem = (float)(1.0 / p.tau_e_m);
    q.sgn_over_taus = (float)(p.sign_eps / p.tau_s_m);
    for (int k = 0; k < 9; k++) { q.s[k] = (float)p.s[k]; q.hs[k] = (float)p.hs[k]; }
    q.c_w_top = (float)p.c_w_top; q.vap_threshold = (float)p.vap_threshold;
    q.lambda_s = (float)p.lambda_s; q.cv_chi = (float)p.cv_chi; q.c_v = (float)p.c_v; q.rho_c_s = (float)p.rho_c_s;
    q.inv_c_v = (float)(1.0 / p.c_v); q.inv_cv_chi = (float)(1.0 / p.cv_chi);
    q.a_kappa = (float)(p.a * p.kappa); q.kappa_over_Tc = (float)(p.kappa / p.Tc);
    q.B_coef = (float)((1.0 + p.kappa) / sqrt(p.Tc));
    q.dTb = (float)(p.T_b - p.T_sat); q.Tb_noise = (float)(p.T_b * p.bc_noise);
    q.sine_amp = (float)p.sine_amp; q.sine_wl = (float)p.sine_wl;
    q.tx_pad = p.tx_pad;
    auto split = [](double v, float *o) { o[0] = (float)v; o[1] = (float)(v - (double)o[0]); };
    split(p.T_sat, q.df_tsat); split(p.b, q.df_b); split(p.R, q.df_R); split(p.a * p.kappa, q.df_akappa);
    split(p.kappa / p.Tc, q.df_koTc); split((1.0 + p.kappa) / sqrt(p.Tc), q.df_Bcoef); split(p.c_v, q.df_cv);
    split(1.0 / 9.0, q.df_w1); split(1.0 / 36.0, q.df_w2);
    return q;
}

// theta = T - T_sat of the bottom row, FP32 (same draws as the FP64 path,
// 24-bit uniform).
__device__ __forceinline__ float bottom_theta(const FParams &q, int x, long long n) {
    if (q.bc_mode == BCM_NOISE) {
        const uint64_t gam = 0x9E3779B97F4A7C15ULL;
        uint64_t h = smix(q.seed + gam);
        h = smix((h ^ (uint64_t)TAG_BOTTOM_NOISE) + gam);
        h = smix((h ^ (uint64_t)n) + gam);
        h = smix((h ^ (uint64_t)x) + gam);
        const float U = (float)(unsigned)(h >> 40) * (1.0f / 16777216.0f);
        return q.dTb + q.Tb_noise * (2.0f * U - 1.0f);
    }
    if (q.bc_mode == BCM_SINE && n > q.sine_t0 && n < q.sine_t1) {
        const float arg = 6.28318530717958647692f * ((float)x - 0.25f * q.sine_wl) / q.sine_wl;
        return q.dTb + q.sine_amp * sinf(arg);
    }
    return q.dTb;
}

// Single-instruction PTX approximations (documented maximum error 1 ulp for
// the reciprocal, 2^-23 relative for the root), flushing subnormals: no
// value of the FP32 path is subnormal, and this skips the special-range
// handling the library intrinsics carry.
__device__ __forceinline__ float fast_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fast_sqrt(float x) {  // x >= 0
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (sm_100 and later): one instruction updates both halves
// of a float2, each rounded as the scalar operation would be.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }  // exact a - b
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(fast_rcp(a.x), fast_rcp(a.y)); }

// psi(rho, T) of Eq. 12-13 in FP32 with approximate reciprocals / roots.
__device__ __forceinline__ float psi_fast(const FParams &q, float rho, float T, unsigned &errbits) {
    const float t1 = fast_sqrt(T * q.inv_Tc);
    const float t2 = 1.0f + q.kappa * (1.0f - t1);
    const float phi = t2 * t2;
    const float br = q.b * rho;
    const float omb = 1.0f - br, den = 1.0f + br * (2.0f - br);
    // p = rho R T / (1 - b rho) - a phi rho^2 / den over one common denominator
    const float p = rho * ((q.R * T) * den - (q.a * phi) * rho * omb) * fast_rcp(omb * den);
    const float arg = q.two_over_G * (p - rho * (1.0f / 3.0f));
    if (!(arg > 0.0f)) {
        if (!(arg == 0.0f)) errbits |= ERRW_PSI;
        return 0.0f;
    }
    return fast_sqrt(arg);
}

// stored population -> float
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// Population stores.  FP32: plain.  FP16 storage rounds stochastically: a
// dither drawn uniformly from the 13 float mantissa bits a half drops is
// added to the magnitude, which is then truncated (Connolly, Higham and Mary,
// SIAM J. Sci. Comput. 43 (2021), "Stochastic rounding and its probabilistic
// backward error analysis").  Expected stored value = exact value, so the
// per-step rounding errors no longer add up to a drift of the mass (values
// in the half-subnormal range are rounded to nearest after the dither).  The dither: a 32-bit
// key per launch from the seed and the step, one 32-bit hash of key and site
// per site (C. Wellons' two-round multiply-xorshift mixer), then a linear
// congruential step per store (Knuth / Numerical Recipes constants) whose
// top 13 bits are the dither.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
struct PopDither {
    uint32_t s;
    __device__ __forceinline__ uint32_t next() {  // 13 uniform bits
        s = s * 1664525u + 1013904223u;
        return s >> 19;
    }
};
// per-launch key of the dither (0 for FP32 storage, which draws nothing)
template <class S>
__device__ __forceinline__ uint32_t dither_key(const FParams &p, long long n) {
    if constexpr (sizeof(S) == 2)
        return mix32((uint32_t)p.seed ^ mix32((uint32_t)(p.seed >> 32) ^ 0x5bd1e995u) ^
                     mix32((uint32_t)n * 0x9e3779b9u + 0x7f4a7c15u));
    return 0u;
}
template <class S>
__device__ __forceinline__ PopDither pop_dither(uint32_t key, int k) {
    PopDither d{1u};
    if constexpr (sizeof(S) == 2) d.s = mix32(key ^ (uint32_t)k);
    return d;
}
__device__ __forceinline__ void st_pop(float *q, float v, PopDither &) { *q = v; }
__device__ __forceinline__ void st_pop(__half *q, float v, PopDither &d) {
    // the dither goes into the magnitude bits (a carry moves into the
    // exponent, never into the sign for |v| < 2^15); with the 13 low bits
    // cleared the value is a half exactly when |v| is in the normal half
    // range [2^-14, 2^15), and the conversion rounds the rest to nearest
    const uint32_t m = (__float_as_uint(v) + d.next()) & ~0x1fffu;
    *q = __float2half_rn(__uint_as_float(m));
}

// One fluid site's forces (Eq. 11, 14, 15), MRT collision with the improved
// forcing (Eq. 3-10) and push streaming with halfway bounce-back (Eq. 8), FP32
// path.  f: the site's shifted populations; sp: its psi in a tile of row
// stride SW (neighbours at +-1, +-SW); k = y nx + x.  Writes the moments and
// the nine post-collision populations to their destinations.  EDGE = false
// is for sites of tiles that touch no boundary (no wall row, no periodic
// wrap): the wall terms and index wraps drop out at compile time.
template <class S, bool EDGE = true>
__device__ __forceinline__ void flow_site(const FParams &p, const float *f, float d, float rho, const float *sp,
                                          int SW, int x, int y, int k, bool py, bool outflow,
                                          const double *__restrict__ cw, S *const *oplane, float *__restrict__ rho_o,
                                          float *__restrict__ ux_o, float *__restrict__ uy_o, PopDither &dz) {
    const int nx = p.nx, nf = p.nf;
    const float w1 = 1.0f / 3.0f, w2 = 1.0f / 12.0f;
    const float mG = p.mG;
    const float inv_drho = p.inv_drho, dtau = p.dtau;
    const float psi = sp[0];
    const float pE = sp[1], pW = sp[-1], pN = sp[SW], pS = sp[-SW];
    float pNE = sp[SW + 1], pNW = sp[SW - 1];
    const float pSW = sp[-SW - 1], pSE = sp[-SW + 1];
    const bool bot = EDGE && !py && y == 0, top = EDGE && !py && y == nf - 1;
    float pNx = pN;
    if (top && outflow) { pNx = psi; pNE = pE; pNW = pW; }  // open top: zero normal gradient
    const float a = pNE - pSW, b = pSE - pNW;
    const float pre = mG * psi;
    const float sx = w1 * (pE - pW) + w2 * (a + b), sy = w1 * (pNx - pS) + w2 * (a - b);
    const float Fmx = pre * sx, Fmy = pre * sy;
    const int xm = EDGE ? wrap1(x - 1, nx) : x - 1, xp = EDGE ? wrap1(x + 1, nx) : x + 1;
    float Fax = 0.0f, Fay = 0.0f;
    if (bot) {  // Eq. 14 with the heater sites below (i = 4, 7, 8)
        const float cm = float(cw[xm]), c0 = float(cw[x]), cp = float(cw[xp]);
        Fax = -psi * (w2 * (cp - cm));
        Fay = psi * (w1 * c0 + w2 * (cm + cp));
    }
    if (top && !outflow) Fay += -psi * ((w1 + 2.0f * w2) * p.c_w_top);
    const float Fx = Fmx + Fax;
    const float Fy = (Fmy + Fay) - (rho - p.rho_mean) * p.g;

    // moments of g (Eq. 6 with the rho0 shift of m0..m2 folded into q0..q2)
    const float s14 = (f[1] + f[2]) + (f[3] + f[4]);
    const float s58 = (f[5] + f[6]) + (f[7] + f[8]);
    const float m1 = -4.0f * f[0] - s14 + 2.0f * s58;
    const float m2 = 4.0f * f[0] - 2.0f * s14 + s58;
    const float f13 = f[1] - f[3], f24 = f[2] - f[4];
    const float f57 = f[5] - f[7], f86 = f[8] - f[6];
    const float m3 = f13 + (f57 + f86);
    const float m4 = -2.0f * f13 + (f57 + f86);
    const float m5 = f24 + (f57 - f86);
    const float m6 = -2.0f * f24 + (f57 - f86);
    const float m7 = (f[1] + f[3]) - (f[2] + f[4]);
    const float m8 = (f[5] + f[7]) - (f[6] + f[8]);
    const float irho = fast_rcp(rho);
    const float ux = (m3 + 0.5f * Fx) * irho, uy = (m5 + 0.5f * Fy) * irho;
    const float tau = p.tau_V + (rho - p.rho_V) * inv_drho * dtau;
    const float s78 = fast_rcp(tau);
    const float ru2 = rho * (ux * ux + uy * uy);
    const float q1 = -2.0f * d + 3.0f * ru2, q2 = d - 3.0f * ru2;
    const float q3 = rho * ux, q5 = rho * uy;
    const float q7 = rho * (ux * ux - uy * uy), q8 = rho * (ux * uy);
    const float uF = ux * Fx + uy * Fy;
    const float eps = (psi > 0.0f) ? p.varpi12G2 * (sx * sx + sy * sy) : 0.0f;
    const float S1 = 6.0f * uF + eps * p.inv_tauem;
    const float S2 = -6.0f * uF + eps * p.sgn_over_taus;
    // Eq. 7 (m0 unchanged; q4 = -q3, q6 = -q5)
    const float z1 = m1 - p.s[1] * (m1 - q1) + p.hs[1] * S1;
    const float z2 = m2 - p.s[2] * (m2 - q2) + p.hs[2] * S2;
    const float z3 = m3 - p.s[3] * (m3 - q3) + p.hs[3] * Fx;
    const float z4 = m4 - p.s[4] * (m4 + q3) - p.hs[4] * Fx;
    const float z5 = m5 - p.s[5] * (m5 - q5) + p.hs[5] * Fy;
    const float z6 = m6 - p.s[6] * (m6 + q5) - p.hs[6] * Fy;
    const float h78 = 1.0f - 0.5f * s78;
    const float z7 = m7 - s78 * (m7 - q7) + h78 * (2.0f * (ux * Fx - uy * Fy));
    const float z8 = m8 - s78 * (m8 - q8) + h78 * (ux * Fy + uy * Fx);
    const float e0 = d * (1.0f / 9.0f), e1 = z1 * (1.0f / 36.0f), e2 = z2 * (1.0f / 36.0f);
    const float e3 = z3 * (1.0f / 6.0f), e4 = z4 * (1.0f / 12.0f), e5 = z5 * (1.0f / 6.0f);
    const float e6 = z6 * (1.0f / 12.0f), e7 = z7 * 0.25f, e8 = z8 * 0.25f;
    const float A0 = e0 - e1 - 2.0f * e2;       // axis-direction common part
    const float B0 = e0 + 2.0f * e1 + e2;       // diagonal common part
    const float fo0 = e0 - 4.0f * e1 + 4.0f * e2;
    const float fo1 = A0 + (e3 - 2.0f * e4) + e7;
    const float fo3 = A0 - (e3 - 2.0f * e4) + e7;
    const float fo2 = A0 + (e5 - 2.0f * e6) - e7;
    const float fo4 = A0 - (e5 - 2.0f * e6) - e7;
    const float cxx = e3 + e4, cyy = e5 + e6;
    const float fo5 = B0 + cxx + cyy + e8;
    const float fo6 = B0 - cxx + cyy - e8;
    const float fo7 = B0 - cxx - cyy + e8;
    const float fo8 = B0 + cxx - cyy - e8;
    rho_o[k] = rho;
    ux_o[k] = ux;
    uy_o[k] = uy;
    // Eq. 8, push; halfway bounce-back at the heater and the top wall
    // (32-bit offsets from this site: east / west columns, rows above / below)
    const int dxp = xp - x, dxm = xm - x;
    const int kn = (EDGE && py && y == nf - 1) ? x : k + nx;                // row above
    const int ks_ = (EDGE && py && y == 0) ? (nf - 1) * nx + x : k - nx;    // row below
    st_pop(oplane[0] + k, fo0, dz);
    st_pop(oplane[1] + k + dxp, fo1, dz);
    st_pop(oplane[3] + k + dxm, fo3, dz);
    if (!top) {
        st_pop(oplane[2] + kn, fo2, dz);
        st_pop(oplane[5] + kn + dxp, fo5, dz);
        st_pop(oplane[6] + kn + dxm, fo6, dz);
    } else if (!outflow) {
        st_pop(oplane[4] + k, fo2, dz);
        st_pop(oplane[7] + k, fo5, dz);
        st_pop(oplane[8] + k, fo6, dz);
    }
    if (!bot) {
        st_pop(oplane[4] + ks_, fo4, dz);
        st_pop(oplane[7] + ks_ + dxm, fo7, dz);
        st_pop(oplane[8] + ks_ + dxp, fo8, dz);
    } else {
        st_pop(oplane[2] + k, fo4, dz);
        st_pop(oplane[5] + k, fo7, dz);
        st_pop(oplane[6] + k, fo8, dz);
    }
    if (top && outflow) {
        st_pop(oplane[4] + k, fo4, dz);
        st_pop(oplane[7] + k + dxm, fo7, dz);
        st_pop(oplane[8] + k + dxp, fo8, dz);
    }
}

// ============================================================================
// Flow kernel, FP32 shifted populations, one tile per block.  Tile TX = BX
// columns x TY = BY * RY rows; thread (tx, ty) owns rows ty + k BY.  psi tile
// with a one-site halo in shared memory; the halo ring is recomputed from the
// neighbours' populations (L2 hits).  Rows outside the fluid hold psi = 0
// (walls add their pull through F_ads) or, for an open top, the psi of the
// top row.
// ============================================================================
template <class P, int BX, int BY, int RY, int MINB>
__global__ void __launch_bounds__(BX *BY, MINB)
k_flow_fast(const FParams p, const typename P::fst *__restrict__ fin, typename P::fst *__restrict__ fout,
            const typename P::tst *__restrict__ Tin, float *__restrict__ rho_o, float *__restrict__ ux_o,
            float *__restrict__ uy_o, const double *__restrict__ cw, double *__restrict__ part,
            unsigned *__restrict__ err, const long long *__restrict__ stepp) {
    using S = typename P::fst;
    constexpr int TX = BX, TY = BY * RY, SW = TX + 2, SH = TY + 2, NT = BX * BY;
    __shared__ float s_psi[SH * SW];
    __shared__ float s_red[2][NT / 32];

    const int nx = p.nx, nf = p.nf;
    const uint32_t dkey = sizeof(S) == 2 ? dither_key<S>(p, *stepp) : 0u;  // keys the FP16 store dither
    const size_t plane = (size_t)nf * nx;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool frozen = (p.flags & FLAG_FROZEN_FLOW) != 0;
    const bool outflow = p.top_mode == TOP_OUTFLOW;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * BX + threadIdx.x;
    const float rho0 = p.rho_shift;
    const float tsat = p.T_sat;
    unsigned errbits = 0;

    float g[RY][9];
    float dd[RY];

    // ---- own sites: load, density, psi ----
    #pragma unroll
    for (int r = 0; r < RY; r++) {
        const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
        const int x = (x0 + lx < nx) ? x0 + lx : wrapi(x0 + lx, nx);
        int y = y0 + ly;
        const bool has = py || y < nf;
        if (py) y = wrapi(y, nf);
        float psi = 0.0f;
        dd[r] = 0.0f;
        if (has) {
            const size_t k = (size_t)y * nx + x;
            #pragma unroll
            for (int i = 0; i < 9; i++) g[r][i] = ld_as<float>(fin + i * plane + k);
            const float d = ((g[r][0] + g[r][1]) + (g[r][2] + g[r][3])) + ((g[r][4] + g[r][5]) + (g[r][6] + g[r][7])) + g[r][8];
            dd[r] = d;
            const float T = ld_as<float>(Tin + (size_t)(p.ns + y) * nx + x) + tsat;
            if (!frozen) psi = psi_fast(p, d + rho0, T, errbits);
        } else {
            #pragma unroll
            for (int i = 0; i < 9; i++) g[r][i] = 0.0f;
        }
        s_psi[(ly + 1) * SW + lx + 1] = psi;
    }
    // ---- halo ring ----
    if (!frozen) {
        for (int k = tid; k < 2 * SW + 2 * TY; k += NT) {
            int hx, hy;
            if (k < SW) { hx = k; hy = 0; }
            else if (k < 2 * SW) { hx = k - SW; hy = SH - 1; }
            else if (k < 2 * SW + TY) { hx = 0; hy = 1 + (k - 2 * SW); }
            else { hx = SW - 1; hy = 1 + (k - 2 * SW - TY); }
            const int x = wrapi(x0 + hx - 1, nx);
            int y = y0 + hy - 1;
            if (py) y = wrapi(y, nf);
            float psi = 0.0f;
            if (y >= 0 && y < nf) {
                const size_t kk = (size_t)y * nx + x;
                float v[9];
                #pragma unroll
                for (int i = 0; i < 9; i++) v[i] = ld_as<float>(fin + i * plane + kk);
                const float d = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
                const float T = ld_as<float>(Tin + (size_t)(p.ns + y) * nx + x) + tsat;
                psi = psi_fast(p, d + rho0, T, errbits);
            }
            s_psi[hy * SW + hx] = psi;
        }
    }
    __syncthreads();

    // ---- collide and push ----
    S *oplane[9];
    #pragma unroll
    for (int i = 0; i < 9; i++) oplane[i] = fout + i * plane;
    float mass = 0.0f, nvap = 0.0f;
    #pragma unroll
    for (int r = 0; r < RY; r++) {
        const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
        const int x = x0 + lx, y = y0 + ly;
        if (x >= nx || y >= nf) continue;
        const int k = y * nx + x;
        PopDither dz = pop_dither<S>(dkey, k);
        const float d = dd[r];
        const float rho = d + rho0;
        if (!(fabsf(rho) < 1e30f)) errbits |= ERRW_NONFINITE_RHO;
        mass += rho;
        nvap += (rho < p.vap_threshold) ? 1.0f : 0.0f;
        if (frozen) {
            #pragma unroll
            for (int i = 0; i < 9; i++) st_pop(oplane[i] + k, g[r][i], dz);
            rho_o[k] = rho;
            ux_o[k] = 0.0f;
            uy_o[k] = 0.0f;
            continue;
        }
        flow_site<S>(p, g[r], d, rho, s_psi + (ly + 1) * SW + (lx + 1), SW, x, y, k, py, outflow, cw, oplane, rho_o,
                     ux_o, uy_o, dz);
    }
    // per-block mass and vapour count: FP32 inside the block, FP64 across blocks
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
        const int bi = blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * bi] = m;
        part[2 * bi + 1] = v;
    }
    if (errbits) atomicOr(err, errbits);
}

// Flow kernel, FP32, persistent: SMs x resident blocks, each looping over
// TX x TY tiles (same per-site work as k_flow_fast, through flow_site).
// While a tile is computed, the next tile's populations, T and psi-ring
// sites are already loading into registers.  Tiles that touch no boundary
// use flow_site's interior form.  WIDE (compile time) promises nx >= TX + 1
// and, if periodic in y, nf >= TY + 2, so that index wraps are a compare.
// The body of the persistent flow kernel over tiles first, first + step, ...
// (below end) of a run.  PER_TILE: each tile writes its own mass and
// vapour-count partials (part[2 tile], part[2 tile + 1]), so the run's sums
// do not depend on which block did which tile; otherwise the block writes
// one pair at part[2 part_slot].
template <class P, int BX, int BY, int RY, bool WIDE, bool PER_TILE>
__device__ __forceinline__ void
flow_pers_body(const FParams &p, int tiles_x, int end, int first, int step, const typename P::fst *__restrict__ fin,
               typename P::fst *__restrict__ fout, const typename P::tst *__restrict__ Tin, float *__restrict__ rho_o,
               float *__restrict__ ux_o, float *__restrict__ uy_o, const double *__restrict__ cw,
               double *__restrict__ part, unsigned *__restrict__ err, const long long *__restrict__ stepp, int part_slot) {
    using S = typename P::fst;
    constexpr int TX = BX, TY = BY * RY, SW = TX + 2, SH = TY + 2, NT = BX * BY;
    __shared__ float s_psi[SH * SW];
    __shared__ float s_red[2][NT / 32];

    const int nx = p.nx, nf = p.nf;
    const uint32_t dkey = sizeof(S) == 2 ? dither_key<S>(p, *stepp) : 0u;  // keys the FP16 store dither
    const size_t plane = (size_t)nf * nx;
    // per-plane base pointers (uniform); site offsets below are 32-bit (the
    // runtime rejects domains of more than 2e9 sites, so one plane indexes in 31 bits)
    const S *fplane[9];
    S *oplane[9];
    #pragma unroll
    for (int i = 0; i < 9; i++) { fplane[i] = fin + i * plane; oplane[i] = fout + i * plane; }
    const typename P::tst *Tfl = Tin + (size_t)p.ns * nx;  // first fluid row of T
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool frozen = (p.flags & FLAG_FROZEN_FLOW) != 0;
    const bool outflow = p.top_mode == TOP_OUTFLOW;
    const int tid = threadIdx.y * BX + threadIdx.x;
    const float rho0 = p.rho_shift;
    const float tsat = p.T_sat;
    unsigned errbits = 0;

    float g[RY][9];
    float dd[RY];
    float gT[RY];
    // WIDE (compile time): nx >= TX + 1 and, if periodic in y, nf >= TY + 2, so
    // every wrap below is one compare instead of an integer modulo
    auto wx = [&](int v) { return WIDE ? wrap1(v, nx) : wrapi(v, nx); };
    auto wy = [&](int v) { return WIDE ? wrap1(v, nf) : wrapi(v, nf); };
    // tile coordinates advance by `step` tiles per iteration without a division
    const int gdx = step % tiles_x, gdy = step / tiles_x;
    // populations (as stored: converted only when the tile starts, so that
    // no instruction waits on the loads before then) and temperature of the
    // next tile, loaded during this tile
    S pg[RY][9];
    float pTv[RY];
    // one halo-ring site per thread (threads 0 .. ring-1): its density and T
    constexpr int RING = 2 * SW + 2 * TY;
    static_assert(RING <= NT, "one ring site per thread");
    S rg[9];
    float rT = 0.0f;
    bool rvalid = false;
    int rslot = 0;  // shared-memory slot of this thread's ring site (set by fetch)
    auto ring_site = [&](int k, int x0, int y0, int &hx, int &hy, int &x, int &y) {
        if (k < SW) { hx = k; hy = 0; }
        else if (k < 2 * SW) { hx = k - SW; hy = SH - 1; }
        else if (k < 2 * SW + TY) { hx = 0; hy = 1 + (k - 2 * SW); }
        else { hx = SW - 1; hy = 1 + (k - 2 * SW - TY); }
        x = wx(x0 + hx - 1);
        y = y0 + hy - 1;
        if (py) y = wy(y);
        return py || (y >= 0 && y < nf);
    };
    auto fetch_ring = [&](int txt, int tyt) {
        const int x0 = txt * TX, y0 = tyt * TY;
        if (tid < RING && !frozen) {
            int hx, hy, x, y;
            rvalid = ring_site(tid, x0, y0, hx, hy, x, y);
            rslot = hy * SW + hx;
            if (rvalid) {
                const int kk = y * nx + x;
                #pragma unroll
                for (int i = 0; i < 9; i++) rg[i] = __ldg(fplane[i] + kk);
                rT = ld_as<float>(Tfl + kk);
            }
        }
    };
    auto fetch_main = [&](int txt, int tyt) {
        const int x0 = txt * TX, y0 = tyt * TY;
        #pragma unroll
        for (int r = 0; r < RY; r++) {
            const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
            const int x = wx(x0 + lx);
            int y = y0 + ly;
            const bool has = py || y < nf;
            if (py) y = wy(y);
            if (has) {
                const int k = y * nx + x;
                #pragma unroll
                for (int i = 0; i < 9; i++) pg[r][i] = __ldg(fplane[i] + k);
                pTv[r] = ld_as<float>(Tfl + k);
            } else {
                #pragma unroll
                for (int i = 0; i < 9; i++) pg[r][i] = S(0.0f);
                pTv[r] = 0.0f;
            }
        }
    };
    float mass = 0.0f, nvap = 0.0f;
    int cxt = first % tiles_x, cyt = first / tiles_x;  // current tile
    if (first < end) { fetch_ring(cxt, cyt); fetch_main(cxt, cyt); }
    for (int tile = first; tile < end; tile += step) {
    const int x0 = cxt * TX, y0 = cyt * TY;
    int nxt = cxt + gdx, nyt = cyt + gdy;  // next tile of this block
    if (nxt >= tiles_x) { nxt -= tiles_x; nyt += 1; }
    #pragma unroll
    for (int r = 0; r < RY; r++) {
        #pragma unroll
        for (int i = 0; i < 9; i++) g[r][i] = to_f(pg[r][i]);
        gT[r] = pTv[r];
    }
    const bool more = tile + step < end;
    // the next tile's own sites load from here on, under this tile's psi and
    // collision work; its ring sites once this tile's ring psi is done
    if (more) fetch_main(nxt, nyt);

    // ---- own sites: density, psi ----
    #pragma unroll
    for (int r = 0; r < RY; r++) {
        const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
        const int y = y0 + ly;
        const bool has = py || y < nf;
        float psi = 0.0f;
        dd[r] = 0.0f;
        if (has) {
            const float d = ((g[r][0] + g[r][1]) + (g[r][2] + g[r][3])) + ((g[r][4] + g[r][5]) + (g[r][6] + g[r][7])) + g[r][8];
            dd[r] = d;
            if (!frozen) psi = psi_fast(p, d + rho0, gT[r] + tsat, errbits);
        }
        s_psi[(ly + 1) * SW + lx + 1] = psi;
    }
    // ---- halo ring, from the prefetched registers ----
    if (!frozen && tid < RING) {
        float psi = 0.0f;
        if (rvalid) {
            float f[9];
            #pragma unroll
            for (int i = 0; i < 9; i++) f[i] = to_f(rg[i]);
            const float d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            psi = psi_fast(p, d + rho0, rT + tsat, errbits);
        }
        s_psi[rslot] = psi;
    }
    if (more) fetch_ring(nxt, nyt);
    __syncthreads();

    // ---- collide and push (tiles that touch no boundary skip the wall terms) ----
    auto collide = [&](auto edge_tag) {
        constexpr bool E = decltype(edge_tag)::value;
        #pragma unroll
        for (int r = 0; r < RY; r++) {
            const int lx = threadIdx.x, ly = threadIdx.y + r * BY;
            const int x = x0 + lx, y = y0 + ly;
            if (E && (x >= nx || y >= nf)) continue;
            const int k = y * nx + x;
            PopDither dz = pop_dither<S>(dkey, (int)k);
            const float d = dd[r];
            const float rho = d + rho0;
            if (!(fabsf(rho) < 1e30f)) errbits |= ERRW_NONFINITE_RHO;
            mass += rho;
            nvap += (rho < p.vap_threshold) ? 1.0f : 0.0f;
            if (frozen) {
                #pragma unroll
                for (int i = 0; i < 9; i++) st_pop(oplane[i] + k, g[r][i], dz);
                rho_o[k] = rho;
                ux_o[k] = 0.0f;
                uy_o[k] = 0.0f;
                continue;
            }
            flow_site<S, E>(p, g[r], d, rho, s_psi + (ly + 1) * SW + (lx + 1), SW, x, y, k, py, outflow, cw, oplane,
                            rho_o, ux_o, uy_o, dz);
        }
    };
    if (x0 == 0 || x0 + TX >= nx || y0 == 0 || y0 + TY >= nf) collide(std::true_type{});
    else collide(std::false_type{});
    if constexpr (PER_TILE) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mass += __shfl_down_sync(0xffffffffu, mass, o);
            nvap += __shfl_down_sync(0xffffffffu, nvap, o);
        }
        if ((tid & 31) == 0) { s_red[0][tid >> 5] = mass; s_red[1][tid >> 5] = nvap; }
        mass = 0.0f;
        nvap = 0.0f;
    }
    __syncthreads();  // s_psi is rewritten by the next tile
    if constexpr (PER_TILE) {
        // (s_red is rewritten only after the next tile's psi barrier)
        if (tid == 0) {
            double m = 0.0, v = 0.0;
            #pragma unroll
            for (int w = 0; w < NT / 32; w++) { m += (double)s_red[0][w]; v += (double)s_red[1][w]; }
            part[2 * tile] = m;
            part[2 * tile + 1] = v;
        }
    }
    cxt = nxt; cyt = nyt;
    }
    if constexpr (!PER_TILE) {
        // per-block mass and vapour count: FP32 inside the block, FP64 across blocks
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
            part[2 * part_slot] = m;
            part[2 * part_slot + 1] = v;
        }
    }
    if (errbits) atomicOr(err, errbits);
}

template <class P, int BX, int BY, int RY, int MINB, bool WIDE>
__global__ void __launch_bounds__(BX *BY, MINB)
k_flow_pers(const __grid_constant__ FParams p, int tiles_x, int ntiles, const typename P::fst *__restrict__ fin,
            typename P::fst *__restrict__ fout, const typename P::tst *__restrict__ Tin, float *__restrict__ rho_o,
            float *__restrict__ ux_o, float *__restrict__ uy_o, const double *__restrict__ cw,
            double *__restrict__ part, unsigned *__restrict__ err, const long long *__restrict__ stepp) {
    flow_pers_body<P, BX, BY, RY, WIDE, false>(p, tiles_x, ntiles, (int)blockIdx.x, (int)gridDim.x, fin, fout, Tin,
                                               rho_o, ux_o, uy_o, cw, part, err, stepp, (int)blockIdx.x);
}



// ============================================================================
// Heat kernel, FP32.  Output tile TX x TY, 4-cell halo.  Shared arrays per
// cell: three temperature buffers, eight link coefficients k_a, their sum,
// -3 u_x w, -3 u_y w folded advection factors, the source coefficients C1, C2.
// Threads are laid out 2-D (BXH x BYH) and stride over the region, so no
// integer division appears in the stage loops.
// ============================================================================
template <int TX, int TY>
struct HeatFastLayout {
    static constexpr int H = 4, SW = TX + 2 * H, SH = TY + 2 * H, NC = SW * SH;
    static constexpr int NARR = 3 + 8 + 1 + 2 + 2;  // T x3, k x8, ksum, adv x2, C1, C2
    static constexpr size_t bytes = (size_t)NC * NARR * sizeof(float) + (size_t)TX * TY * sizeof(float) + NC + 64;
};

template <class P, int TX, int TY, int BXH, int BYH>
__global__ void __launch_bounds__(BXH *BYH)
k_heat_fast(const FParams p, const typename P::tst *__restrict__ Tin, typename P::tst *__restrict__ Tout,
            const float *__restrict__ rho_i, const float *__restrict__ ux_i, const float *__restrict__ uy_i,
            const long long *__restrict__ stepp, unsigned *__restrict__ err) {
    using L = HeatFastLayout<TX, TY>;
    constexpr int H = L::H, SW = L::SW, SH = L::SH, NC = L::NC;
    extern __shared__ __align__(16) unsigned char smraw[];
    float *base = reinterpret_cast<float *>(smraw);
    float *sTn = base, *sA = base + NC, *sB = base + 2 * NC;
    float *sk = base + 3 * NC;          // 8 arrays: k_a for a = 1..8
    float *sks = base + 11 * NC;        // sum of k_a
    float *sax = base + 12 * NC, *say = base + 13 * NC;
    float *sc1 = base + 14 * NC, *sc2 = base + 15 * NC;
    float *sAcc = base + 16 * NC;
    unsigned char *kind = reinterpret_cast<unsigned char *>(sAcc + TX * TY);
    // load phase: lambda in sA (neighbour reads), -3u in sax/say (final form,
    // neighbour reads for div u), own-cell rho c in sc1 and rho in sc2
    float *sLam = sA, *sRcv = sc1, *sRho = sc2;

    const int nx = p.nx, nt = p.nt, ns = p.ns, nf = p.nf;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool iso = (p.flags & FLAG_ISOTHERMAL) != 0;
    const int x0 = blockIdx.x * TX, r0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long n = *stepp;
    unsigned errbits = 0;

    constexpr int NTH = BXH * BYH;
    const int tid = ty * BXH + tx;
    // ---- load (flattened: constant divisor SW) ----
    for (int c = tid; c < NC; c += NTH) {
        const int hy = c / SW, hx = c - (c / SW) * SW;
        int row = r0 + hy - H;
        unsigned char kd;
        if (py) { row = wrapi(row, nt); kd = 2; }
        else if (row < 0 || row > nt) kd = 0;
        else if (row == 0 || row == nt) kd = 3;
        else kd = (row < ns) ? 1 : 2;
        {
            const int x = wrapi(x0 + hx - H, nx);
            float T = 0.0f, lam = 0.0f, ux = 0.0f, uy = 0.0f, rcv = 1.0f, rho = 0.0f;
            if (kd == 1) {
                T = Tin[(size_t)row * nx + x];
                lam = p.lambda_s;
                rcv = p.rho_c_s;
            } else if (kd == 2) {
                const size_t kf = (size_t)(row - ns) * nx + x;
                T = Tin[(size_t)row * nx + x];
                rho = rho_i[kf];
                ux = ux_i[kf];
                uy = uy_i[kf];
                lam = p.cv_chi * rho;
                rcv = rho * p.c_v;
            } else if (kd == 3) {
                if (row == 0) {  // Model A: the wall row conducts like the first fluid row
                    T = bottom_theta(p, x, n);
                    lam = (p.flags & FLAG_MODEL_A) ? p.cv_chi * rho_i[x] : p.lambda_s;
                } else {
                    T = 0.0f;
                    lam = p.cv_chi * rho_i[(size_t)(nf - 1) * nx + x];
                }
            }
            sTn[c] = T; sB[c] = T;
            sLam[c] = lam; sax[c] = -3.0f * ux; say[c] = -3.0f * uy; sRcv[c] = rcv; sRho[c] = rho;
            kind[c] = kd;
        }
    }
    __syncthreads();
    // ---- coefficients, same thread-cell map as the load (own-cell slots only
    // are rewritten; neighbours are read from sA = lambda and sax/say) ----
    // k_a = 6 w_a lambda_face / (rho c), lambda_face = harmonic mean
    const float w1 = 1.0f / 9.0f, w2 = 1.0f / 36.0f;
    for (int c = tid; c < NC; c += NTH) {
        const int hy = c / SW, hx = c - (c / SW) * SW;
        {
            const unsigned char kd = kind[c];
            float kk[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            float ks = 0.0f, c1 = 0.0f, c2 = 0.0f;
            const bool inner = hx >= 1 && hx < SW - 1 && hy >= 1 && hy < SH - 1;
            if (inner && (kd == 1 || kd == 2)) {
                const float l0 = sLam[c];
                const float inv6 = 6.0f * fast_rcp(sRcv[c]);
                const int off[8] = {1, SW, -1, -SW, SW + 1, SW - 1, -SW - 1, -SW + 1};
                #pragma unroll
                for (int a = 0; a < 8; a++) {
                    const float la = sLam[c + off[a]];
                    const float hm = 2.0f * l0 * la * fast_rcp(l0 + la);
                    kk[a] = (a < 4 ? w1 : w2) * hm * inv6;
                    ks += kk[a];
                }
                if (kd == 2) {
                    // Eq. 27 divergence of the frozen velocity (sax, say hold -3 u)
                    const float dx = w1 * (sax[c + 1] - sax[c - 1]) +
                                     w2 * ((sax[c + SW + 1] - sax[c - SW - 1]) + (sax[c - SW + 1] - sax[c + SW - 1]));
                    const float dy = w1 * (say[c + SW] - say[c - SW]) +
                                     w2 * ((say[c + SW + 1] - say[c - SW - 1]) - (say[c - SW + 1] - say[c + SW - 1]));
                    const float divu = -(dx + dy);  // 3 (sum w e.u) with the -3 folded out
                    // (dp/dT)_rho = A + B / sqrt(T) (Eq. 13), rho-only A, B
                    const float rho = sRho[c];
                    const float br = p.b * rho;
                    const float iden = fast_rcp(1.0f + br * (2.0f - br));
                    const float pa = p.a_kappa * rho * rho * iden;
                    const float A = rho * p.R * fast_rcp(1.0f - br) - pa * p.kappa_over_Tc;
                    const float B = pa * p.B_coef;
                    const float g0 = -divu * fast_rcp(sRcv[c]);
                    c1 = g0 * A;   // times T
                    c2 = g0 * B;   // times sqrt(T)
                }
            }
            #pragma unroll
            for (int a = 0; a < 8; a++) sk[a * NC + c] = kk[a];
            sks[c] = ks;
            sc1[c] = c1;
            sc2[c] = c2;
        }
    }
    __syncthreads();
    for (int c = tid; c < NC; c += NTH) sA[c] = sTn[c];
    __syncthreads();

    // ---- four RK stages on shrinking regions (region width a compile-time
    // constant per stage, cells dealt out densely) ----
    const float tsat = p.T_sat;
    auto stage = [&](auto mtag, const float *Tk, float *To) {
        constexpr int m = decltype(mtag)::value;
        constexpr int st = m - 1;
        constexpr int RW = SW - 2 * m, RH = SH - 2 * m;
        for (int q = tid; q < RW * RH; q += NTH) {
            const int hy = m + q / RW, hx = m + (q - (q / RW) * RW);
            const int c = hy * SW + hx;
            const unsigned char kd = kind[c];
            if (kd != 1 && kd != 2) continue;
            const float T0 = Tk[c];
            const float T1 = Tk[c + 1], T2 = Tk[c + SW], T3 = Tk[c - 1], T4 = Tk[c - SW];
            const float T5 = Tk[c + SW + 1], T6 = Tk[c + SW - 1], T7 = Tk[c - SW - 1], T8 = Tk[c - SW + 1];
            float h = sk[c] * T1 + sk[NC + c] * T2 + sk[2 * NC + c] * T3 + sk[3 * NC + c] * T4 +
                      sk[4 * NC + c] * T5 + sk[5 * NC + c] * T6 + sk[6 * NC + c] * T7 +
                      sk[7 * NC + c] * T8 - sks[c] * T0;
            if (kd == 2) {
                const float a = T5 - T7, b = T8 - T6;
                const float gx = w1 * (T1 - T3) + w2 * (a + b);
                const float gy = w1 * (T2 - T4) + w2 * (a - b);
                const float Ta = fmaxf(T0 + tsat, 1e-30f);
                h += sax[c] * gx + say[c] * gy + sc1[c] * Ta + sc2[c] * fast_sqrt(Ta);
            }
            const bool in_tile = hx >= H && hx < H + TX && hy >= H && hy < H + TY;
            const int ai = (hy - H) * TX + (hx - H);
            const float Tn = sTn[c];
            if constexpr (st == 0) {
                if (in_tile) sAcc[ai] = h;
                To[c] = Tn + 0.5f * h;
            } else if constexpr (st == 1) {
                if (in_tile) sAcc[ai] += 2.0f * h;
                To[c] = Tn + 0.5f * h;
            } else if constexpr (st == 2) {
                if (in_tile) sAcc[ai] += 2.0f * h;
                To[c] = Tn + h;
            } else {
                sAcc[ai] += h;
            }
        }
        __syncthreads();
    };
    if (!iso) {
        stage(std::integral_constant<int, 1>{}, sTn, sA);
        stage(std::integral_constant<int, 2>{}, sA, sB);
        stage(std::integral_constant<int, 3>{}, sB, sA);
        stage(std::integral_constant<int, 4>{}, sA, nullptr);
    }
    // ---- write ----
    for (int a = tid; a < TX * TY; a += NTH) {
        const int yy = a / TX, xx = a - (a / TX) * TX;
        const int row = r0 + yy, x = x0 + xx;
        if (row < nt && x < nx) {
            const int c = (yy + H) * SW + (xx + H);
            const unsigned char kd = kind[c];
            float v = sTn[c];
            if ((kd == 1 || kd == 2) && !iso) v = sTn[c] + sAcc[yy * TX + xx] * (1.0f / 6.0f);
            if (!(fabsf(v) < 1e30f)) errbits |= ERRW_NONFINITE_T;
            Tout[(size_t)row * nx + x] = v;
        }
    }
    if (errbits) atomicOr(err, errbits);
}

template <class P, int BX, int BY, int RY, int MINB>
struct FlowFastShape {
    static cudaError_t prepare() { return cudaSuccess; }
    static dim3 grid(const DevParams &p) { return dim3((p.nx + BX - 1) / BX, (p.nf + BY * RY - 1) / (BY * RY)); }
    static int blocks(const DevParams &p) { dim3 g = grid(p); return (int)(g.x * g.y); }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        k_flow_fast<P, BX, BY, RY, MINB><<<grid(p), dim3(BX, BY), 0, s>>>(
            make_fparams(p), (const typename P::fst *)b.f_in, (typename P::fst *)b.f_out, (const typename P::tst *)b.T_in,
            (float *)b.rho, (float *)b.ux, (float *)b.uy, b.cw, b.part, b.err, b.step);
        return cudaGetLastError();
    }
};

template <class P, int BX, int BY, int RY, int MINB>
struct FlowPersShape {
    static int grid_blocks;
    static cudaError_t prepare() {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_flow_pers<P, BX, BY, RY, MINB, true>, BX * BY, 0);
        if (e != cudaSuccess) return e;
        grid_blocks = sms * (per > 0 ? per : 1);
        return cudaSuccess;
    }
    static int tiles(const DevParams &p) { return ((p.nx + BX - 1) / BX) * ((p.nf + BY * RY - 1) / (BY * RY)); }
    static int blocks(const DevParams &p) { const int t = tiles(p); return t < grid_blocks ? t : grid_blocks; }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        const bool wide = p.nx >= BX + 1 && (!(p.flags & FLAG_PERIODIC_Y) || p.nf >= BY * RY + 2);
        auto k = wide ? k_flow_pers<P, BX, BY, RY, MINB, true> : k_flow_pers<P, BX, BY, RY, MINB, false>;
        k<<<blocks(p), dim3(BX, BY), 0, s>>>(
            make_fparams(p), (p.nx + BX - 1) / BX, tiles(p), (const typename P::fst *)b.f_in, (typename P::fst *)b.f_out,
            (const typename P::tst *)b.T_in, (float *)b.rho, (float *)b.ux, (float *)b.uy, b.cw, b.part, b.err, b.step);
        return cudaGetLastError();
    }
};
template <class P, int BX, int BY, int RY, int MINB>
int FlowPersShape<P, BX, BY, RY, MINB>::grid_blocks = 152;

template <class P, int TX, int TY, int BXH, int BYH>
struct HeatFastShape {
    static constexpr size_t smem = HeatFastLayout<TX, TY>::bytes;
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(k_heat_fast<P, TX, TY, BXH, BYH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        dim3 g((p.nx + TX - 1) / TX, (p.nt + TY - 1) / TY);
        k_heat_fast<P, TX, TY, BXH, BYH><<<g, dim3(BXH, BYH), smem, s>>>(
            make_fparams(p), (const typename P::tst *)b.T_in, (typename P::tst *)b.T_out, (const float *)b.rho,
            (const float *)b.ux, (const float *)b.uy, b.step, b.err);
        return cudaGetLastError();
    }
};

}  // namespace lbmgb

namespace lbmgb {

// ============================================================================
// Heat kernel, FP32, row-strip persistent variant.  A block covers BW
// columns x SH = R BY rows of cells (4-cell halo for the four RK stages, so
// (BW - 8) x (SH - 8) outputs per tile) and loops over tiles; thread (tx, ty)
// owns the R vertically adjacent cells of rows R ty .. R ty + R - 1:
// their vertical neighbours are its own registers, and one stage of all R
// cells reads 2 R + 6 words of shared memory (bank-conflict free).  Cells
// that do not evolve (outside the domain, the Dirichlet bottom row, the top
// ghost) get zero coefficients, so every cell runs the same branch-free
// update and keeps T^n; cells outside a stage's shrinking region compute
// values nobody reads.  The source of Eq. 24 is folded into the link form
//   K(T) = sum_a k_a T_a - ks T_0 + c0 + c2 sqrt(T_0 + T_sat),
// with ks = sum of the conduction weights - C1 and c0 = C1 T_sat.  The next
// tile's raw inputs are staged in shared memory by cp.async (no registers).
// ============================================================================
enum : int { HK_OUT = 0, HK_SOLID = 1, HK_FLUID = 2, HK_BOTTOM = 3, HK_GHOST = 4 };

// 4-byte global -> shared copy that does not pass through registers
// (zero-filled and not read when !pred; src must still be a valid address)
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(pred ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// 16-byte global -> shared copy (zero-filled and not read when !pred; src
// must still be a valid, 16-byte aligned address)
__device__ __forceinline__ void cp_async16z(float *dst, const float *src, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(pred ? 16 : 0) : "memory");
}

// DF: the phase-change source of Eq. 24 in double-float arithmetic (the
// rho-only EOS factors, 1 / (rho c), div u and C1, C2 once per step; C1 T +
// C2 sqrt(T) per stage), everything else as in the FP32 kernel.
template <class P, int BW, int BY, int R, int MINB, bool WIDE, bool DF = false>
__global__ void __launch_bounds__(BW * BY, MINB)
k_heat_rows(const FParams p, int tiles_x, int ntiles, const typename P::tst *__restrict__ Tin,
            typename P::tst *__restrict__ Tout, const float *__restrict__ rho_i, const float *__restrict__ ux_i,
            const float *__restrict__ uy_i, const long long *__restrict__ stepp, unsigned *__restrict__ err) {
    constexpr int H = 4, SH = R * BY, TXO = BW - 2 * H, TYO = SH - 2 * H;
    static_assert(BW % 32 == 0, "a warp must cover whole columns of one row strip");
    __shared__ float sT[2][SH][BW];
    // 1/lambda, u_x, u_y of the tile for the coefficient pass; afterwards the
    // same arrays (and gV) stage the next tile's raw T, rho, u_x, u_y, each
    // cell's slot written and read by its owning thread only
    __shared__ float sL[SH][BW], sU[SH][BW], sV[SH][BW], gV[SH][BW];
    const int tx = threadIdx.x, ty = threadIdx.y, y0 = R * ty;
    const int nx = p.nx, nt = p.nt, ns = p.ns;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool model_a = (p.flags & FLAG_MODEL_A) != 0;
    const bool iso = (p.flags & FLAG_ISOTHERMAL) != 0;
    const float tsat = p.T_sat;
    unsigned errbits = 0;

    float Tn[R], Tc[R], acc[R], kk[R][8], ks[R], c0[R], c2[R];
    dfloat C1d[R], C2d[R];  // DF: the source coefficients in double-float
    int pk = 0, px = 0;  // kinds of the staged cells (3 bits per cell) and their column

    const int gdx = (int)gridDim.x % tiles_x, gdy = (int)gridDim.x / tiles_x;
    // a tile whose rows are all fluid rows (walled domains): every cell is
    // HK_FLUID, so the kind logic drops out of its fetch, load and
    // coefficient passes
    auto interior = [&](int tyt) {
        const int rlo = tyt * TYO - H;
        return !py && rlo >= ns && rlo + SH <= nt;
    };
    auto fetch_tile = [&](int txt, int tyt, auto itag) {
        constexpr bool I = decltype(itag)::value;
        const int x0 = txt * TXO, r0 = tyt * TYO;
        const int x = WIDE ? wrap1(x0 + tx - H, nx) : wrapi(x0 + tx - H, nx);
        px = x;
        pk = 0;
        #pragma unroll
        for (int c = 0; c < R; c++) {
            int row = r0 + y0 + c - H, k;
            if (I) k = HK_FLUID;
            else if (py) { row = WIDE ? wrap1(row, nt) : wrapi(row, nt); k = HK_FLUID; }
            else if (row < 0 || row > nt) k = HK_OUT;
            else if (row == 0) k = HK_BOTTOM;
            else if (row == nt) k = HK_GHOST;
            else k = (row < ns) ? HK_SOLID : HK_FLUID;
            pk |= k << (3 * c);
            const bool inT = k == HK_SOLID || k == HK_FLUID, fl = k == HK_FLUID, gh = k == HK_GHOST;
            const bool wa = k == HK_BOTTOM && model_a;  // Model A wall row: rho of the first fluid row
            const int kt = inT ? row * nx + x : 0;                                   // T index
            const int kf = fl ? kt - ns * nx : (gh ? (nt - ns - 1) * nx + x : (wa ? x : 0));  // fluid index
            cp_async4(&sL[y0 + c][tx], Tin + kt, inT);
            cp_async4(&sU[y0 + c][tx], rho_i + kf, fl || gh || wa);
            cp_async4(&sV[y0 + c][tx], ux_i + kf, fl);
            cp_async4(&gV[y0 + c][tx], uy_i + kf, fl);
        }
    };
    auto fetch = [&](int txt, int tyt) {
        if (interior(tyt)) fetch_tile(txt, tyt, std::true_type{});
        else fetch_tile(txt, tyt, std::false_type{});
    };
    const float w1 = 1.0f / 9.0f, w2 = 1.0f / 36.0f;
    int cxt = (int)blockIdx.x % tiles_x, cyt = (int)blockIdx.x / tiles_x;
    if ((int)blockIdx.x < ntiles) fetch(cxt, cyt);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int nxt = cxt + gdx, nyt = cyt + gdy;
        if (nxt >= tiles_x) { nxt -= tiles_x; nyt += 1; }
        const bool more = tile + (int)gridDim.x < ntiles;
        // neighbour columns and rows, clamped into the tile (edge cells compute
        // values nobody reads from them)
        const int xl = tx > 0 ? tx - 1 : 0, xr = tx < BW - 1 ? tx + 1 : BW - 1;
        const int yb = y0 > 0 ? y0 - 1 : 0, yt = y0 + R < SH ? y0 + R : SH - 1;
        // rows y0 - 1 .. y0 + R of column x - 1 / x + 1 (index j = row - y0 + 1)
        auto column = [&](const float (*a)[BW], int x, float *v) {
            v[0] = a[yb][x];
            #pragma unroll
            for (int j = 0; j < R; j++) v[j + 1] = a[y0 + j][x];
            v[R + 1] = a[yt][x];
        };
        // ---- load and per-step coefficients (interior tiles: compile-time fluid) ----
        auto prepare = [&](auto itag) {
        constexpr bool I = decltype(itag)::value;
        int kd[R];
        float irc[R], rho[R], ux[R], uy[R], lam[R];
        cp_async_wait_all();
        #pragma unroll
        for (int c = 0; c < R; c++) {
            const float Tr = sL[y0 + c][tx];
            rho[c] = sU[y0 + c][tx]; ux[c] = sV[y0 + c][tx]; uy[c] = gV[y0 + c][tx];
            const int k = I ? (int)HK_FLUID : (pk >> (3 * c)) & 7;
            kd[c] = k;
            float T = Tr, l = 0.0f, rc = 1.0f;
            if (k == HK_SOLID) { l = p.lambda_s; rc = p.rho_c_s; }
            else if (k == HK_FLUID) { l = p.cv_chi * rho[c]; rc = rho[c] * p.c_v; }
            else if (k == HK_BOTTOM) { T = bottom_theta(p, px, *stepp); l = model_a ? p.cv_chi * rho[c] : p.lambda_s; }
            else if (k == HK_GHOST) l = p.cv_chi * rho[c];
            Tn[c] = T; Tc[c] = T; irc[c] = fast_rcp(rc);
            // 1/lambda: the harmonic mean of a link is 2 / (1/l0 + 1/la)
            lam[c] = (l > 0.0f) ? fast_rcp(l) : 1e30f;
            sT[0][y0 + c][tx] = T;
            sT[1][y0 + c][tx] = T;
            sL[y0 + c][tx] = lam[c];
            sU[y0 + c][tx] = ux[c];
            sV[y0 + c][tx] = uy[c];
        }
        __syncthreads();
        // ---- per-step coefficients (neighbour order E, N, W, S, NE, NW, SW, SE) ----
        {
            // conduction: 6 w_a lambda_face / (rho c), lambda_face = 2 / (1/l0 + 1/la)
            float Ll[R + 2], Lr[R + 2];
            column(sL, xl, Ll);
            column(sL, xr, Lr);
            const float Lb = sL[yb][tx], Lt = sL[yt][tx];
            #pragma unroll
            for (int c = 0; c < R; c++) {
                const float l0 = lam[c];
                const float lN = c + 1 < R ? lam[c + 1] : Lt, lS = c > 0 ? lam[c - 1] : Lb;
                const int k = kd[c];
                const bool moves = (k == HK_SOLID || k == HK_FLUID) && !iso;
                const float f12 = moves ? 12.0f * irc[c] : 0.0f;
                const float cax = w1 * f12, cdg = w2 * f12;
                kk[c][0] = cax * fast_rcp(l0 + Lr[c + 1]);
                kk[c][1] = cax * fast_rcp(l0 + lN);
                kk[c][2] = cax * fast_rcp(l0 + Ll[c + 1]);
                kk[c][3] = cax * fast_rcp(l0 + lS);
                kk[c][4] = cdg * fast_rcp(l0 + Lr[c + 2]);
                kk[c][5] = cdg * fast_rcp(l0 + Ll[c + 2]);
                kk[c][6] = cdg * fast_rcp(l0 + Ll[c]);
                kk[c][7] = cdg * fast_rcp(l0 + Lr[c]);
                ks[c] = ((kk[c][0] + kk[c][1]) + (kk[c][2] + kk[c][3])) + ((kk[c][4] + kk[c][5]) + (kk[c][6] + kk[c][7]));
                c0[c] = 0.0f;
                c2[c] = 0.0f;
                C1d[c] = C2d[c] = df_from(0.0f);
                acc[c] = 0.0f;
            }
        }
        bool any_fluid = false;
        #pragma unroll
        for (int c = 0; c < R; c++) any_fluid |= kd[c] == HK_FLUID;
        if (!iso && any_fluid) {
            // advection (-u . grad T = sum_a adv_a T_a, adv_a = -3 w_a (e_a . u))
            // and the (dp/dT)_rho div u source of Eq. 24, with the Eq. 27 gradient
            float dd[R];
            [[maybe_unused]] dfloat Dd[R];  // DF: the same divergence sum in double-float
            const dfloat dw1 = {p.df_w1[0], p.df_w1[1]}, dw2 = {p.df_w2[0], p.df_w2[1]};
            auto ddiff = [](float a, float b) { return df_two_sum(a, -b); };  // a - b exactly
            {
                float Ul[R + 2], Ur[R + 2];
                column(sU, xl, Ul);
                column(sU, xr, Ur);
                #pragma unroll
                for (int c = 0; c < R; c++) {
                    dd[c] = w1 * (Ur[c + 1] - Ul[c + 1]) + w2 * ((Ur[c + 2] - Ul[c]) + (Ur[c] - Ul[c + 2]));
                    if constexpr (DF)
                        Dd[c] = df_add(df_mul(dw1, ddiff(Ur[c + 1], Ul[c + 1])),
                                       df_mul(dw2, df_add(ddiff(Ur[c + 2], Ul[c]), ddiff(Ur[c], Ul[c + 2]))));
                }
            }
            {
                float Vl[R + 2], Vr[R + 2];
                column(sV, xl, Vl);
                column(sV, xr, Vr);
                const float Vb = sV[yb][tx], Vt = sV[yt][tx];
                #pragma unroll
                for (int c = 0; c < R; c++) {
                    const float vN = c + 1 < R ? uy[c + 1] : Vt, vS = c > 0 ? uy[c - 1] : Vb;
                    dd[c] += w1 * (vN - vS) + w2 * ((Vr[c + 2] - Vl[c]) - (Vr[c] - Vl[c + 2]));
                    if constexpr (DF)
                        Dd[c] = df_add(Dd[c], df_add(df_mul(dw1, ddiff(vN, vS)),
                                                     df_mul(dw2, df_sub(ddiff(Vr[c + 2], Vl[c]), ddiff(Vr[c], Vl[c + 2])))));
                }
            }
            #pragma unroll
            for (int c = 0; c < R; c++) {
                if (kd[c] != HK_FLUID) continue;
                const float vx = -3.0f * ux[c], vy = -3.0f * uy[c];
                kk[c][0] += w1 * vx;          // e = ( 1,  0)
                kk[c][1] += w1 * vy;          // e = ( 0,  1)
                kk[c][2] -= w1 * vx;          // e = (-1,  0)
                kk[c][3] -= w1 * vy;          // e = ( 0, -1)
                kk[c][4] += w2 * (vx + vy);   // e = ( 1,  1)
                kk[c][5] += w2 * (vy - vx);   // e = (-1,  1)
                kk[c][6] -= w2 * (vx + vy);   // e = (-1, -1)
                kk[c][7] += w2 * (vx - vy);   // e = ( 1, -1)
                const float divu = 3.0f * dd[c];
                const float r = rho[c];
                const float br = p.b * r;
                const float omb = 1.0f - br, den = 1.0f + br * (2.0f - br);
                const float iod = fast_rcp(omb * den);
                const float pa = p.a_kappa * r * r * (omb * iod);
                const float A = r * p.R * (den * iod) - pa * p.kappa_over_Tc;
                [[maybe_unused]] const float B = pa * p.B_coef;
                const float g0 = -divu * irc[c];
                [[maybe_unused]] const float C1 = g0 * A;
                if constexpr (DF) {
                    // (dp/dT)_rho = A + B / sqrt(T), C1 = -(3 D / (rho C_V)) A, C2 = -(3 D / (rho C_V)) B
                    const dfloat one = df_from(1.0f);
                    const dfloat db = {p.df_b[0], p.df_b[1]}, dR = {p.df_R[0], p.df_R[1]};
                    const dfloat dak = {p.df_akappa[0], p.df_akappa[1]}, dko = {p.df_koTc[0], p.df_koTc[1]};
                    const dfloat dBc = {p.df_Bcoef[0], p.df_Bcoef[1]}, dcv = {p.df_cv[0], p.df_cv[1]};
                    const dfloat bR = df_mul_f(db, r);
                    const dfloat iomb = df_rcp(df_sub(one, bR));
                    const dfloat iden = df_rcp(df_add(one, df_mul(bR, df_sub(df_from(2.0f), bR))));
                    const dfloat akr2 = df_mul(dak, df_two_prod(r, r));
                    const dfloat Ad = df_sub(df_mul(df_mul_f(dR, r), iomb), df_mul(akr2, df_mul(dko, iden)));
                    const dfloat Bd = df_mul(akr2, df_mul(dBc, iden));
                    const dfloat g0d = df_mul(df_mul_f(Dd[c], -3.0f), df_rcp(df_mul_f(dcv, r)));
                    C1d[c] = df_mul(g0d, Ad);
                    C2d[c] = df_mul(g0d, Bd);
                } else {
                    ks[c] -= C1;
                    c0[c] = C1 * tsat;
                    c2[c] = g0 * B;
                }
            }
        }
        };
        if (interior(cyt)) prepare(std::true_type{});
        else prepare(std::false_type{});
        // ---- four RK stages; stage s reads sT[s & 1], writes sT[(s + 1) & 1] ----
        if (!iso) {
            #pragma unroll
            for (int st = 0; st < 4; st++) {
                const int m = st + 1;
                const int rb = st & 1, wb = rb ^ 1;
                if (st > 0) __syncthreads();  // the previous stage's writes are visible
                // the coefficient arrays are no longer read: stage the next tile
                if (st == 1 && more) fetch(nxt, nyt);
                if (y0 + R - 1 < m || y0 >= SH - m) continue;  // whole warp outside the region
                float Tl[R + 2], Tr[R + 2];
                column(sT[rb], xl, Tl);
                column(sT[rb], xr, Tr);
                const float Tb = sT[rb][yb][tx], Tt = sT[rb][yt][tx];
                float h[R];
                #pragma unroll
                for (int c = 0; c < R; c++) {
                    const float t0 = Tc[c];
                    const float tN = c + 1 < R ? Tc[c + 1] : Tt, tS = c > 0 ? Tc[c - 1] : Tb;
                    // T_0 + T_sat > 0 in every cell whose value is used
                    float v;
                    if constexpr (DF) {
                        v = df_source(C1d[c], C2d[c], t0, dfloat{p.df_tsat[0], p.df_tsat[1]});
                    } else {
                        v = c0[c] + c2[c] * fast_sqrt(t0 + tsat);
                    }
                    v += kk[c][0] * Tr[c + 1] + kk[c][1] * tN + kk[c][2] * Tl[c + 1] + kk[c][3] * tS +
                         kk[c][4] * Tr[c + 2] + kk[c][5] * Tl[c + 2] + kk[c][6] * Tl[c] + kk[c][7] * Tr[c] - ks[c] * t0;
                    h[c] = v;
                }
                #pragma unroll
                for (int c = 0; c < R; c++) {
                    if (st == 0) { acc[c] = h[c]; Tc[c] = Tn[c] + 0.5f * h[c]; }
                    else if (st == 1) { acc[c] += 2.0f * h[c]; Tc[c] = Tn[c] + 0.5f * h[c]; }
                    else if (st == 2) { acc[c] += 2.0f * h[c]; Tc[c] = Tn[c] + h[c]; }
                    else acc[c] += h[c];
                    if (st < 3) sT[wb][y0 + c][tx] = Tc[c];
                }
            }
        } else if (more) {
            __syncthreads();  // the coefficient arrays are staged into next
            fetch(nxt, nyt);
        }
        // ---- write the tile (fixed cells have acc = 0) ----
        const int x0 = cxt * TXO, r0 = cyt * TYO;
        #pragma unroll
        for (int c = 0; c < R; c++) {
            const int hy = y0 + c;
            const int row = r0 + hy - H, xo = x0 + tx - H;
            if (tx >= H && tx < BW - H && hy >= H && hy < SH - H && row < nt && xo < nx) {
                const float v = Tn[c] + acc[c] * (1.0f / 6.0f);
                if (!(fabsf(v) < 1e30f)) errbits |= ERRW_NONFINITE_T;
                Tout[row * nx + xo] = v;
            }
        }
        __syncthreads();  // shared tiles are rewritten by the next tile
        cxt = nxt; cyt = nyt;
    }
    if (errbits) atomicOr(err, errbits);
}

template <class P, int BW, int BY, int R, int MINB, bool DF = false>
struct HeatRowsShape {
    static int grid_blocks;
    static cudaError_t prepare() {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_heat_rows<P, BW, BY, R, MINB, true, DF>, BW * BY, 0);
        if (e != cudaSuccess) return e;
        grid_blocks = sms * (per > 0 ? per : 1);
        return cudaSuccess;
    }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        constexpr int TXO = BW - 8, TYO = R * BY - 8;
        const int tx = (p.nx + TXO - 1) / TXO, ty = (p.nt + TYO - 1) / TYO;
        const int ntiles = tx * ty;
        const int g = ntiles < grid_blocks ? ntiles : grid_blocks;
        const bool wide = p.nx >= BW && (!(p.flags & FLAG_PERIODIC_Y) || p.nt >= R * BY);
        auto k = wide ? k_heat_rows<P, BW, BY, R, MINB, true, DF> : k_heat_rows<P, BW, BY, R, MINB, false, DF>;
        k<<<g, dim3(BW, BY), 0, s>>>(
            make_fparams(p), tx, ntiles, (const typename P::tst *)b.T_in, (typename P::tst *)b.T_out,
            (const float *)b.rho, (const float *)b.ux, (const float *)b.uy, b.step, b.err);
        return cudaGetLastError();
    }
};
template <class P, int BW, int BY, int R, int MINB, bool DF>
int HeatRowsShape<P, BW, BY, R, MINB, DF>::grid_blocks = 152;

// ============================================================================
// Heat kernel, FP32, paired columns.  The tiles, halo, strips and per-cell
// algebra of k_heat_rows (64-column tiles, R-row strips per thread), but each
// thread owns two columns of its strip, x and x + 32, and keeps every
// per-cell value as a float2 (column x in .x, x + 32 in .y).  The arithmetic
// then runs as packed FP32 instructions (one issue slot for two cells;
// reciprocals and roots stay scalar), and shared memory holds the tile as
// pairs (T[x], T[x + 32]) in slot x, so that a neighbour read is one 64-bit
// load.  The west pair of lane x is slot x - 1 and its east pair slot x + 1,
// taken modulo 32: lane 0 reads slot 31 and moves its .x (column 31, the
// west neighbour of column 32) into .y; lane 31 reads slot 0 and moves its
// .y (column 32, the east neighbour of column 31) into .x.  The other half of
// those two pairs stands for columns -1 and 64, outside the tile, and is
// read only by halo cells.
// ============================================================================

// The body of the paired heat kernel over tiles first, first + step, ...
// (below end) of a run: a persistent block of a single-run launch, or a
// block's contiguous share of a run in a multi-run launch; p may live in the
// constant bank or in shared memory.
// RAW: the next tile's T, rho, u_x, u_y arrive as whole rows in 16-byte
// cp.async chunks (four per row and array per thread pair of passes)
// instead of one 4-byte copy per cell and array; needs nx a multiple of 4
// and at least 64.
template <class P, int BY, int R, bool WIDE, bool RAW = false>
__device__ __forceinline__ void
heat_pair_body(const FParams &p, int tiles_x, int end, int first, int step, const typename P::tst *__restrict__ Tin,
               typename P::tst *__restrict__ Tout, const float *__restrict__ rho_i, const float *__restrict__ ux_i,
               const float *__restrict__ uy_i, const long long *__restrict__ stepp, unsigned *__restrict__ err,
               int ymirror = -1) {
    constexpr int HW = 32, BW = 2 * HW, NSL = HW, H = 4, SH = R * BY, TXO = BW - 2 * H, TYO = SH - 2 * H;
    __shared__ float2 sT[2][SH][NSL];
    // 1/lambda, u_x, u_y of the tile for the coefficient pass; afterwards the
    // same arrays (and gV) stage the next tile's raw T, rho, u_x, u_y, each
    // slot written and read by its owning thread only
    __shared__ __align__(16) float2 sL[SH][NSL], sU[SH][NSL], sV[SH][NSL], gV[SH][NSL];
    const int tx = threadIdx.x, ty = threadIdx.y, y0 = R * ty;
    const int so = tx, sl = (tx + HW - 1) & (HW - 1), sr = (tx + 1) & (HW - 1);  // own, west, east slots
    const bool wrap_w = tx == 0, wrap_e = tx == HW - 1;  // lanes whose west / east pair is the wrapped one
    const int nx = p.nx, nt = p.nt, ns = p.ns;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool model_a = (p.flags & FLAG_MODEL_A) != 0;
    const bool iso = (p.flags & FLAG_ISOTHERMAL) != 0;
    const float tsat = p.T_sat;
    unsigned errbits = 0;

    float2 Tn[R], Tc[R], acc[R], kk[R][8], nks[R], c0[R], c2[R];
    int pk = 0, pxa = 0, pxb = 0;  // kinds of the staged rows (3 bits per row) and their columns

    const int gdx = step % tiles_x, gdy = step / tiles_x;
    auto interior = [&](int tyt) {
        const int rlo = tyt * TYO - H;
        return !py && rlo >= ns && rlo + SH <= nt;
    };
    auto fetch_tile = [&](int txt, int tyt, auto itag) {
        constexpr bool I = decltype(itag)::value;
        const int x0 = txt * TXO, r0 = tyt * TYO;
        const int xa = WIDE ? wrap1(x0 + tx - H, nx) : wrapi(x0 + tx - H, nx);
        const int xb = WIDE ? wrap1(x0 + tx + HW - H, nx) : wrapi(x0 + tx + HW - H, nx);
        pxa = xa;
        pxb = xb;
        pk = 0;
        if constexpr (RAW) {
            static_assert(R % 2 == 0 && WIDE, "whole-row staging: even strips, one column wrap");
            // this thread's chunks: column chunk q of rows tid / 16 + 2 BY h
            const int tid = ty * 32 + tx, q = tid & 15;
            int col = x0 - H + 4 * q;
            col = col < 0 ? col + nx : (col >= nx ? col - nx : col);
            #pragma unroll
            for (int h = 0; h < R / 2; h++) {
                const int hr = (tid >> 4) + 2 * BY * h;  // tile row
                int row = r0 + hr - H, k;
                if (I) k = HK_FLUID;
                else if (py) { row = row < 0 ? row + nt : (row >= nt ? row - nt : row); k = HK_FLUID; }
                else if (row < 0 || row > nt) k = HK_OUT;
                else if (row == 0) k = HK_BOTTOM;
                else if (row == nt) k = HK_GHOST;
                else k = (row < ns) ? HK_SOLID : HK_FLUID;
                const bool inT = k == HK_SOLID || k == HK_FLUID, fl = k == HK_FLUID, gh = k == HK_GHOST;
                const bool wa = k == HK_BOTTOM && model_a;
                const int kt = inT ? row * nx + col : 0;
                const int kf = fl ? kt - ns * nx : (gh ? (nt - ns - 1) * nx + col : (wa ? col : 0));
                float *dT = reinterpret_cast<float *>(&sL[0][0]) + hr * BW + 4 * q;
                float *dR = reinterpret_cast<float *>(&sU[0][0]) + hr * BW + 4 * q;
                float *dX = reinterpret_cast<float *>(&sV[0][0]) + hr * BW + 4 * q;
                float *dY = reinterpret_cast<float *>(&gV[0][0]) + hr * BW + 4 * q;
                cp_async16z(dT, Tin + kt, inT);
                cp_async16z(dR, rho_i + kf, fl || gh || wa);
                cp_async16z(dX, ux_i + kf, fl);
                cp_async16z(dY, uy_i + kf, fl);
            }
        }
        #pragma unroll
        for (int c = 0; c < R; c++) {
            int row = r0 + y0 + c - H, k;
            if (I) k = HK_FLUID;
            else if (py) { row = WIDE ? wrap1(row, nt) : wrapi(row, nt); k = HK_FLUID; }
            else if (row < 0 || row > nt) k = HK_OUT;
            else if (row == 0) k = HK_BOTTOM;
            else if (row == nt) k = HK_GHOST;
            else k = (row < ns) ? HK_SOLID : HK_FLUID;
            pk |= k << (3 * c);
            if constexpr (RAW) continue;  // (the rows were staged above)
            const bool inT = k == HK_SOLID || k == HK_FLUID, fl = k == HK_FLUID, gh = k == HK_GHOST;
            const bool wa = k == HK_BOTTOM && model_a;  // Model A wall row: rho of the first fluid row
            const int kta = inT ? row * nx + xa : 0, ktb = inT ? row * nx + xb : 0;
            const int kfa = fl ? kta - ns * nx : (gh ? (nt - ns - 1) * nx + xa : (wa ? xa : 0));
            const int kfb = fl ? ktb - ns * nx : (gh ? (nt - ns - 1) * nx + xb : (wa ? xb : 0));
            float *dL = &sL[y0 + c][so].x, *dU = &sU[y0 + c][so].x, *dV = &sV[y0 + c][so].x, *dW = &gV[y0 + c][so].x;
            cp_async4(dL, Tin + kta, inT);
            cp_async4(dL + 1, Tin + ktb, inT);
            cp_async4(dU, rho_i + kfa, fl || gh || wa);
            cp_async4(dU + 1, rho_i + kfb, fl || gh || wa);
            cp_async4(dV, ux_i + kfa, fl);
            cp_async4(dV + 1, ux_i + kfb, fl);
            cp_async4(dW, uy_i + kfa, fl);
            cp_async4(dW + 1, uy_i + kfb, fl);
        }
    };
    // tile rows in sequence order -> tile rows in the domain (ymirror >= 0:
    // the last tile row first, so that the sweep runs down the rows)
    auto ymap = [&](int tyt) { return ymirror >= 0 ? ymirror - tyt : tyt; };
    auto fetch = [&](int txt, int tyt) {
        tyt = ymap(tyt);
        if (interior(tyt)) fetch_tile(txt, tyt, std::true_type{});
        else fetch_tile(txt, tyt, std::false_type{});
    };
    const float w1 = 1.0f / 9.0f, w2 = 1.0f / 36.0f;
    int cxt = first % tiles_x, cyt = first / tiles_x;
    if (first < end) fetch(cxt, cyt);
    for (int tile = first; tile < end; tile += step) {
        int nxt = cxt + gdx, nyt = cyt + gdy;
        if (nxt >= tiles_x) { nxt -= tiles_x; nyt += 1; }
        const bool more = tile + step < end;
        // neighbour rows, clamped into the tile (edge cells compute values
        // nobody reads from them)
        const int yb = y0 > 0 ? y0 - 1 : 0, yt = y0 + R < SH ? y0 + R : SH - 1;
        // rows y0 - 1 .. y0 + R of the west / east neighbour pairs (index
        // j = row - y0 + 1), the wrapped halves moved into place
        auto west = [&](const float2 (*a)[NSL], float2 *v) {
            v[0] = a[yb][sl];
            #pragma unroll
            for (int j = 0; j < R; j++) v[j + 1] = a[y0 + j][sl];
            v[R + 1] = a[yt][sl];
            #pragma unroll
            for (int j = 0; j < R + 2; j++) v[j].y = wrap_w ? v[j].x : v[j].y;
        };
        auto east = [&](const float2 (*a)[NSL], float2 *v) {
            v[0] = a[yb][sr];
            #pragma unroll
            for (int j = 0; j < R; j++) v[j + 1] = a[y0 + j][sr];
            v[R + 1] = a[yt][sr];
            #pragma unroll
            for (int j = 0; j < R + 2; j++) v[j].x = wrap_e ? v[j].y : v[j].x;
        };
        // ---- load and per-step coefficients (interior tiles: compile-time fluid) ----
        auto prepare = [&](auto itag) {
        constexpr bool I = decltype(itag)::value;
        int kd[R];
        float2 irc[R], rho[R], ux[R], uy[R], lam[R], Tw[R];
        cp_async_wait_all();
        if constexpr (RAW) {
            __syncthreads();  // every thread's chunks have landed
            const float *rT = reinterpret_cast<const float *>(&sL[0][0]), *rR = reinterpret_cast<const float *>(&sU[0][0]);
            const float *rX = reinterpret_cast<const float *>(&sV[0][0]), *rY = reinterpret_cast<const float *>(&gV[0][0]);
            #pragma unroll
            for (int c = 0; c < R; c++) {
                const int o = (y0 + c) * BW + tx;
                Tw[c] = make_float2(rT[o], rT[o + HW]);
                rho[c] = make_float2(rR[o], rR[o + HW]);
                ux[c] = make_float2(rX[o], rX[o + HW]);
                uy[c] = make_float2(rY[o], rY[o + HW]);
            }
            __syncthreads();  // read before the arrays take the coefficients
        } else {
            #pragma unroll
            for (int c = 0; c < R; c++) {
                Tw[c] = sL[y0 + c][so];
                rho[c] = sU[y0 + c][so]; ux[c] = sV[y0 + c][so]; uy[c] = gV[y0 + c][so];
            }
        }
        #pragma unroll
        for (int c = 0; c < R; c++) {
            const float2 Tr = Tw[c];
            const int k = I ? (int)HK_FLUID : (pk >> (3 * c)) & 7;
            kd[c] = k;
            Tn[c] = Tr; Tc[c] = Tr;
            if (k == HK_FLUID) {
                // 1 / (rho c_v) and 1 / lambda = 1 / (C_V chi rho) from one reciprocal of rho
                const float2 ir = rcp2(rho[c]);
                irc[c] = mul2(ir, f2(p.inv_c_v));
                lam[c] = mul2(ir, f2(p.inv_cv_chi));
                continue;
            }
            float2 T = Tr, l = f2(0.0f), rc = f2(1.0f);
            if (k == HK_SOLID) { l = f2(p.lambda_s); rc = f2(p.rho_c_s); }
            else if (k == HK_BOTTOM) {
                const long long n = *stepp;
                T = make_float2(bottom_theta(p, pxa, n), bottom_theta(p, pxb, n));
                l = model_a ? mul2(f2(p.cv_chi), rho[c]) : f2(p.lambda_s);
            }
            else if (k == HK_GHOST) l = mul2(f2(p.cv_chi), rho[c]);
            Tn[c] = T; Tc[c] = T; irc[c] = rcp2(rc);
            // 1/lambda: the harmonic mean of a link is 2 / (1/l0 + 1/la)
            lam[c] = make_float2(l.x > 0.0f ? fast_rcp(l.x) : 1e30f, l.y > 0.0f ? fast_rcp(l.y) : 1e30f);
        }
        #pragma unroll
        for (int c = 0; c < R; c++) {
            sT[0][y0 + c][so] = Tn[c];
            sT[1][y0 + c][so] = Tn[c];
            sL[y0 + c][so] = lam[c];
            sU[y0 + c][so] = ux[c];
            sV[y0 + c][so] = uy[c];
        }
        __syncthreads();
        // ---- per-step coefficients (neighbour order E, N, W, S, NE, NW, SW, SE) ----
        {
            // conduction: 6 w_a lambda_face / (rho c), lambda_face = 2 / (1/l0 + 1/la)
            float2 Ll[R + 2], Lr[R + 2];
            west(sL, Ll);
            east(sL, Lr);
            const float2 Lb = sL[yb][so], Lt = sL[yt][so];
            // the vertical link between rows c and c + 1 of the strip is the
            // north link of one and the south link of the other: one reciprocal
            float2 hN[R];
            #pragma unroll
            for (int c = 0; c < R; c++) hN[c] = rcp2(add2(lam[c], c + 1 < R ? lam[c + 1] : Lt));
            const float2 hS0 = rcp2(add2(lam[0], Lb));
            // likewise the east link of a cell is the west link of its east
            // neighbour, and the north-east (north-west) link the south-west
            // (south-east) link of the cell above it to the east (west): those
            // come from the neighbouring lane (the column pairs are x, x + 32,
            // so lane 0's second column meets lane 31's first).  Lane 0's first
            // and lane 31's second column are the tile's outermost halo
            // cells, whose coefficients no kept value depends on.
            float2 hE[R], hNE[R], hNW[R];
            #pragma unroll
            for (int c = 0; c < R; c++) {
                hE[c] = rcp2(add2(lam[c], Lr[c + 1]));
                hNE[c] = rcp2(add2(lam[c], Lr[c + 2]));
                hNW[c] = rcp2(add2(lam[c], Ll[c + 2]));
            }
            auto from_west = [&](float2 v) {  // v of the west neighbour's column pair
                const float a = __shfl_up_sync(0xffffffffu, v.x, 1), b = __shfl_up_sync(0xffffffffu, v.y, 1);
                const float w = __shfl_sync(0xffffffffu, v.x, HW - 1);
                return make_float2(a, wrap_w ? w : b);
            };
            auto from_east = [&](float2 v) {  // v of the east neighbour's column pair
                const float a = __shfl_down_sync(0xffffffffu, v.x, 1), b = __shfl_down_sync(0xffffffffu, v.y, 1);
                const float e = __shfl_sync(0xffffffffu, v.y, 0);
                return make_float2(wrap_e ? e : a, b);
            };
            #pragma unroll
            for (int c = 0; c < R; c++) {
                const float2 l0 = lam[c];
                const int k = kd[c];
                const bool moves = (k == HK_SOLID || k == HK_FLUID) && !iso;
                const float2 f12 = moves ? mul2(f2(12.0f), irc[c]) : f2(0.0f);
                const float2 cax = mul2(f2(w1), f12), cdg = mul2(f2(w2), f12);
                kk[c][0] = mul2(cax, hE[c]);
                kk[c][1] = mul2(cax, hN[c]);
                kk[c][2] = mul2(cax, from_west(hE[c]));
                kk[c][3] = mul2(cax, c > 0 ? hN[c - 1] : hS0);
                kk[c][4] = mul2(cdg, hNE[c]);
                kk[c][5] = mul2(cdg, hNW[c]);
                kk[c][6] = mul2(cdg, c > 0 ? from_west(hNE[c - 1]) : rcp2(add2(l0, Ll[c])));
                kk[c][7] = mul2(cdg, c > 0 ? from_east(hNW[c - 1]) : rcp2(add2(l0, Lr[c])));
                const float2 ks = add2(add2(add2(kk[c][0], kk[c][1]), add2(kk[c][2], kk[c][3])),
                                       add2(add2(kk[c][4], kk[c][5]), add2(kk[c][6], kk[c][7])));
                nks[c] = mul2(ks, f2(-1.0f));
                c0[c] = f2(0.0f);
                c2[c] = f2(0.0f);
                acc[c] = f2(0.0f);
            }
        }
        bool any_fluid = false;
        #pragma unroll
        for (int c = 0; c < R; c++) any_fluid |= kd[c] == HK_FLUID;
        if (!iso && any_fluid) {
            // advection (-u . grad T = sum_a adv_a T_a, adv_a = -3 w_a (e_a . u))
            // and the (dp/dT)_rho div u source of Eq. 24, with the Eq. 27 gradient
            float2 dd[R];
            {
                float2 Ul[R + 2], Ur[R + 2];
                west(sU, Ul);
                east(sU, Ur);
                #pragma unroll
                for (int c = 0; c < R; c++)
                    dd[c] = fma2(f2(w1), sub2(Ur[c + 1], Ul[c + 1]),
                                 mul2(f2(w2), add2(sub2(Ur[c + 2], Ul[c]), sub2(Ur[c], Ul[c + 2]))));
            }
            {
                float2 Vl[R + 2], Vr[R + 2];
                west(sV, Vl);
                east(sV, Vr);
                const float2 Vb = sV[yb][so], Vt = sV[yt][so];
                #pragma unroll
                for (int c = 0; c < R; c++) {
                    const float2 vN = c + 1 < R ? uy[c + 1] : Vt, vS = c > 0 ? uy[c - 1] : Vb;
                    dd[c] = add2(dd[c], fma2(f2(w1), sub2(vN, vS),
                                             mul2(f2(w2), sub2(sub2(Vr[c + 2], Vl[c]), sub2(Vr[c], Vl[c + 2])))));
                }
            }
            #pragma unroll
            for (int c = 0; c < R; c++) {
                if (kd[c] != HK_FLUID) continue;
                const float2 vx = mul2(f2(-3.0f), ux[c]), vy = mul2(f2(-3.0f), uy[c]);
                kk[c][0] = fma2(f2(w1), vx, kk[c][0]);            // e = ( 1,  0)
                kk[c][1] = fma2(f2(w1), vy, kk[c][1]);            // e = ( 0,  1)
                kk[c][2] = fma2(f2(-w1), vx, kk[c][2]);           // e = (-1,  0)
                kk[c][3] = fma2(f2(-w1), vy, kk[c][3]);           // e = ( 0, -1)
                kk[c][4] = fma2(f2(w2), add2(vx, vy), kk[c][4]);  // e = ( 1,  1)
                kk[c][5] = fma2(f2(w2), sub2(vy, vx), kk[c][5]);  // e = (-1,  1)
                kk[c][6] = fma2(f2(-w2), add2(vx, vy), kk[c][6]); // e = (-1, -1)
                kk[c][7] = fma2(f2(w2), sub2(vx, vy), kk[c][7]);  // e = ( 1, -1)
                const float2 r = rho[c];
                const float2 br = mul2(f2(p.b), r);
                const float2 omb = sub2(f2(1.0f), br), den = fma2(br, sub2(f2(2.0f), br), f2(1.0f));
                const float2 iod = rcp2(mul2(omb, den));
                const float2 pa = mul2(mul2(f2(p.a_kappa), mul2(r, r)), mul2(omb, iod));
                const float2 A = fma2(pa, f2(-p.kappa_over_Tc), mul2(mul2(r, f2(p.R)), mul2(den, iod)));
                const float2 B = mul2(pa, f2(p.B_coef));
                const float2 g0 = mul2(mul2(f2(-3.0f), dd[c]), irc[c]);  // -div u / (rho c)
                const float2 C1 = mul2(g0, A);
                nks[c] = add2(nks[c], C1);
                c0[c] = mul2(C1, f2(tsat));
                c2[c] = mul2(g0, B);
            }
        }
        };
        if (interior(ymap(cyt))) prepare(std::true_type{});
        else prepare(std::false_type{});
        // ---- four RK stages; stage s reads sT[s & 1], writes sT[(s + 1) & 1] ----
        if (!iso) {
            #pragma unroll
            for (int st = 0; st < 4; st++) {
                const int m = st + 1;
                const int rb = st & 1, wb = rb ^ 1;
                if (st > 0) __syncthreads();  // the previous stage's writes are visible
                // the coefficient arrays are no longer read: stage the next tile
                if (st == 1 && more) fetch(nxt, nyt);
                if (y0 + R - 1 < m || y0 >= SH - m) continue;  // whole warp outside the region
                float2 Tl[R + 2], Tr[R + 2];
                west(sT[rb], Tl);
                east(sT[rb], Tr);
                const float2 Tb = sT[rb][yb][so], Tt = sT[rb][yt][so];
                float2 h[R];
                #pragma unroll
                for (int c = 0; c < R; c++) {
                    const float2 t0 = Tc[c];
                    const float2 tN = c + 1 < R ? Tc[c + 1] : Tt, tS = c > 0 ? Tc[c - 1] : Tb;
                    // T_0 + T_sat > 0 in every cell whose value is used
                    const float2 u = add2(t0, f2(tsat));
                    float2 v = fma2(c2[c], make_float2(fast_sqrt(u.x), fast_sqrt(u.y)), c0[c]);
                    v = fma2(kk[c][0], Tr[c + 1], v);
                    v = fma2(kk[c][1], tN, v);
                    v = fma2(kk[c][2], Tl[c + 1], v);
                    v = fma2(kk[c][3], tS, v);
                    v = fma2(kk[c][4], Tr[c + 2], v);
                    v = fma2(kk[c][5], Tl[c + 2], v);
                    v = fma2(kk[c][6], Tl[c], v);
                    v = fma2(kk[c][7], Tr[c], v);
                    h[c] = fma2(nks[c], t0, v);
                }
                #pragma unroll
                for (int c = 0; c < R; c++) {
                    if (st == 0) { acc[c] = h[c]; Tc[c] = fma2(f2(0.5f), h[c], Tn[c]); }
                    else if (st == 1) { acc[c] = fma2(f2(2.0f), h[c], acc[c]); Tc[c] = fma2(f2(0.5f), h[c], Tn[c]); }
                    else if (st == 2) { acc[c] = fma2(f2(2.0f), h[c], acc[c]); Tc[c] = add2(Tn[c], h[c]); }
                    else acc[c] = add2(acc[c], h[c]);
                    if (st < 3) sT[wb][y0 + c][so] = Tc[c];
                }
            }
        } else if (more) {
            __syncthreads();  // the coefficient arrays are staged into next
            fetch(nxt, nyt);
        }
        // ---- write the tile (fixed cells have acc = 0) ----
        const int x0 = cxt * TXO, r0 = ymap(cyt) * TYO;
        const int xa = x0 + tx - H, xb = x0 + tx + HW - H;
        #pragma unroll
        for (int c = 0; c < R; c++) {
            const int hy = y0 + c;
            const int row = r0 + hy - H;
            if (hy >= H && hy < SH - H && row < nt) {
                const float2 v = fma2(acc[c], f2(1.0f / 6.0f), Tn[c]);
                if (tx >= H && xa < nx) {
                    if (!(fabsf(v.x) < 1e30f)) errbits |= ERRW_NONFINITE_T;
                    Tout[row * nx + xa] = v.x;
                }
                if (tx + HW < BW - H && xb < nx) {
                    if (!(fabsf(v.y) < 1e30f)) errbits |= ERRW_NONFINITE_T;
                    Tout[row * nx + xb] = v.y;
                }
            }
        }
        __syncthreads();  // shared tiles are rewritten by the next tile
        cxt = nxt; cyt = nyt;
    }
    if (errbits) atomicOr(err, errbits);
}


template <class P, int BY, int R, int MINB, bool WIDE, bool RAW = false>
__global__ void __launch_bounds__(32 * BY, MINB)
k_heat_pair(const __grid_constant__ FParams p, int tiles_x, int ntiles, const typename P::tst *__restrict__ Tin,
            typename P::tst *__restrict__ Tout, const float *__restrict__ rho_i, const float *__restrict__ ux_i,
            const float *__restrict__ uy_i, const long long *__restrict__ stepp, unsigned *__restrict__ err,
            int ymirror) {
    heat_pair_body<P, BY, R, WIDE, RAW>(p, tiles_x, ntiles, (int)blockIdx.x, (int)gridDim.x, Tin, Tout, rho_i, ux_i,
                                        uy_i, stepp, err, ymirror);
}

// DOWN: the tiles are taken from the top tile row down, so that the rows the
// flow kernel (sweeping up) wrote last are read first, while they are still
// in L2, and the next flow kernel finds the bottom rows of T there.
template <class P, int BY, int R, int MINB, bool RAW = false, bool DOWN = false>
struct HeatPairShape {
    static int grid_blocks;
    static cudaError_t prepare() {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_heat_pair<P, BY, R, MINB, true, RAW>, 32 * BY, 0);
        if (e != cudaSuccess) return e;
        grid_blocks = sms * (per > 0 ? per : 1);
        return cudaSuccess;
    }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        constexpr int TXO = 64 - 8, TYO = R * BY - 8;
        const int tx = (p.nx + TXO - 1) / TXO, ty = (p.nt + TYO - 1) / TYO;
        const int ntiles = tx * ty;
        const int g = ntiles < grid_blocks ? ntiles : grid_blocks;
        const bool wide = p.nx >= 64 && (!(p.flags & FLAG_PERIODIC_Y) || p.nt >= R * BY);
        // whole-row staging: whole 16-byte chunks (nx a multiple of 4), one column wrap
        auto k = (RAW && wide && p.nx % 4 == 0) ? k_heat_pair<P, BY, R, MINB, true, RAW>
                 : wide                       ? k_heat_pair<P, BY, R, MINB, true>
                                              : k_heat_pair<P, BY, R, MINB, false>;
        k<<<g, dim3(32, BY), 0, s>>>(
            make_fparams(p), tx, ntiles, (const typename P::tst *)b.T_in, (typename P::tst *)b.T_out,
            (const float *)b.rho, (const float *)b.ux, (const float *)b.uy, b.step, b.err,
            DOWN ? ty - 1 : -1);
        return cudaGetLastError();
    }
};
template <class P, int BY, int R, int MINB, bool RAW, bool DOWN>
int HeatPairShape<P, BY, R, MINB, RAW, DOWN>::grid_blocks = 152;

}  // namespace lbmgb

namespace lbmgb {

// Diagnostics kernel, FP32 path, single pass: every global load is issued
// before the first reduction, then one block-wide reduction of four sums.
template <class P, int NT>
__device__ __forceinline__ void
diag_flat_body(const FParams &p, const float *__restrict__ T, const float *__restrict__ rho,
               const double *__restrict__ part, int nblk, double *__restrict__ q_top, double *__restrict__ series,
               int cap, double *__restrict__ last, long long *__restrict__ stepp, double inv_nx, double inv_nfl) {
    __shared__ double sh[4][NT / 32];
    const int nx = p.nx, ns = p.ns, t = threadIdx.x;
    const bool model_a = (p.flags & FLAG_MODEL_A) != 0;  // no heater: wall flux for both
    const bool flux = !(p.flags & FLAG_PERIODIC_Y) && (ns >= 3 || model_a);
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // mass, vapour count, bottom flux, surface flux
    for (int b = t; b < nblk; b += NT) {
        v[0] += part[2 * b];
        v[1] += part[2 * b + 1];
    }
    if (flux) {
        const float lams = p.lambda_s, cvchi = p.cv_chi;
        for (int x = t; x < nx; x += NT) {
            const float t0 = T[x], t1 = T[nx + x], t2 = T[2 * nx + x];
            const float tu = T[(size_t)ns * nx + x], td = T[(size_t)(ns - 1) * nx + x];
            const float lf1 = cvchi * rho[x], lw = model_a ? lf1 : lams;
            // the face flux, and Eq. 36 (theta differences: T_sat cancels)
            const float lf = 2.0f * lw * lf1 * fast_rcp(lw + lf1);
            const float q = -lf * (tu - td);
            const float qb = model_a ? q : -lams * (0.5f * ((4.0f * t1 - t2) - 3.0f * t0));
            q_top[x] = (double)q;
            v[2] += (double)qb;
            v[3] += (double)q;
        }
    }
    #pragma unroll
    for (int k = 0; k < 4; k++) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if ((t & 31) == 0) {
        #pragma unroll
        for (int k = 0; k < 4; k++) sh[k][t >> 5] = v[k];
    }
    __syncthreads();
    if (t < 32) {
        #pragma unroll
        for (int k = 0; k < 4; k++) {
            double s = (t < NT / 32) ? sh[k][t] : 0.0;
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[k] = s;
        }
        if (t == 0) {
            const long long n = *stepp;
            const double out[SERIES_WIDTH] = {v[2] * inv_nx, v[3] * inv_nx, v[1] * inv_nfl, v[0]};
            const long long slot = n % cap;
            #pragma unroll
            for (int k = 0; k < SERIES_WIDTH; k++) {
                series[slot * SERIES_WIDTH + k] = out[k];
                last[k] = out[k];
            }
            *stepp = n + 1;
        }
    }
}

template <class P, int NT>
__global__ void __launch_bounds__(NT)
k_diag_flat(const __grid_constant__ FParams p, const float *__restrict__ T, const float *__restrict__ rho,
            const double *__restrict__ part, int nblk, double *__restrict__ q_top, double *__restrict__ series,
            int cap, double *__restrict__ last, long long *__restrict__ stepp, double inv_nx, double inv_nfl) {
    diag_flat_body<P, NT>(p, T, rho, part, nblk, q_top, series, cap, last, stepp, inv_nx, inv_nfl);
}

template <class P, int NT>
cudaError_t launch_diag_flat(const DevParams &p, const StepBuffers &b, int nblk, cudaStream_t s) {
    k_diag_flat<P, NT><<<1, NT, 0, s>>>(make_fparams(p), (const float *)b.T_out, (const float *)b.rho, b.part, nblk,
                                        b.q_top, b.series, b.series_cap, b.last, b.step, 1.0 / (double)p.nx,
                                        1.0 / ((double)p.nx * (double)p.nf));
    return cudaGetLastError();
}

}  // namespace lbmgb
