// Heat kernel, FP32, row wavefront (Sec. 2.2: one RK4 step, Eq. 25-26, of
// Eq. 24 with the isotropic differences of Eq. 27-28, rho and u frozen).
//
// Each warp owns a strip of 32 CL adjacent columns (CL = 1: one column per
// lane; CL = 2: two adjacent columns per lane, updated as packed FP32 pairs)
// and marches up a segment of rows.  Row j of the inputs arrives, and in the
// same iteration
//   - the conduction links between rows j - 1 and j are formed (each link's
//     harmonic-mean conductance is computed once and handed to both cells:
//     four reciprocals per cell instead of eight),
//   - the per-step coefficients of row j - 1 are completed (link weights with
//     the advection of Eq. 27 folded in, the phase-change source of Eq. 24
//     as C1 T + C2 sqrt(T) with (dp/dT)_rho = A(rho) + B(rho) / sqrt(T)),
//   - stage 1 runs on row j - 1, stage 2 on row j - 2, stage 3 on row j - 3
//     and stage 4 on row j - 4, whose new temperature is stored.
// A stage needs the previous stage on the rows above and below, which is
// why the stages trail each other by one row.  Everything a row needs until
// its fourth stage stays in registers (rings of four rows); the east and
// west neighbours come from the adjacent lanes by warp shuffles.  There is
// no shared memory, no block barrier and no halo in the row direction; the
// four columns at each side of a strip are halo (their results are
// recomputed by the neighbouring strips), and a segment starts four rows
// early and ends four rows late to fill and drain the pipeline.
#pragma once
#include <type_traits>

#include "lbm_fast.cuh"

namespace lbmgb {

// Per-lane column vectors: CL = 1, one column per lane (float); CL = 2, two
// adjacent columns per lane (float2, packed FP32 instructions; reciprocals and
// roots stay scalar).
template <int CL> struct LaneVec;
template <> struct LaneVec<1> {
    using V = float;
    static __device__ __forceinline__ V set(float a) { return a; }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
    static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ V rcp(V a) { return fast_rcp(a); }
    static __device__ __forceinline__ V sqrt(V a) { return fast_sqrt(a); }
    // the value at the column to the west / east (from the adjacent lane)
    static __device__ __forceinline__ V west(V a) { return __shfl_up_sync(0xffffffffu, a, 1); }
    static __device__ __forceinline__ V east(V a) { return __shfl_down_sync(0xffffffffu, a, 1); }
    static __device__ __forceinline__ float get(V a, int) { return a; }
    static __device__ __forceinline__ void put(V &a, int, float v) { a = v; }
    static __device__ __forceinline__ V c(float2 v) { return v.x; }
};
template <> struct LaneVec<2> {
    using V = float2;
    static __device__ __forceinline__ V set(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V rcp(V a) { return make_float2(fast_rcp(a.x), fast_rcp(a.y)); }
    static __device__ __forceinline__ V sqrt(V a) { return make_float2(fast_sqrt(a.x), fast_sqrt(a.y)); }
    // columns (2l - 1, 2l) and (2l + 1, 2l + 2) of lane l
    static __device__ __forceinline__ V west(V a) { return make_float2(__shfl_up_sync(0xffffffffu, a.y, 1), a.x); }
    static __device__ __forceinline__ V east(V a) { return make_float2(a.y, __shfl_down_sync(0xffffffffu, a.x, 1)); }
    static __device__ __forceinline__ float get(V a, int h) { return h ? a.y : a.x; }
    static __device__ __forceinline__ void put(V &a, int h, float v) { if (h) a.y = v; else a.x = v; }
    static __device__ __forceinline__ V c(float2 v) { return v; }
};

// The kernel's constants, each held in both halves of a pair and passed as a
// kernel parameter: packed instructions then read them from the constant
// bank instead of holding them in registers.
struct WaveConsts {
    float2 w1, w2, g1, g2, half, two, m3, sixth, tsat, cvchi, cv, b, one, akappa, mkoTc, R, Bcoef, zero;
};
inline WaveConsts make_wave_consts(const FParams &q) {
    auto d = [](float v) { return make_float2(v, v); };
    WaveConsts k;
    k.w1 = d(1.0f / 9.0f); k.w2 = d(1.0f / 36.0f);
    k.g1 = d(12.0f / 9.0f); k.g2 = d(12.0f / 36.0f);  // 6 w_a x 2 of the harmonic mean
    k.half = d(0.5f); k.two = d(2.0f); k.m3 = d(-3.0f); k.sixth = d(1.0f / 6.0f);
    k.tsat = d(q.T_sat); k.cvchi = d(q.cv_chi); k.cv = d(q.c_v); k.b = d(q.b); k.one = d(1.0f);
    k.akappa = d(q.a_kappa); k.mkoTc = d(-q.kappa_over_Tc); k.R = d(q.R); k.Bcoef = d(q.B_coef);
    k.zero = d(0.0f);
    return k;
}

// CL columns per lane; WPB warps per block (each warp independent); WIDE:
// nx >= 32 CL, so column wraps are one compare; VEC: CL = 2 and nx even, so a
// lane's two columns are adjacent in memory (64-bit loads and stores).
template <class P, int CL, int WPB, int MINB, int RS, bool WIDE, bool VEC>
__global__ void __launch_bounds__(32 * WPB, MINB)
k_heat_wave(const FParams p, const WaveConsts wk, int nstrips, int seg, int nunits, const typename P::tst *__restrict__ Tin,
            typename P::tst *__restrict__ Tout, const float *__restrict__ rho_i, const float *__restrict__ ux_i,
            const float *__restrict__ uy_i, const long long *__restrict__ stepp, unsigned *__restrict__ err) {
    using L = LaneVec<CL>;
    using V = typename L::V;
    constexpr int H = 4, SW = 32 * CL, OUTW = SW - 2 * H;
    static_assert(!VEC || CL == 2, "vector access is for column pairs");
    static_assert(RS >= 4 && (RS & (RS - 1)) == 0, "input ring: a power of two of at least four rows");
    const int lane = threadIdx.x & 31;
    const int unit = blockIdx.x * WPB + (int)(threadIdx.x >> 5);
    if (unit >= nunits) return;  // whole warps
    const int strip = unit % nstrips, sgi = unit / nstrips;
    const int nx = p.nx, nt = p.nt, ns = p.ns, nf = p.nf;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool model_a = (p.flags & FLAG_MODEL_A) != 0;
    const bool iso = (p.flags & FLAG_ISOTHERMAL) != 0;
    const float irc_s = fast_rcp(p.rho_c_s);  // used on heater rows only
    // this lane's columns; the H columns at each side of the strip are halo
    int xc[CL];
    bool wc[CL];
    #pragma unroll
    for (int h = 0; h < CL; h++) {
        const int l = CL * lane + h, xr = strip * OUTW - H + l;
        xc[h] = WIDE ? wrap1(xr, nx) : wrapi(xr, nx);
        wc[h] = l >= H && l < SW - H && xr < nx;
    }
    const int ys = sgi * seg, ye = min(ys + seg, nt);
    const int j0 = ys - H;                             // first row taken in
    const int nit = ((ye - ys) + 2 * H + 3) & ~3;      // rows taken in, padded to whole unrolled passes
    const long long n = *stepp;
    unsigned errbits = 0;

    auto kind = [&](int r) -> int {
        if (py) return HK_FLUID;
        if (r < 0 || r > nt) return HK_OUT;
        if (r == 0) return HK_BOTTOM;
        if (r == nt) return HK_GHOST;
        return r < ns ? HK_SOLID : HK_FLUID;
    };
    auto wrow = [&](int r) { return py ? wrapi(r, nt) : r; };
    // Inputs are staged by cp.async into a per-warp ring of RS row slots in
    // shared memory, RS - 1 rows ahead; each lane copies and reads only its
    // own columns, so no synchronisation beyond the copy groups is needed.
    // The slot a copy refills was read one iteration earlier.
    __shared__ __align__(16) V sbuf[WPB][RS][4][32];  // [warp][row slot][T, rho, u_x, u_y][lane]
    V (*wb)[4][32] = sbuf[threadIdx.x >> 5];
    auto cp = [&](V *dst, const float *base, int off, bool pred) {
        if constexpr (VEC) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(base + off + xc[0]),
                         "r"(pred ? 8 : 0) : "memory");
        } else {
            #pragma unroll
            for (int h = 0; h < CL; h++)
                cp_async4(reinterpret_cast<float *>(dst) + h, base + (pred ? off + xc[h] : 0), pred);
        }
    };
    // raw T, rho, u_x, u_y of row r into slot s (zero where the row has none)
    auto fetch = [&](int r, int s, auto itag) {
        constexpr bool I = decltype(itag)::value;
        const int k = I ? (int)HK_FLUID : kind(r), rr = I ? r : wrow(r);
        const bool inT = k == HK_SOLID || k == HK_FLUID, fl = k == HK_FLUID;
        // fluid row of rho: its own; the ghost row continues the top row's
        // conductivity; model A's wall row conducts like the first fluid row
        const int orho = fl ? (rr - ns) * nx : (k == HK_GHOST ? (nf - 1) * nx : 0);
        const bool prho = fl || k == HK_GHOST || (k == HK_BOTTOM && model_a);
        cp(&wb[s][0][lane], Tin, inT ? rr * nx : 0, inT);
        cp(&wb[s][1][lane], rho_i, orho, prho);
        cp(&wb[s][2][lane], ux_i, fl ? orho : 0, fl);
        cp(&wb[s][3][lane], uy_i, fl ? orho : 0, fl);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    const V w1 = L::c(wk.w1), w2 = L::c(wk.w2), g1 = L::c(wk.g1), g2 = L::c(wk.g2);
    const V zero = L::c(wk.zero), half = L::c(wk.half), two = L::c(wk.two), m3 = L::c(wk.m3);
    const V vtsat = L::c(wk.tsat);

    // k_a T_a over the 9-point stencil (a: E, N, W, S, NE, NW, SW, SE), plus
    // the centre and source terms: K = sum k_a T_a + nks T0 + c0 + c2 sqrt(T0 + T_sat)
    // The north row (T_N, T_NE, T_NW) is the newest input of every stage, so
    // its three terms come last: the rest of the sum is ready before it arrives.
    auto stencil = [&](const V *k, V T0, V TE, V TW, V TN, V TS, V TNE, V TNW, V TSW, V TSE) -> V {
        const V s = L::fma(k[10], L::sqrt(L::add(T0, vtsat)), k[9]);  // T0 + T_sat > 0 wherever used
        const V a = L::fma(k[0], TE, L::mul(k[2], TW));
        const V b = L::fma(k[6], TSW, L::fma(k[7], TSE, L::mul(k[3], TS)));
        const V old = L::add(L::fma(k[8], T0, s), L::add(a, b));
        return L::fma(k[5], TNW, L::fma(k[4], TNE, L::fma(k[1], TN, old)));
    };

    auto march = [&](auto itag) {
        constexpr bool I = decltype(itag)::value;
        // the first RS - 1 rows' inputs (slot = row mod RS relative to j0)
        #pragma unroll
        for (int q = 0; q < RS - 1; q++) fetch(j0 + q, q, itag);
        // rings of four rows (slot = row mod 4 relative to j0): T^n, stage
        // values Y1..Y3 with their west / east neighbours, the RK sum, and the
        // eleven coefficients of each row
        V Tn[4], TnW[4], TnE[4], Y1[4], Y1W[4], Y1E[4], Y2[4], Y2W[4], Y2E[4], Y3[4], Y3W[4], Y3E[4], acc[4];
        V K[4][11];
        #pragma unroll
        for (int s = 0; s < 4; s++) {
            Tn[s] = TnW[s] = TnE[s] = Y1[s] = Y1W[s] = Y1E[s] = zero;
            Y2[s] = Y2W[s] = Y2E[s] = Y3[s] = Y3W[s] = Y3E[s] = acc[s] = zero;
            #pragma unroll
            for (int a = 0; a < 11; a++) K[s][a] = zero;
        }
        // values of the previous row (j - 1) carried into the next pass:
        // 1/lambda, the evolving cell's 1/(rho c) (0 if it does not evolve),
        // -3 u, the EOS factors A, B, its east link and the links to the row
        // below, and the partial Eq. 27 divergence
        V lamI_p = L::set(1e30f), q_p = zero, uxp_p = zero, uyp_p = zero, A_p = zero, B_p = zero;
        V gE_p = zero, gS_p = zero, gSW_p = zero, gSE_p = zero, P_p = zero, dn_p = zero;

        for (int t0 = 0; t0 < nit; t0 += 4) {
            #pragma unroll
            for (int u = 0; u < 4; u++) {
                const int j = j0 + t0 + u;
                const int r1 = (u + 3) & 3, r2 = (u + 2) & 3, r3 = (u + 1) & 3;  // rows j - 1, j - 2, j - 3
                // ---- row j in (rows j + 1 .. j + RS - 2 may still be in flight), row j + RS - 1 requested ----
                asm volatile("cp.async.wait_group %0;\n" ::"n"(RS - 2) : "memory");
                const int sl = (t0 + u) & (RS - 1);
                const V cT = wb[sl][0][lane], cR = wb[sl][1][lane], cU = wb[sl][2][lane], cW = wb[sl][3][lane];
                fetch(j + RS - 1, (sl + RS - 1) & (RS - 1), itag);
                const int kd = I ? (int)HK_FLUID : kind(j);
                V T = cT, lamI, q = zero, uxp = zero, uyp = zero, A = zero, B = zero;
                if (kd == HK_FLUID) {
                    lamI = L::rcp(L::mul(L::c(wk.cvchi), cR));
                    if (!iso) {
                        q = L::rcp(L::mul(cR, L::c(wk.cv)));
                        uxp = L::mul(m3, cU);
                        uyp = L::mul(m3, cW);
                        // (dp/dT)_rho = A + B / sqrt(T) (Eq. 13), rho-only A, B
                        const V br = L::mul(L::c(wk.b), cR);
                        const V omb = L::sub(L::c(wk.one), br), den = L::fma(br, L::sub(two, br), L::c(wk.one));
                        const V iod = L::rcp(L::mul(omb, den));
                        const V pa = L::mul(L::mul(L::c(wk.akappa), L::mul(cR, cR)), L::mul(omb, iod));
                        A = L::fma(pa, L::c(wk.mkoTc), L::mul(L::mul(cR, L::c(wk.R)), L::mul(den, iod)));
                        B = L::mul(pa, L::c(wk.Bcoef));
                    }
                } else {
                    float lam = 0.0f;
                    V lamv = zero;
                    if (kd == HK_SOLID) {
                        lam = p.lambda_s;
                        if (!iso) q = L::set(irc_s);
                    } else if (kd == HK_BOTTOM) {
                        #pragma unroll
                        for (int h = 0; h < CL; h++) L::put(T, h, bottom_theta(p, xc[h], n));
                        lam = p.lambda_s;
                    }
                    if (kd == HK_GHOST || (kd == HK_BOTTOM && model_a)) lamv = L::mul(L::c(wk.cvchi), cR);
                    else lamv = L::set(lam);
                    #pragma unroll
                    for (int h = 0; h < CL; h++) {
                        const float l = L::get(lamv, h);
                        L::put(lamI, h, l > 0.0f ? fast_rcp(l) : 1e30f);
                    }
                }
                const V Tn4 = Tn[u];  // T^n of row j - 4, for its output
                Tn[u] = T;
                TnW[u] = L::west(T);
                TnE[u] = L::east(T);

                // ---- links between rows j - 1 and j; coefficients of row j - 1 ----
                const V lW = L::west(lamI), lE = L::east(lamI);
                const V gN = L::mul(g1, L::rcp(L::add(lamI_p, lamI)));
                const V gNE = L::mul(g2, L::rcp(L::add(lamI_p, lE)));
                const V gNW = L::mul(g2, L::rcp(L::add(lamI_p, lW)));
                const V gE = L::mul(g1, L::rcp(L::add(lamI, lE)));
                const V gW_p = L::west(gE_p);
                V *kc = K[r1];
                kc[0] = L::mul(q_p, gE_p);
                kc[1] = L::mul(q_p, gN);
                kc[2] = L::mul(q_p, gW_p);
                kc[3] = L::mul(q_p, gS_p);
                kc[4] = L::mul(q_p, gNE);
                kc[5] = L::mul(q_p, gNW);
                kc[6] = L::mul(q_p, gSW_p);
                kc[7] = L::mul(q_p, gSE_p);
                const V ks = L::add(L::add(L::add(kc[0], kc[1]), L::add(kc[2], kc[3])),
                                    L::add(L::add(kc[4], kc[5]), L::add(kc[6], kc[7])));
                // advection (-u . grad T = sum_a -3 w_a (e_a . u) T_a, zero off
                // the fluid) and the Eq. 27 divergence of u, whose row-j part
                // goes to row j - 1 (as its N, NE, NW neighbours) and to row
                // j + 1 (as its S, SE, SW neighbours)
                kc[0] = L::fma(w1, uxp_p, kc[0]);
                kc[1] = L::fma(w1, uyp_p, kc[1]);
                kc[2] = L::sub(kc[2], L::mul(w1, uxp_p));
                kc[3] = L::sub(kc[3], L::mul(w1, uyp_p));
                kc[4] = L::fma(w2, L::add(uxp_p, uyp_p), kc[4]);
                kc[5] = L::fma(w2, L::sub(uyp_p, uxp_p), kc[5]);
                kc[6] = L::sub(kc[6], L::mul(w2, L::add(uxp_p, uyp_p)));
                kc[7] = L::fma(w2, L::sub(uxp_p, uyp_p), kc[7]);
                const V uW = L::west(cU), uE = L::east(cU), vW = L::west(cW), vE = L::east(cW);
                const V dux = L::sub(uE, uW);
                const V ea = L::mul(w2, dux), eb = L::fma(w1, cW, L::mul(w2, L::add(vE, vW)));
                const V up = L::add(ea, eb), dn = L::sub(ea, eb), mid = L::mul(w1, dux);
                // source: -(T / rho C_V)(dp/dT)_rho div u = C1 T + C2 sqrt(T)
                // (A = B = 0 off the fluid, q = 0 when the cell does not evolve)
                const V g0 = L::mul(L::mul(m3, L::add(P_p, up)), q_p);
                const V C1 = L::mul(g0, A_p);
                kc[8] = L::sub(C1, ks);
                kc[9] = L::mul(C1, vtsat);
                kc[10] = L::mul(g0, B_p);

                // ---- stage 1 on row j - 1 (T^n of rows j - 2 .. j) ----
                {
                    const V h = stencil(kc, Tn[r1], TnE[r1], TnW[r1], Tn[u], Tn[r2], TnE[u], TnW[u], TnW[r2], TnE[r2]);
                    acc[r1] = h;
                    Y1[r1] = L::fma(half, h, Tn[r1]);
                    Y1W[r1] = L::west(Y1[r1]);
                    Y1E[r1] = L::east(Y1[r1]);
                }
                // ---- stage 2 on row j - 2 ----
                {
                    const V h = stencil(K[r2], Y1[r2], Y1E[r2], Y1W[r2], Y1[r1], Y1[r3], Y1E[r1], Y1W[r1], Y1W[r3], Y1E[r3]);
                    acc[r2] = L::fma(two, h, acc[r2]);
                    Y2[r2] = L::fma(half, h, Tn[r2]);
                    Y2W[r2] = L::west(Y2[r2]);
                    Y2E[r2] = L::east(Y2[r2]);
                }
                // ---- stage 3 on row j - 3 ----
                {
                    const V h = stencil(K[r3], Y2[r3], Y2E[r3], Y2W[r3], Y2[r2], Y2[u], Y2E[r2], Y2W[r2], Y2W[u], Y2E[u]);
                    acc[r3] = L::fma(two, h, acc[r3]);
                    Y3[r3] = L::add(Tn[r3], h);
                    Y3W[r3] = L::west(Y3[r3]);
                    Y3E[r3] = L::east(Y3[r3]);
                }
                // ---- stage 4 on row j - 4, new temperature stored ----
                {
                    const V h = stencil(K[u], Y3[u], Y3E[u], Y3W[u], Y3[r3], Y3[r1], Y3E[r3], Y3W[r3], Y3W[r1], Y3E[r1]);
                    const V out = L::fma(L::add(acc[u], h), L::c(wk.sixth), Tn4);
                    const int r4 = j - H;
                    const bool rowok = r4 >= ys && r4 < ye;
                    const int off = wrow(r4) * nx;
                    if constexpr (VEC) {
                        // a lane's two columns are both output columns or both halo
                        const bool ok = rowok && wc[0];
                        if (ok && !(fabsf(out.x) < 1e30f && fabsf(out.y) < 1e30f)) errbits |= ERRW_NONFINITE_T;
                        if (ok) *reinterpret_cast<float2 *>(Tout + off + xc[0]) = out;
                    } else {
                        #pragma unroll
                        for (int hh = 0; hh < CL; hh++) {
                            const bool ok = rowok && wc[hh];
                            if (ok && !(fabsf(L::get(out, hh)) < 1e30f)) errbits |= ERRW_NONFINITE_T;
                            if (ok) Tout[off + xc[hh]] = L::get(out, hh);
                        }
                    }
                }
                // ---- row j becomes the previous row ----
                lamI_p = lamI; q_p = q; uxp_p = uxp; uyp_p = uyp; A_p = A; B_p = B;
                gE_p = gE;
                gS_p = gN;
                gSW_p = L::west(gNE);
                gSE_p = L::east(gNW);
                P_p = L::add(mid, dn_p);
                dn_p = dn;
            }
        }
        // the last requested rows are not used, but their copies must land
        // before the block's shared memory is released
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    };
    // a segment whose rows (with the pipeline's fill and drain) are all fluid
    // rows takes the compile-time fluid path
    // (rows j0 .. j0 + nit + RS - 2 are fetched: each pass requests RS - 1 ahead)
    const bool interior = !py && j0 >= ns && j0 + nit + RS - 2 <= nt - 1;
    if (interior) march(std::true_type{});
    else march(std::false_type{});
    if (errbits) atomicOr(err, errbits);
}

template <class P, int CL, int WPB, int MINB, int RS>
struct HeatWaveShape {
    static int slots;  // warps resident on the device at once
    static cudaError_t prepare() {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_heat_wave<P, CL, WPB, MINB, RS, true, CL == 2>, 32 * WPB, 0);
        if (e != cudaSuccess) return e;
        slots = sms * (per > 0 ? per : 1) * WPB;
        return cudaSuccess;
    }
    // segment length: one wave of resident warps over the strips, at least 24
    // rows (the pipeline's fill and drain cost 8 rows per segment)
    static void geometry(const DevParams &p, int &nstrips, int &seg, int &nunits) {
        constexpr int OUTW = 32 * CL - 8;
        nstrips = (p.nx + OUTW - 1) / OUTW;
        int per = slots / nstrips;
        if (per < 1) per = 1;
        seg = (p.nt + per - 1) / per;
        if (seg < 24) seg = 24;
        const int nseg = (p.nt + seg - 1) / seg;
        nunits = nstrips * nseg;
    }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        int nstrips, seg, nunits;
        geometry(p, nstrips, seg, nunits);
        const bool wide = p.nx >= 32 * CL;
        const bool vec = CL == 2 && (p.nx % 2) == 0;
        auto k = wide ? (vec ? k_heat_wave<P, CL, WPB, MINB, RS, true, CL == 2> : k_heat_wave<P, CL, WPB, MINB, RS, true, false>)
                      : (vec ? k_heat_wave<P, CL, WPB, MINB, RS, false, CL == 2> : k_heat_wave<P, CL, WPB, MINB, RS, false, false>);
        const int grid = (nunits + WPB - 1) / WPB;
        const FParams fp = make_fparams(p);
        k<<<grid, 32 * WPB, 0, s>>>(fp, make_wave_consts(fp), nstrips, seg, nunits, (const typename P::tst *)b.T_in,
                                    (typename P::tst *)b.T_out, (const float *)b.rho, (const float *)b.ux,
                                    (const float *)b.uy, b.step, b.err);
        return cudaGetLastError();
    }
};
template <class P, int CL, int WPB, int MINB, int RS>
int HeatWaveShape<P, CL, WPB, MINB, RS>::slots = 152 * 8;

}  // namespace lbmgb
