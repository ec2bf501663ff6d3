// Flow kernel, FP32, row wavefront (Sec. 2.1: Eq. 3-15, push streaming with
// halfway bounce-back).  The same step as k_flow_pers, arranged so that no
// block barrier and no shared psi tile are needed.
//
// Each warp takes work units -- a strip of 64 columns x a segment of rows --
// from a per-run counter and sweeps the segment upward one row at a time.
// Lane l owns the two adjacent columns x0 + 2l, x0 + 2l + 1 and updates them
// as a packed FP32 pair.  For row r of the sweep:
//   - the row's nine population planes and T, with four columns on each side
//     of the strip, arrive in the warp's ring of three shared-memory rows by
//     tensor copies (TMA) that one lane issues two rows ahead, completion
//     counted in bytes on the row's mbarrier; at the periodic x edges of the
//     domain a second, 4-column box brings the wrapped halo columns;
//   - rho and psi (Eq. 10, 12-13) of row r are formed, and in every lane the
//     psi of one halo column (x0 - 1; x0 + 64 in lane 31); the west and east
//     psi of each pair come from the adjacent lanes by warp shuffles;
//   - row r - 1 is collided (Eq. 3-11, 14-15) with psi of rows r - 2, r - 1,
//     r, and its populations are pushed to their destinations (Eq. 8);
//   - row r's populations are taken from the ring into registers for the
//     next row's collision.
// A segment starts one row below its first row and ends one row above its
// last, for psi of the neighbouring rows.  Rows outside a walled domain hold
// psi = 0 (the walls act through F_ads), above an open top psi continues
// with zero normal gradient, and a domain periodic in y wraps.
//
// Requirements (checked by the launcher, which otherwise runs k_flow_pers):
// FP32 storage, nx a multiple of 64 and at least 128 (16-byte aligned box
// origins; strips cover the columns exactly; the two wrapped halos of a
// domain belong to different strips), flow not frozen.
//
// The work counter (two words per run) is zero between launches: the last
// warp to finish resets it.  Row waits are bounded (100 ms): a row that does
// not arrive sets ERRW_TIMEOUT, the warp stops, waits (bounded) for the
// copies it still has in flight, and leaves; the host reports LBM_E_TIMEOUT.
#pragma once

#include <algorithm>
#include <type_traits>

#include "lbm_fast.cuh"
#include "lbm_tma.cuh"

namespace lbmgb {

constexpr int FW_W = 64;                // strip columns
constexpr int FW_H = 4;                 // staged columns on each side of a strip (16 bytes)
constexpr int FW_SC = FW_W + 2 * FW_H;  // staged columns per array (72)
constexpr int FW_RS = 3;                // rows in a warp's ring
// one staged row (floats; every tensor-copy destination 128-byte aligned):
// populations [9][72] at 0, T [72] at FW_OT, the wrapped halo box of an edge
// strip -- populations [9][4] at FW_OSF, T [4] at FW_OST
constexpr int FW_OT = 672, FW_OSF = 768, FW_OST = 832, FW_SLOT = 864;
constexpr uint32_t FW_BYTES = 10u * FW_SC * 4u;     // main boxes of a row
constexpr uint32_t FW_SIDE_BYTES = 10u * FW_H * 4u;  // wrapped halo boxes

// The run's constants of the packed arithmetic, each in both halves of a
// pair, passed as a kernel parameter.
struct FlowWaveConsts {
    float2 mG, topc, rho_mean, g, rho0, tsat, rhoV, idtau, tauV, varpi, itauem, sgnts;
    float2 ms[7], hs[7];  // -s_k and 1 - s_k / 2 for k = 1..6 (index k)
    float2 invTc, kappa, b, R, a, two_over_G;  // psi (Eq. 12-13)
};
inline FlowWaveConsts make_flowwave_consts(const FParams &q) {
    auto d = [](float v) { return make_float2(v, v); };
    FlowWaveConsts k{};
    const float w1 = 1.0f / 3.0f, w2 = 1.0f / 12.0f;
    k.mG = d(q.mG);
    k.topc = d(-((w1 + 2.0f * w2) * q.c_w_top));  // top-wall adhesion per unit psi
    k.rho_mean = d(q.rho_mean); k.g = d(q.g); k.rho0 = d(q.rho_shift); k.tsat = d(q.T_sat);
    k.rhoV = d(q.rho_V); k.idtau = d(q.inv_drho * q.dtau); k.tauV = d(q.tau_V);
    k.varpi = d(q.varpi12G2); k.itauem = d(q.inv_tauem); k.sgnts = d(q.sgn_over_taus);
    for (int i = 1; i <= 6; i++) { k.ms[i] = d(-q.s[i]); k.hs[i] = d(q.hs[i]); }
    k.invTc = d(q.inv_Tc); k.kappa = d(q.kappa); k.b = d(q.b); k.R = d(q.R); k.a = d(q.a);
    k.two_over_G = d(q.two_over_G);
    return k;
}

// psi(rho, T) of Eq. 12-13 for a pair of sites (psi_fast's steps in packed
// FP32; reciprocals and roots per half)
__device__ __forceinline__ float2 psi_pair(const FlowWaveConsts &K, float2 rho, float2 T, unsigned &errbits) {
    const float2 tt = mul2(T, K.invTc);
    const float2 t1 = make_float2(fast_sqrt(tt.x), fast_sqrt(tt.y));
    const float2 t2 = fma2(K.kappa, sub2(f2(1.0f), t1), f2(1.0f));
    const float2 phi = mul2(t2, t2);
    const float2 br = mul2(K.b, rho);
    const float2 omb = sub2(f2(1.0f), br), den = fma2(br, sub2(f2(2.0f), br), f2(1.0f));
    const float2 num = sub2(mul2(mul2(K.R, T), den), mul2(mul2(mul2(K.a, phi), rho), omb));
    const float2 pr = mul2(mul2(rho, num), rcp2(mul2(omb, den)));
    const float2 arg = mul2(K.two_over_G, sub2(pr, mul2(rho, f2(1.0f / 3.0f))));
    // psi = 0 where the radicand is not positive; a negative (or NaN) one is a fault
    const bool bx = !(arg.x > 0.0f) && !(arg.x == 0.0f), by = !(arg.y > 0.0f) && !(arg.y == 0.0f);
    errbits |= (bx || by) ? (unsigned)ERRW_PSI : 0u;
    const float sx = fast_sqrt(fmaxf(arg.x, 0.0f)), sy = fast_sqrt(fmaxf(arg.y, 0.0f));
    return make_float2(arg.x > 0.0f ? sx : 0.0f, arg.y > 0.0f ? sy : 0.0f);
}

// Collision (Eq. 3-11, 14-15) and push (Eq. 8) of the pair of row y owned
// by this lane: populations gp, their sum d (rho - rho0), psi of the pair
// (psi), of its west / east neighbours (W0, E0) and of the rows below (Pm,
// Wm, Em) and above (P1, W1, E1).
__device__ __forceinline__ void wave_collide(const FParams &p, const FlowWaveConsts &K, const float2 (&gp)[9], float2 d,
                                             float2 psi, float2 W0, float2 E0, float2 Pm, float2 Wm, float2 Em,
                                             float2 P1, float2 W1, float2 E1, int y, bool py, bool outflow, int c0,
                                             int c1, int xw, int xe, const double *__restrict__ cw,
                                             float *const (&op)[9], float *__restrict__ rho_o, float *__restrict__ ux_o,
                                             float *__restrict__ uy_o, float &mass, float &nvap, unsigned &errbits) {
    const int nx = p.nx, nf = p.nf;
    const bool bot = !py && y == 0, top = !py && y == nf - 1;
    const float2 a = sub2(E1, Wm);  // pNE - pSW
    const float2 b = sub2(Em, W1);  // pSE - pNW
    const float2 pre = mul2(K.mG, psi);
    const float2 sx = fma2(f2(1.0f / 3.0f), sub2(E0, W0), mul2(f2(1.0f / 12.0f), add2(a, b)));
    const float2 sy = fma2(f2(1.0f / 3.0f), sub2(P1, Pm), mul2(f2(1.0f / 12.0f), sub2(a, b)));
    const float2 rho = add2(d, K.rho0);
    float2 Fx = mul2(pre, sx);
    float2 Fy = mul2(pre, sy);
    if (bot) {  // Eq. 14 with the heater sites below (i = 4, 7, 8)
        const float cW = float(cw[xw]), cA = float(cw[c0]), cB = float(cw[c1]), cE = float(cw[xe]);
        const float2 cm = make_float2(cW, cA), cc = make_float2(cA, cB), cp = make_float2(cB, cE);
        Fx = sub2(Fx, mul2(psi, mul2(f2(1.0f / 12.0f), sub2(cp, cm))));
        float2 Fay = mul2(psi, fma2(f2(1.0f / 3.0f), cc, mul2(f2(1.0f / 12.0f), add2(cm, cp))));
        if (top && !outflow) Fay = add2(Fay, mul2(psi, K.topc));
        Fy = add2(Fy, Fay);
    } else if (top && !outflow) {
        Fy = add2(Fy, mul2(psi, K.topc));
    }
    Fy = sub2(Fy, mul2(sub2(rho, K.rho_mean), K.g));
    // moments of g (Eq. 6 with the rho0 shift folded into q0..q2)
    const float2 s14 = add2(add2(gp[1], gp[2]), add2(gp[3], gp[4]));
    const float2 s58 = add2(add2(gp[5], gp[6]), add2(gp[7], gp[8]));
    const float2 m1 = fma2(f2(2.0f), s58, sub2(mul2(f2(-4.0f), gp[0]), s14));
    const float2 m2 = add2(fma2(f2(-2.0f), s14, mul2(f2(4.0f), gp[0])), s58);
    const float2 f13 = sub2(gp[1], gp[3]), f24 = sub2(gp[2], gp[4]);
    const float2 f57 = sub2(gp[5], gp[7]), f86 = sub2(gp[8], gp[6]);
    const float2 sp = add2(f57, f86), sm = sub2(f57, f86);
    const float2 m3 = add2(f13, sp), m4 = fma2(f2(-2.0f), f13, sp);
    const float2 m5 = add2(f24, sm), m6 = fma2(f2(-2.0f), f24, sm);
    const float2 m7 = sub2(add2(gp[1], gp[3]), add2(gp[2], gp[4]));
    const float2 m8 = sub2(add2(gp[5], gp[7]), add2(gp[6], gp[8]));
    const float2 irho = rcp2(rho);
    const float2 ux = mul2(fma2(f2(0.5f), Fx, m3), irho), uy = mul2(fma2(f2(0.5f), Fy, m5), irho);
    const float2 tau = fma2(sub2(rho, K.rhoV), K.idtau, K.tauV);
    const float2 s78 = rcp2(tau);
    const float2 uxx = mul2(ux, ux), uyy = mul2(uy, uy);
    const float2 ru2 = mul2(rho, add2(uxx, uyy));
    const float2 q1 = fma2(f2(3.0f), ru2, mul2(f2(-2.0f), d)), q2 = fma2(f2(-3.0f), ru2, d);
    const float2 q3 = mul2(rho, ux), q5 = mul2(rho, uy);
    const float2 q7 = mul2(rho, sub2(uxx, uyy)), q8 = mul2(rho, mul2(ux, uy));
    const float2 uF = fma2(ux, Fx, mul2(uy, Fy));
    const float2 e2v = mul2(K.varpi, fma2(sx, sx, mul2(sy, sy)));
    const float2 eps = make_float2(psi.x > 0.0f ? e2v.x : 0.0f, psi.y > 0.0f ? e2v.y : 0.0f);
    const float2 S1 = fma2(f2(6.0f), uF, mul2(eps, K.itauem));
    const float2 S2 = fma2(f2(-6.0f), uF, mul2(eps, K.sgnts));
    // Eq. 7 (m0 unchanged; q4 = -q3, q6 = -q5)
    const float2 z1 = fma2(K.hs[1], S1, fma2(K.ms[1], sub2(m1, q1), m1));
    const float2 z2 = fma2(K.hs[2], S2, fma2(K.ms[2], sub2(m2, q2), m2));
    const float2 z3 = fma2(K.hs[3], Fx, fma2(K.ms[3], sub2(m3, q3), m3));
    const float2 z4 = sub2(fma2(K.ms[4], add2(m4, q3), m4), mul2(K.hs[4], Fx));
    const float2 z5 = fma2(K.hs[5], Fy, fma2(K.ms[5], sub2(m5, q5), m5));
    const float2 z6 = sub2(fma2(K.ms[6], add2(m6, q5), m6), mul2(K.hs[6], Fy));
    const float2 h78 = fma2(f2(-0.5f), s78, f2(1.0f));
    const float2 z7 = fma2(h78, mul2(f2(2.0f), sub2(mul2(ux, Fx), mul2(uy, Fy))),
                           sub2(m7, mul2(s78, sub2(m7, q7))));
    const float2 z8 = fma2(h78, fma2(ux, Fy, mul2(uy, Fx)), sub2(m8, mul2(s78, sub2(m8, q8))));
    const float2 e0 = mul2(d, f2(1.0f / 9.0f)), e1 = mul2(z1, f2(1.0f / 36.0f)), e2 = mul2(z2, f2(1.0f / 36.0f));
    const float2 e3 = mul2(z3, f2(1.0f / 6.0f)), e4 = mul2(z4, f2(1.0f / 12.0f)), e5 = mul2(z5, f2(1.0f / 6.0f));
    const float2 e6 = mul2(z6, f2(1.0f / 12.0f)), e7 = mul2(z7, f2(0.25f)), e8 = mul2(z8, f2(0.25f));
    const float2 A0 = fma2(f2(-2.0f), e2, sub2(e0, e1));  // axis-direction common part
    const float2 B0 = add2(fma2(f2(2.0f), e1, e0), e2); // diagonal common part
    const float2 fo0 = fma2(f2(4.0f), e2, fma2(f2(-4.0f), e1, e0));
    const float2 t34 = fma2(f2(-2.0f), e4, e3), t56 = fma2(f2(-2.0f), e6, e5);
    const float2 fo1 = add2(add2(A0, t34), e7), fo3 = add2(sub2(A0, t34), e7);
    const float2 fo2 = sub2(add2(A0, t56), e7), fo4 = sub2(sub2(A0, t56), e7);
    const float2 cxx = add2(e3, e4), cyy = add2(e5, e6);
    const float2 fo5 = add2(add2(add2(B0, cxx), cyy), e8), fo6 = sub2(add2(sub2(B0, cxx), cyy), e8);
    const float2 fo7 = add2(sub2(sub2(B0, cxx), cyy), e8), fo8 = sub2(sub2(add2(B0, cxx), cyy), e8);
    if (!(fabsf(rho.x) < 1e30f) || !(fabsf(rho.y) < 1e30f)) errbits |= ERRW_NONFINITE_RHO;
    mass += rho.x + rho.y;
    nvap += (rho.x < p.vap_threshold ? 1.0f : 0.0f) + (rho.y < p.vap_threshold ? 1.0f : 0.0f);
    const int ko = y * nx;
    *reinterpret_cast<float2 *>(rho_o + ko + c0) = rho;
    *reinterpret_cast<float2 *>(ux_o + ko + c0) = ux;
    *reinterpret_cast<float2 *>(uy_o + ko + c0) = uy;
    // Eq. 8, push; halfway bounce-back at the heater and the top wall
    auto st2 = [](float *q, float2 v) { *reinterpret_cast<float2 *>(q) = v; };
    st2(op[0] + ko + c0, fo0);
    op[1][ko + c1] = fo1.x; op[1][ko + xe] = fo1.y;   // east
    op[3][ko + xw] = fo3.x; op[3][ko + c0] = fo3.y;   // west
    const int kn = (py && y == nf - 1) ? 0 : ko + nx;             // row above
    const int ks = (py && y == 0) ? (nf - 1) * nx : ko - nx;      // row below
    if (!top) {
        st2(op[2] + kn + c0, fo2);
        op[5][kn + c1] = fo5.x; op[5][kn + xe] = fo5.y;
        op[6][kn + xw] = fo6.x; op[6][kn + c0] = fo6.y;
    } else if (!outflow) {
        st2(op[4] + ko + c0, fo2);
        st2(op[7] + ko + c0, fo5);
        st2(op[8] + ko + c0, fo6);
    }
    if (!bot) {
        st2(op[4] + ks + c0, fo4);
        op[7][ks + xw] = fo7.x; op[7][ks + c0] = fo7.y;
        op[8][ks + c1] = fo8.x; op[8][ks + xe] = fo8.y;
    } else {
        st2(op[2] + ko + c0, fo4);
        st2(op[5] + ko + c0, fo7);
        st2(op[6] + ko + c0, fo8);
    }
    if (top && outflow) {
        st2(op[4] + ko + c0, fo4);
        op[7][ko + xw] = fo7.x; op[7][ko + c0] = fo7.y;
        op[8][ko + c1] = fo8.x; op[8][ko + xe] = fo8.y;
    }
}

// A warp's ring of staged rows and the state of its copies.
struct WaveRing {
    float *ring;    // FW_RS rows of FW_SLOT floats, 128-byte aligned
    uint64_t *bar;  // their mbarriers (one arrival: lane 0's, plus the bytes)
    uint32_t ph;    // bit s: parity of ring row s's next completion
    int busy;       // bit s: ring row s has copies nobody waited for
    bool failed;    // a row wait ran out
};

// lane 0 initialises the warp's barriers
__device__ __forceinline__ void wave_ring_init(WaveRing &w, float *ring, uint64_t *bar, int lane) {
    w.ring = ring;
    w.bar = bar;
    w.ph = 0;
    w.busy = 0;
    w.failed = false;
    if (lane == 0) {
        #pragma unroll
        for (int s = 0; s < FW_RS; s++) mbar_init(&bar[s], 1);
        fence_proxy_async();  // the initialised barriers are visible to the copy engine
    }
    __syncwarp();
}

// after a wait ran out: let the copies still owed to the ring land before
// its shared memory is released (each wait bounded)
__device__ __forceinline__ void wave_ring_drain(WaveRing &w) {
    #pragma unroll
    for (int s = 0; s < FW_RS; s++)
        if (w.busy & (1 << s)) mbar_wait(&w.bar[s], (w.ph >> s) & 1u);
}

// One work unit of one run: the 64-column strip at x0, rows ys .. ye - 1,
// swept upward through the warp's ring; the mass and vapour count of the
// collided sites are added to mass and nvap (FP32, per lane).
__device__ __forceinline__ void wave_unit(const FParams &p, const FlowWaveConsts &K, const CUtensorMap *map_f,
                                          const CUtensorMap *map_t, const CUtensorMap *map_fs,
                                          const CUtensorMap *map_ts, int x0, int ys, int ye, float *const (&op)[9],
                                          float *__restrict__ rho_o, float *__restrict__ ux_o,
                                          float *__restrict__ uy_o, const double *__restrict__ cw, WaveRing &w,
                                          int lane, float &mass, float &nvap, unsigned &errbits) {
    const unsigned FULL = 0xffffffffu;
    const int nx = p.nx, nf = p.nf, ns = p.ns;
    const bool py = (p.flags & FLAG_PERIODIC_Y) != 0;
    const bool outflow = p.top_mode == TOP_OUTFLOW;
    const int po = FW_H + 2 * lane;  // this lane's pair in a staged array
    const bool wedge = x0 == 0, eedge = x0 + FW_W == nx;
    const int nit = ye - ys + 2;  // rows ys - 1 .. ye
    const int c0 = x0 + 2 * lane, c1 = c0 + 1;
    const int xw = c0 == 0 ? nx - 1 : c0 - 1, xe = c0 + 2 == nx ? 0 : c0 + 2;
    // this lane's halo column in a staged row: the west one (x0 - 1), in
    // lane 31 the east one (x0 + 64); at the periodic edges of the domain
    // the wrapped box's column is moved into that place first
    const int hb = lane == 31 ? FW_H + FW_W : FW_H - 1;
    const uint32_t bytes = FW_BYTES + ((wedge || eedge) ? FW_SIDE_BYTES : 0u) + p.tx_pad;
    // row r = ys - 1 + o is staged if the sweep reads it: every o < nit
    // if periodic in y (r wrapped), else those of rows 0 .. nf - 1
    const int kfirst = (!py && ys == 0) ? 1 : 0, klast = (!py && ye == nf) ? nit - 2 : nit - 1;
    auto staged = [&](int o, int &rr) {
        const int r = ys - 1 + o;
        rr = r < 0 ? r + nf : (r >= nf ? r - nf : r);
        return o >= kfirst && o <= klast;
    };
    // lane 0: stage row o into ring row s (its previous contents read)
    auto issue = [&](int o, int s) {
        int rr;
        if (!staged(o, rr)) return;
        w.busy |= 1 << s;
        if (lane != 0) return;
        float *dst = w.ring + s * FW_SLOT;
        fence_proxy_async();  // the warp's earlier reads of this row come first
        mbar_arrive_expect_tx(&w.bar[s], bytes);
        tma_load_3d(dst, map_f, x0 - FW_H, rr, 0, &w.bar[s]);
        tma_load_2d(dst + FW_OT, map_t, x0 - FW_H, ns + rr, &w.bar[s]);
        if (wedge) {
            tma_load_3d(dst + FW_OSF, map_fs, nx - FW_H, rr, 0, &w.bar[s]);
            tma_load_2d(dst + FW_OST, map_ts, nx - FW_H, ns + rr, &w.bar[s]);
        } else if (eedge) {
            tma_load_3d(dst + FW_OSF, map_fs, 0, rr, 0, &w.bar[s]);
            tma_load_2d(dst + FW_OST, map_ts, 0, ns + rr, &w.bar[s]);
        }
    };
    __syncwarp();  // the previous unit's reads of the ring are done
    issue(0, 0);
    issue(1, 1);

    float2 gp[9];  // populations of the row to collide next
    // psi, west / east psi of the rows below it (m), of it (c), above it
    // (n); the sum g (rho - rho0) of it and of the row just read
    float2 Pm = f2(0.0f), Wm = f2(0.0f), Em = f2(0.0f), Pc = f2(0.0f), Wc = f2(0.0f), Ec = f2(0.0f);
    float2 Dc = f2(0.0f);
    int s = 0;  // ring row of ordinal k (k % 3)
    for (int k = 0; k < nit; k++) {
        const int r = ys - 1 + k;
        const int sn = s == 0 ? FW_RS - 1 : s - 1;  // ring row of ordinals k - 1 and k + 2
        int rr;
        const bool ld = staged(k, rr);
        if (ld) {
            const bool ok = mbar_wait(&w.bar[s], (w.ph >> s) & 1u);
            if (!__all_sync(FULL, ok)) {  // the row stays owed: drained below
                w.failed = true;
                break;
            }
            w.ph ^= 1u << s;
            w.busy &= ~(1 << s);
        }
        __syncwarp();  // ring row sn (ordinal k - 1) is read
        issue(k + 2, sn);
        float *const sr = w.ring + s * FW_SLOT;
        if (ld && (wedge || eedge)) {
            // the wrapped halo column into its place in the main box (whose
            // copy read zeros there): lane 0 west, lane 31 east
            if (lane == (wedge ? 0 : 31)) {
                const int to = wedge ? FW_H - 1 : FW_H + FW_W, from = wedge ? FW_H - 1 : 0;
                #pragma unroll
                for (int i = 0; i < 9; i++) sr[i * FW_SC + to] = sr[FW_OSF + i * FW_H + from];
                sr[FW_OT + to] = sr[FW_OST + from];
            }
            __syncwarp();
        }
        float2 Pn, Wn, En, Dn = f2(0.0f);
        if (ld) {
            float2 gr[9];
            #pragma unroll
            for (int i = 0; i < 9; i++) gr[i] = *reinterpret_cast<const float2 *>(sr + i * FW_SC + po);
            const float2 Tr = *reinterpret_cast<const float2 *>(sr + FW_OT + po);
            Dn = add2(add2(add2(add2(gr[0], gr[1]), add2(gr[2], gr[3])), add2(add2(gr[4], gr[5]), add2(gr[6], gr[7]))),
                      gr[8]);
            float hg[9];
            #pragma unroll
            for (int i = 0; i < 9; i++) hg[i] = sr[hb + i * FW_SC];
            const float hd = ((hg[0] + hg[1]) + (hg[2] + hg[3])) + ((hg[4] + hg[5]) + (hg[6] + hg[7])) + hg[8];
            Pn = psi_pair(K, add2(Dn, K.rho0), add2(Tr, K.tsat), errbits);
            const float hp = psi_fast(p, hd + p.rho_shift, sr[FW_OT + hb] + p.T_sat, errbits);
            const float wn = __shfl_up_sync(FULL, Pn.y, 1), en = __shfl_down_sync(FULL, Pn.x, 1);
            Wn = make_float2(lane == 0 ? hp : wn, Pn.x);
            En = make_float2(Pn.y, lane == 31 ? hp : en);
        } else if (r >= nf && outflow) {
            Pn = Pc; Wn = Wc; En = Ec;  // open top: zero normal gradient
        } else {
            Pn = f2(0.0f); Wn = f2(0.0f); En = f2(0.0f);  // wall rows
        }
        if (k >= 2)
            wave_collide(p, K, gp, Dc, Pc, Wc, Ec, Pm, Wm, Em, Pn, Wn, En, r - 1, py, outflow, c0, c1, xw, xe, cw,
                         op, rho_o, ux_o, uy_o, mass, nvap, errbits);
        if (ld && k >= 1 && k <= nit - 2) {
            #pragma unroll
            for (int i = 0; i < 9; i++) gp[i] = *reinterpret_cast<const float2 *>(sr + i * FW_SC + po);
        }
        Pm = Pc; Wm = Wc; Em = Ec;
        Pc = Pn; Wc = Wn; Ec = En;
        Dc = Dn;
        s = s == FW_RS - 1 ? 0 : s + 1;
    }
}

// Work units of the wavefront flow kernel: strips of 64 columns times row
// segments, taken in counter order one band of rows (all strips) at a time.
// Rows [0, y2) come in segments of seg rows, rows [y2, nf) in shorter
// segments of seg2 rows, so that the units taken last, while the other
// warps run out of work, are short.
struct WaveUnits {
    int nstrips, seg, nmain, y2, seg2, nunits;
    __device__ __forceinline__ void unit(int u, int nf, int &strip, int &ys, int &ye) const {
        if (u < nmain) {
            strip = u % nstrips;
            ys = (u / nstrips) * seg;
            ye = min(ys + seg, y2);
        } else {
            const int v = u - nmain;
            strip = v % nstrips;
            ys = y2 + (v / nstrips) * seg2;
            ye = min(ys + seg2, nf);
        }
    }
};

template <int WPB, int MINB>
__global__ void __launch_bounds__(32 * WPB, MINB)
k_flow_wave(const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_t,
            const __grid_constant__ CUtensorMap map_fs, const __grid_constant__ CUtensorMap map_ts,
            const __grid_constant__ FParams p, const __grid_constant__ FlowWaveConsts K, WaveUnits wu,
            float *__restrict__ fout, float *__restrict__ rho_o, float *__restrict__ ux_o,
            float *__restrict__ uy_o, const double *__restrict__ cw, double *__restrict__ part,
            unsigned *__restrict__ err, unsigned *__restrict__ wq) {
    extern __shared__ float4 fw_raw[];  // the warps' rings (+128 bytes of slack)
    __shared__ __align__(8) uint64_t fw_bar[WPB][FW_RS];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // 128-byte aligned, by an offset from the array (so that accesses stay
    // shared-memory loads)
    float *const ring = reinterpret_cast<float *>(fw_raw) + ((128u - (smem_u32(fw_raw) & 127u)) & 127u) / 4u +
                        warp * (FW_RS * FW_SLOT);
    const size_t plane = (size_t)p.nf * p.nx;
    float *op[9];
    #pragma unroll
    for (int i = 0; i < 9; i++) op[i] = fout + i * plane;
    unsigned errbits = 0;
    float mass = 0.0f, nvap = 0.0f;
    WaveRing w;
    wave_ring_init(w, ring, fw_bar[warp], lane);
    for (;;) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(wq, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= wu.nunits) break;
        int ys, ye, strip;
        wu.unit(u, p.nf, strip, ys, ye);
        wave_unit(p, K, &map_f, &map_t, &map_fs, &map_ts, strip * FW_W, ys, ye, op, rho_o, ux_o, uy_o, cw, w, lane,
                  mass, nvap, errbits);
        if (w.failed) break;
    }
    if (w.failed) {
        errbits |= ERRW_TIMEOUT;
        wave_ring_drain(w);
    }
    // per-warp mass and vapour count: FP32 inside the warp, FP64 across warps
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mass += __shfl_down_sync(FULL, mass, o);
        nvap += __shfl_down_sync(FULL, nvap, o);
    }
    const int gw = blockIdx.x * WPB + warp;
    if (lane == 0) {
        part[2 * gw] = (double)mass;
        part[2 * gw + 1] = (double)nvap;
        // the last warp of the launch to finish leaves the counter at zero
        __threadfence();
        const unsigned done = atomicAdd(wq + 1, 1u);
        if (done == gridDim.x * WPB - 1) {
            wq[0] = 0u;
            wq[1] = 0u;
        }
    }
    if (errbits) atomicOr(err, errbits);
}

// Launch shape of k_flow_wave (U2: work units per resident warp, times
// two; SEGM > 0: segments of SEGM rows, and a last band of SEGT-row segments
// with about TU2 / 2 units per resident warp); domains it cannot take run
// k_flow_pers (32 x 16-site tiles) instead.
template <int WPB, int MINB, int U2, int SEGM = 0, int SEGT = 0, int TU2 = 2>
struct FlowWaveShape {
    using Fallback = FlowPersShape<PolicyF32, 32, 8, 2, 2>;
    static constexpr size_t smem_bytes = (size_t)WPB * FW_RS * FW_SLOT * sizeof(float) + 128;
    static int grid_blocks;  // resident blocks on the device
    static bool eligible(const DevParams &p) {
        return p.nx % FW_W == 0 && p.nx >= 2 * FW_W && !(p.flags & FLAG_FROZEN_FLOW) && tensor_map_encoder() != nullptr;
    }
    static cudaError_t prepare() {
        cudaError_t e = Fallback::prepare();
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_flow_wave<WPB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_flow_wave<WPB, MINB>, 32 * WPB, smem_bytes);
        if (e != cudaSuccess) return e;
        grid_blocks = sms * (per > 0 ? per : 1);
        return cudaSuccess;
    }
    // without SEGM: segments of at least 8 rows, about U2 / 2 units per
    // resident warp (taken from the counter, so a warp that starts late takes
    // fewer; longer segments re-read fewer rows at their ends)
    static WaveUnits shape(const DevParams &p) {
        WaveUnits wu;
        wu.nstrips = p.nx / FW_W;
        if (SEGM > 0) {
            const long long warps = (long long)grid_blocks * WPB * TU2 / 2;
            const int tail_bands = (int)((warps + wu.nstrips - 1) / wu.nstrips);
            int tail_rows = std::min(p.nf, SEGT * tail_bands);
            if (p.nf - tail_rows < SEGM) tail_rows = p.nf;  // too small for a main band
            wu.seg = SEGM;
            wu.y2 = p.nf - tail_rows;
            wu.seg2 = SEGT;
        } else {
            const long long want = (long long)U2 * grid_blocks * WPB / 2;
            const int nseg = (int)std::max<long long>(1, want / wu.nstrips);
            wu.seg = std::max(8, (p.nf + nseg - 1) / nseg);
            wu.y2 = p.nf;
            wu.seg2 = wu.seg;
        }
        wu.nmain = wu.nstrips * ((wu.y2 + wu.seg - 1) / wu.seg);
        wu.nunits = wu.nmain + wu.nstrips * ((p.nf - wu.y2 + wu.seg2 - 1) / wu.seg2);
        return wu;
    }
    static int grid(const DevParams &p) { return std::min(grid_blocks, (shape(p).nunits + WPB - 1) / WPB); }
    // one pair of partial sums per warp
    static int blocks(const DevParams &p) { return eligible(p) ? grid(p) * WPB : Fallback::blocks(p); }
    static cudaError_t launch(const DevParams &p, const StepBuffers &b, cudaStream_t s) {
        if (!eligible(p)) return Fallback::launch(p, b, s);
        const WaveUnits wu = shape(p);
        // boxes: 72 columns x 1 row x 9 planes of the populations and 72 x 1
        // of T (all T rows, heater included: fluid row y sits at ns + y);
        // the wrapped halo boxes 4 columns wide
        CUtensorMap mf, mt, mfs, mts;
        const cuuint64_t nxu = (cuuint64_t)p.nx, nfu = (cuuint64_t)p.nf, ntu = (cuuint64_t)p.nt;
        const cuuint64_t gd_f[3] = {nxu, nfu, 9}, gs_f[2] = {nxu * 4, nxu * nfu * 4};
        const cuuint64_t gd_t[2] = {nxu, ntu}, gs_t[1] = {nxu * 4};
        const cuuint32_t bx_f[3] = {(cuuint32_t)FW_SC, 1, 9}, bx_t[2] = {(cuuint32_t)FW_SC, 1};
        const cuuint32_t bs_f[3] = {(cuuint32_t)FW_H, 1, 9}, bs_t[2] = {(cuuint32_t)FW_H, 1}, one[3] = {1, 1, 1};
        auto enc = tensor_map_encoder();
        auto make = [&](CUtensorMap *m, int rank, const void *base, const cuuint64_t *gd, const cuuint64_t *gs,
                        const cuuint32_t *bx) {
            return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void *>(base), gd, gs, bx, one,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        };
        CUresult r = make(&mf, 3, b.f_in, gd_f, gs_f, bx_f);
        if (r == CUDA_SUCCESS) r = make(&mt, 2, b.T_in, gd_t, gs_t, bx_t);
        if (r == CUDA_SUCCESS) r = make(&mfs, 3, b.f_in, gd_f, gs_f, bs_f);
        if (r == CUDA_SUCCESS) r = make(&mts, 2, b.T_in, gd_t, gs_t, bs_t);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        const FParams q = make_fparams(p);
        k_flow_wave<WPB, MINB><<<grid(p), 32 * WPB, smem_bytes, s>>>(
            mf, mt, mfs, mts, q, make_flowwave_consts(q), wu, (float *)b.f_out, (float *)b.rho,
            (float *)b.ux, (float *)b.uy, b.cw, b.part, b.err, b.wq);
        return cudaGetLastError();
    }
};
template <int WPB, int MINB, int U2, int SEGM, int SEGT, int TU2>
int FlowWaveShape<WPB, MINB, U2, SEGM, SEGT, TU2>::grid_blocks = 152;

}  // namespace lbmgb
