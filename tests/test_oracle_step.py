"""Whole-step pins of the FP64 oracle: invariants, closed-form limits of the
heat half, symmetries and the two physics checks the method fixes (flat
interface coexistence densities and the Laplace law).  No GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1911_10747_gb300 import workloads as W

WL = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def uniform_f(rho, nf, nx):
    return np.broadcast_to(WL[:, None, None] * rho, (9, nf, nx)).copy()


def test_uniform_box_stays_at_rest():
    """Uniform density in a periodic box: the pseudopotential force cancels
    pairwise (Eq. 11), u = 0 and the populations stay at equilibrium."""
    cfg = W.periodic_box(8, 8, liquid_rows=8)
    r = O.OracleRun(cfg)
    f0 = r.f
    r.step(50)
    assert r.err == 0
    np.testing.assert_array_equal(r.ux, 0.0)
    np.testing.assert_array_equal(r.uy, 0.0)
    np.testing.assert_allclose(r.f, f0, rtol=2e-15, atol=0)


def test_rk4_amplification_of_a_conduction_mode():
    """Frozen uniform fluid, T = T_sat + eps cos(k x): Eq. 24 reduces to
    dT/dt = alpha Lap T with alpha = C_V chi / C_V, the Laplacian (Eq. 28)
    has eigenvalue 2 (cos k - 1), so each RK4 step (Eq. 25-26) multiplies the
    amplitude by 1 + z + z^2/2 + z^3/6 + z^4/24, z = 2 alpha (cos k - 1)."""
    nx, ny = 16, 4
    cfg = W.periodic_box(nx, ny, liquid_rows=ny, isothermal=False, frozen_flow=True,
                         cv_chi=0.9, c_v=1.0)
    r = O.OracleRun(cfg)
    tsat = 0.86 * r.Tc
    k = 2 * math.pi * 2 / nx
    x = np.arange(nx)
    eps = 1e-3 * tsat
    r.set_T(np.broadcast_to(tsat + eps * np.cos(k * x), (ny, nx)))
    z = 2 * (cfg.cv_chi / cfg.c_v) * (math.cos(k) - 1)
    amp = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    r.step(10)
    expect = tsat + eps * amp ** 10 * np.cos(k * x)
    np.testing.assert_allclose(r.T, np.broadcast_to(expect, (ny, nx)), rtol=0, atol=1e-15)
    assert abs(amp) < 1 and amp ** 10 < 0.5  # the mode really decays


def test_steady_conduction_through_heater_and_fluid_slab():
    """Frozen liquid over the heater, bottom T_b, top T_sat: the steady
    discrete solution is piecewise linear with the flux set by the series sum
    of the link resistances 1/lambda_face (harmonic means at the jump)."""
    nx, ns, nf = 4, 6, 6
    cfg = W.RunConfig(nx=nx, nf=nf, ns=ns, liquid_rows=nf, frozen_flow=True, bc_mode="spots",
                      init_noise=0.0, lambda_s=3.25, rho_c_s=39.0, T_b_over_Tc=0.96, g=0.0)
    r = O.OracleRun(cfg)
    r.step(40000)
    tc = r.Tc
    tb, tsat = 0.96 * tc, 0.86 * tc
    lam = np.array([3.25] * ns + [0.05 * 6.5] * nf + [0.05 * 6.5])  # rows 0..nt, ghost last
    faces = 2 * lam[:-1] * lam[1:] / (lam[:-1] + lam[1:])
    q = (tsat - tb) / np.sum(1 / faces)
    prof = tb + q * np.concatenate([[0.0], np.cumsum(1 / faces)[:-1]])
    np.testing.assert_allclose(r.T, np.broadcast_to(prof[:, None], (ns + nf, nx)), rtol=0, atol=1e-13)
    d = r.diagnostics()
    # Eq. 36 on a linear profile inside the heater is exact: Q = -lambda_s dT/dy = -q
    assert d["q_bottom"] == pytest.approx(-q, rel=1e-9)
    assert d["q_top"] == pytest.approx(-q, rel=1e-9)


def test_model_a_steady_conduction_is_linear_between_the_two_dirichlet_rows():
    """Model A (no heater): frozen uniform liquid between the wall row (row
    0, T_b) and the top ghost (row nt, T_sat).  Every link conducts with the
    same lambda_f, so the steady discrete solution is linear in the row
    index with slope (T_sat - T_b) / nt, and the wall flux the diagnostics
    report is -lambda_f times that slope.  A heater conductivity on the
    wall link would put a kink at row 0."""
    nx, nf = 4, 6
    cfg = W.RunConfig(nx=nx, nf=nf, ns=0, liquid_rows=nf, frozen_flow=True, bc_mode="spots",
                      init_noise=0.0, lambda_s=3.25, rho_c_s=39.0, T_b_over_Tc=0.96, g=0.0)
    assert cfg.model_a and cfg.t_rows == nf + 1
    r = O.OracleRun(cfg)
    r.step(20000)
    tc = r.Tc
    tb, tsat = 0.96 * tc, 0.86 * tc
    nt = nf + 1
    prof = tb + (tsat - tb) * np.arange(nt) / nt
    np.testing.assert_allclose(r.T, np.broadcast_to(prof[:, None], (nt, nx)), rtol=0, atol=1e-13)
    d = r.diagnostics()
    lam_f = 0.05 * 6.5
    q = -lam_f * (tsat - tb) / nt
    assert d["q_bottom"] == pytest.approx(q, rel=1e-9)
    assert d["q_top"] == pytest.approx(q, rel=1e-9)
    np.testing.assert_allclose(r.q_top, q, rtol=1e-9)


def test_model_a_wall_row_follows_the_bottom_condition_and_sets_the_flux():
    """Model A with the noisy bottom: after a step row 0 holds
    T_b (1 + A (2U - 1)) with U the counter-based draw of that column and
    step, and the wall flux is -lambda_f (T(row 1) - T(row 0)) with
    lambda_f = cv_chi rho of the first fluid row."""
    nx, nf = 16, 8
    cfg = W.RunConfig(nx=nx, nf=nf, ns=0, liquid_rows=nf, frozen_flow=True, isothermal=True,
                      bc_mode="noise", init_noise=0.0, T_b_over_Tc=0.96, g=0.0, seed=11)
    r = O.OracleRun(cfg)
    r.step(3)
    tb = 0.96 * r.Tc
    U = np.array([O.uniform(11, 2, 2, x) for x in range(nx)])
    np.testing.assert_allclose(r.T[0], tb * (1 + cfg.bc_noise * (2 * U - 1)), rtol=1e-15, atol=0)
    q = -(cfg.cv_chi * r.rho[0]) * (r.T[1] - r.T[0])
    np.testing.assert_allclose(r.q_top, q, rtol=1e-13)
    assert r.diagnostics()["q_bottom"] == pytest.approx(q.mean(), rel=1e-13)


def test_wall_flux_formula_exact_on_quadratic_profile():
    """Eq. 36 is second-order one-sided: exact for T = T_b + alpha y + beta y^2."""
    nx, ns, nf = 6, 4, 4
    cfg = W.RunConfig(nx=nx, nf=nf, ns=ns, liquid_rows=nf, frozen_flow=True, isothermal=True,
                      init_noise=0.0, lambda_s=3.25, g=0.0)
    r = O.OracleRun(cfg)
    tb = 0.96 * r.Tc
    y = np.arange(ns + nf, dtype=float)[:, None]
    alpha, beta = -2e-4, 3e-5
    r.set_T(np.broadcast_to(tb + alpha * y + beta * y ** 2, (ns + nf, nx)))
    r.step(1)
    assert r.diagnostics()["q_bottom"] == pytest.approx(-3.25 * alpha, rel=1e-11)


def test_mass_is_conserved_with_bounce_back_walls():
    cfg = W.small_parity()
    r = O.OracleRun(cfg)
    r.step(1)
    m0 = r.diagnostics()["mass"]
    r.step(300)
    assert r.err == 0
    assert r.diagnostics()["mass"] == pytest.approx(m0, rel=1e-12)
    # and the post-stream populations carry the same mass
    assert r.f.sum() == pytest.approx(m0, rel=1e-12)


def test_column_invariance_without_spots_or_noise():
    """With every column identical (no spots, no noise, constant bottom) the
    periodic step keeps the columns bit-identical: each column does the same
    arithmetic in the same order."""
    cfg = W.RunConfig(nx=8, nf=24, ns=4, liquid_rows=8, init_noise=0.0, bc_mode="spots",
                      lambda_s=3.25, rho_c_s=39.0)
    r = O.OracleRun(cfg)
    r.step(100)
    for a in (r.rho, r.ux, r.uy, r.T):
        assert np.array_equal(a, np.broadcast_to(a[:, :1], a.shape))
    np.testing.assert_array_equal(r.ux, 0.0)


def test_mirror_symmetry():
    """A mirror-symmetric start (one spot centred on column 0, no noise) stays
    mirror-symmetric: rho(x) = rho(-x), u_x(x) = -u_x(-x).  A wrong velocity
    sign, opposite index or neighbour offset breaks it."""
    nx = 32
    cfg = W.RunConfig(nx=nx, nf=24, ns=4, liquid_rows=8, init_noise=0.0, bc_mode="spots",
                      spot_x=(0,), spot_half_width=2, c_w_spot=(-0.5,), lambda_s=3.25,
                      rho_c_s=39.0, T_b_over_Tc=1.0)
    r = O.OracleRun(cfg)
    r.step(200)
    mir = (-np.arange(nx)) % nx
    rho, ux, uy, T = r.rho, r.ux, r.uy, r.T
    assert np.abs(ux).max() > 1e-8  # the spot really drives a flow
    np.testing.assert_allclose(rho[:, mir], rho, rtol=1e-12)
    np.testing.assert_allclose(-ux[:, mir], ux, atol=1e-14)
    np.testing.assert_allclose(uy[:, mir], uy, atol=1e-14)
    np.testing.assert_allclose(T[:, mir], T, rtol=1e-13)


def test_fluctuating_bottom_temperature_statistics():
    cfg = W.RunConfig(nx=256, nf=4, ns=4, liquid_rows=4, bc_mode="noise", isothermal=True,
                      frozen_flow=True, bc_noise=0.01, init_noise=0.0)
    r = O.OracleRun(cfg)
    tb = 0.96 * r.Tc
    rows = []
    for _ in range(4):
        r.step(1)
        rows.append(r.T[0].copy())
    rows = np.array(rows)
    assert np.all(np.abs(rows / tb - 1) <= 0.01)
    assert abs((rows / tb - 1).mean()) < 0.002
    assert (rows / tb - 1).std() == pytest.approx(0.01 / math.sqrt(3), rel=0.1)
    assert not np.array_equal(rows[0], rows[1])


def test_flat_interface_coexistence_matches_maxwell():
    """Sec. 3.1: at 0.86 Tc the two phases must sit at the Maxwell densities.
    Pins the improved forcing of Eq. 9 with the default varpi: without the
    epsilon term (varpi = 0) the vapour density is off by tens of percent."""
    rl, rv, _ = O.maxwell(0.86)
    cfg = W.periodic_box(4, 160, liquid_rows=80)
    r = O.OracleRun(cfg)
    r.step(10000)
    rho = r.rho[:, 0]
    assert r.err == 0
    assert rho[40] == pytest.approx(rl, rel=0.02)
    assert rho[120] == pytest.approx(rv, rel=0.02)
    plain = O.OracleRun(cfg.replace(varpi=0.0))
    plain.step(10000)
    assert abs(plain.rho[120, 0] / rv - 1) > 0.2


def test_laplace_law_for_drops_in_a_periodic_box():
    """Young-Laplace in 2-D: a drop's pressure jump is sigma / R, so
    dp * R is the same for every radius.  Three drops (R about 9 to 16) in a
    64^2 periodic box at T_sat, 2000 steps: the jump between the bulk inside
    and the bulk outside, p_EOS(rho_in) - p_EOS(rho_out) (the pseudopotential
    pressure equals p_EOS by Eq. 12), times the equivalent radius of the
    liquid area, agrees across the drops to 6 %, and the jump falls with R."""
    from paper_1911_10747_gb300 import validation as V
    n = 64
    cfg = V.laplace_config(n, "fp64")
    T = cfg.T_sat_over_Tc * V.critical_temperature(cfg.a, cfg.b, cfg.R)
    out = []
    for R0 in (10.0, 13.0, 16.0):
        o = O.OracleRun(cfg)
        rho = V.disc_density(cfg, R0)
        o.set_f(WL[:, None, None] * rho[None])
        o.set_T(np.full((cfg.t_rows, n), T))
        o.step(2000)
        assert o.err == 0
        rho = o.rho
        c = (n - 1) // 2
        rin = rho[c - 1:c + 2, c - 1:c + 2].mean()
        rout = np.mean([rho[0, 0], rho[0, -1], rho[-1, 0], rho[-1, -1]])
        R = math.sqrt(np.sum((rho - rout) / (rin - rout)) / math.pi)
        dp = O.pressure(rin, T) - O.pressure(rout, T)
        out.append((R, dp))
    dpR = [R * dp for R, dp in out]
    assert out[0][1] > out[1][1] > out[2][1] > 0
    assert max(dpR) / min(dpR) - 1 < 0.06, out


@pytest.mark.parametrize("liquid_rows", [0, 7, 20, 32])
def test_vapour_fraction_counts_the_vapour_rows_of_a_layered_state(liquid_rows):
    """Frozen flow keeps the initial layer exactly (liquid rho_L below, vapour
    rho_V above, no noise): the vapour fraction (sites with rho below
    (rho_L + rho_V) / 2) is the share of vapour rows, and the mass is the
    sum of the layer densities."""
    nx, nf = 8, 32
    cfg = W.RunConfig(nx=nx, nf=nf, ns=4, liquid_rows=liquid_rows, frozen_flow=True, isothermal=True,
                      init_noise=0.0, bc_mode="spots", g=0.0)
    r = O.OracleRun(cfg)
    r.step(2)
    d = r.diagnostics()
    assert d["vapour_fraction"] == (nf - liquid_rows) / nf
    assert d["mass"] == pytest.approx(nx * (liquid_rows * cfg.rho_L + (nf - liquid_rows) * cfg.rho_V), rel=1e-14)


def test_vapour_fraction_threshold_is_the_mean_coexistence_density():
    """Sites just below (rho_L + rho_V) / 2 count as vapour, sites at or just
    above it do not: a wrong threshold or comparison changes the count."""
    nx, nf = 8, 16
    cfg = W.RunConfig(nx=nx, nf=nf, ns=4, liquid_rows=8, frozen_flow=True, isothermal=True,
                      init_noise=0.0, bc_mode="spots", g=0.0)
    r = O.OracleRun(cfg)
    thr = 0.5 * (cfg.rho_L + cfg.rho_V)
    rng = np.random.default_rng(11)
    pick = rng.integers(0, 3, size=(nf, nx))
    rho = np.choose(pick, [thr * (1 - 1e-9), thr, thr * (1 + 1e-9)])
    f = np.zeros((9, nf, nx))
    f[0] = rho  # all mass at rest: the zeroth moment is rho without rounding
    r.set_f(f)
    r.step(1)
    np.testing.assert_array_equal(r.rho, rho)
    assert r.diagnostics()["vapour_fraction"] == np.count_nonzero(r.rho < thr) / (nx * nf)
    assert r.diagnostics()["vapour_fraction"] == np.count_nonzero(pick == 0) / (nx * nf)


def test_sine_bottom_condition_phase_amplitude_and_window():
    """Sec. 3.2's fluctuating wall: T_b + 0.02 Tc sin(2 pi (x - lambda/4) /
    lambda) strictly inside t0 < n < t1, the plain T_b outside.  With
    lambda = 24 the minimum sits on column 0, the zero crossing on column 6,
    the maximum on column 12, and two whole wavelengths average to T_b."""
    nx, lam = 48, 24.0
    cfg = W.RunConfig(nx=nx, nf=8, ns=4, liquid_rows=4, frozen_flow=True, isothermal=True,
                      bc_mode="sine", init_noise=0.0, T_b_over_Tc=1.1, g=0.0,
                      sine_amp_over_Tc=0.02, sine_wavelength=lam, sine_t0=1, sine_t1=4)
    r = O.OracleRun(cfg)
    tc = r.Tc
    tb = 1.1 * tc
    seen = {}
    for n in range(5):  # step n -> n + 1 imposes T_b(x, n) on row 0
        r.step(1)
        seen[n] = r.T[0].copy()
    for n in (0, 1, 4):
        np.testing.assert_array_equal(seen[n], np.full(nx, tb))
    x = np.arange(nx)
    want = tb + 0.02 * tc * np.sin(2 * np.pi * (x - lam / 4) / lam)
    for n in (2, 3):
        np.testing.assert_allclose(seen[n], want, rtol=1e-14)
        assert seen[n][0] == pytest.approx(tb - 0.02 * tc, rel=1e-14)
        assert seen[n][12] == pytest.approx(tb + 0.02 * tc, rel=1e-14)
        assert seen[n][6] == pytest.approx(tb, rel=1e-14)
        assert seen[n].mean() == pytest.approx(tb, rel=1e-14)


@pytest.mark.parametrize("top_mode", ["outflow", "wall"])
def test_open_top_keeps_a_uniform_flow_uniform(top_mode):
    """A uniform horizontal flow at uniform density (equilibrium populations,
    no gravity, no wall adhesion) is a steady state of the interior.  With
    the open top (psi continued with zero normal gradient, the unknown
    downward populations taken from the top row itself) the rows above the
    disturbance climbing from the bottom wall -- two rows per step, one
    through the psi stencil and one through streaming -- stay exactly
    uniform after three steps; a top wall (bounce-back, no psi above)
    changes the top row at once."""
    nx, nf, U = 12, 16, 0.02
    cfg = W.RunConfig(nx=nx, nf=nf, ns=4, liquid_rows=nf, top_mode=top_mode, isothermal=True,
                      init_noise=0.0, g=0.0, bc_mode="spots", spot_x=(), c_w_spot=(), c_w_base=0.0)
    r = O.OracleRun(cfg)
    feq = O.inverse_moments(O.meq(cfg.rho_L, U, 0.0))
    f0 = np.broadcast_to(feq[:, None, None], (9, nf, nx)).copy()
    r.set_f(f0)
    r.step(3)
    f = r.f
    if top_mode == "outflow":
        np.testing.assert_allclose(f[:, 8:, :], f0[:, 8:, :], rtol=1e-13, atol=0)
        np.testing.assert_allclose(r.ux[8:], U, rtol=1e-12)
        np.testing.assert_allclose(r.uy[8:], 0.0, atol=1e-16)
    else:
        assert np.max(np.abs(f[:, -1, :] - f0[:, -1, :])) > 1e-6
    # the bottom wall disturbs only the rows it has reached
    assert np.max(np.abs(f[:, 0, :] - f0[:, 0, :])) > 1e-6


def test_momentum_changes_by_the_total_force_in_a_periodic_box():
    """Doubly periodic, no walls: the psi-psi force of Eq. 11 sums to zero
    over the box (each pair of sites pulls equally and oppositely) and
    streaming moves populations without changing their sums, so one step
    changes the population momentum by the sum of Eq. 15 alone,
    -g (M - N rho_bar) in y and nothing in x -- exactly, given the
    half-force velocity of Eq. 10 and the forcing moments of Eq. 7 / 9.
    rho_bar is set away from the true mean so that the sum is not zero."""
    nx, ny, g = 24, 20, 3e-4
    cfg = W.periodic_box(nx, ny, liquid_rows=8, init_noise=1e-2).replace(g=g)
    r = O.OracleRun(cfg)
    r.step(5)  # interfaces move: the psi force is far from zero site by site
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
    f = r.f
    M = f.sum()
    rho_bar = M / (nx * ny) + 0.05
    r.set_rho_bar(rho_bar)
    jx0, jy0 = np.tensordot(ex, f, 1).sum(), np.tensordot(ey, f, 1).sum()
    r.step(1)
    f1 = r.f
    jx1, jy1 = np.tensordot(ex, f1, 1).sum(), np.tensordot(ey, f1, 1).sum()
    want = -g * (M - nx * ny * rho_bar)
    assert abs(want) > 1e-3
    assert jy1 - jy0 == pytest.approx(want, rel=1e-10)
    assert abs(jx1 - jx0) < 1e-12 * M
    assert f1.sum() == pytest.approx(M, rel=1e-14)
    # the box is not at rest: the forces cancel in the sum, not site by site
    assert np.max(r.rho * np.hypot(r.ux, r.uy)) > 1e-4


@pytest.mark.parametrize("scale", [1.0, 1.2, 0.0])
def test_neutral_wall_adhesion_cancels_the_missing_psi_neighbours(scale):
    """Uniform liquid at rest over the heater, open top, no gravity.  On the
    fluid row next to the wall the psi force of Eq. 11 lacks its three solid
    neighbours: F_y = -G psi^2 (1/3 + 2/12) = psi^2 / 2 with G = -1.  The
    adhesion of Eq. 14 from those neighbours, -psi sum w c_w e, adds
    psi c_w / 2.  With c_w = -psi(rho_L, T_sat) the two cancel: without the
    varpi term of Eq. 9 the fluid stays exactly at rest; with it (it uses
    |F_m|^2, not zero on the wall row) one step keeps u = 0 everywhere and
    changes the populations of the two rows next to the wall only.  Any
    other c_w sets the wall row in motion at once."""
    nx, nf = 12, 10
    probe = W.RunConfig(nx=nx, nf=nf, ns=4, liquid_rows=nf)
    r0 = O.OracleRun(probe)
    psi_l, bad = O.psi(probe.rho_L, probe.T_sat_over_Tc * r0.Tc)
    assert not bad and psi_l > 0
    base = probe.replace(top_mode="outflow", isothermal=True, g=0.0, init_noise=0.0,
                         bc_mode="spots", spot_x=(), c_w_spot=(), c_w_base=-scale * psi_l)
    r = O.OracleRun(base)
    f0 = r.f
    r.step(1)
    umax = np.max(np.hypot(r.ux, r.uy))
    if scale != 1.0:
        assert np.max(np.abs(r.uy[0])) > 1e-5 and np.max(np.abs(r.uy[1:])) == 0.0
        return
    assert umax < 1e-16
    np.testing.assert_allclose(r.f[:, 2:, :], f0[:, 2:, :], rtol=1e-14, atol=0)
    assert np.max(np.abs(r.f[:, 0, :] - f0[:, 0, :])) > 1e-3
    r = O.OracleRun(base.replace(varpi=0.0))
    r.step(5)
    np.testing.assert_allclose(r.f, f0, rtol=1e-13, atol=0)
    assert np.max(np.hypot(r.ux, r.uy)) < 1e-15


@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_shear_wave_decays_at_the_phase_viscosity(phase):
    """Eq. 4-5: s7 = s8 = 1 / tau(rho), tau = tau_V + (rho - rho_V) / (rho_L -
    rho_V) (tau_L - tau_V), tau = 3 nu + 1/2.  A shear wave u_x = U sin(k y) in
    a uniform periodic box (no psi force: the density is uniform) decays as
    exp(-nu k^2 t); its measured rate gives nu_L = 0.1 in the liquid and
    nu_V = 1/6 in the vapour to within the lattice's O(k^2) error."""
    nx, ny, U = 4, 64, 1e-3
    cfg = W.periodic_box(nx, ny, liquid_rows=ny if phase == "liquid" else 0, init_noise=0.0)
    rho = cfg.rho_L if phase == "liquid" else cfg.rho_V
    nu = cfg.nu_L if phase == "liquid" else cfg.nu_V
    r = O.OracleRun(cfg)
    k = 2 * np.pi / ny
    y = np.arange(ny)
    f = np.zeros((9, ny, nx))
    for j in range(ny):
        f[:, j, :] = O.inverse_moments(O.meq(rho, U * np.sin(k * y[j]), 0.0))[:, None]
    r.set_f(f)

    def amplitude():
        return 2.0 / ny * float(np.sum(r.ux.mean(axis=1) * np.sin(k * y)))

    r.step(20)
    a0 = amplitude()
    n = 300
    r.step(n)
    a1 = amplitude()
    rate = -np.log(a1 / a0) / (n * k * k)
    assert rate == pytest.approx(nu, rel=5e-3)
    # a shear wave still: u_y and the density ripple are second order in U
    assert np.abs(r.uy).max() < 1e-6 * U and np.abs(r.rho - rho).max() < U * U * rho


def test_phase_change_source_responds_to_the_velocity_divergence():
    """Eq. 24's source -T / (rho C_V) (dp/dT)_rho div u, alone: uniform
    density and temperature (no psi force, no gradient of T) under a
    compressive wave u_x = U sin(k x).  The Eq. 27 divergence of that field is
    U sin(k) cos(k x), so one step changes T by
    -T0 (dp/dT)_rho(rho, T0) / (rho C_V) U sin(k) cos(k x), up to terms of
    second order in U."""
    nx, ny, U = 16, 4, 1e-4
    cfg = W.periodic_box(nx, ny, liquid_rows=ny, isothermal=False, init_noise=0.0)
    r = O.OracleRun(cfg)
    rho, T0 = cfg.rho_L, r.T[0, 0]
    k = 2 * np.pi / nx
    x = np.arange(nx)
    f = np.zeros((9, ny, nx))
    for i in range(nx):
        f[:, :, i] = O.inverse_moments(O.meq(rho, U * np.sin(k * x[i]), 0.0))[:, None]
    r.set_f(f)
    r.step(1)
    dT = r.T - T0
    want = -T0 * O.dpdT(rho, T0) / (rho * cfg.c_v) * U * np.sin(k) * np.cos(k * x)
    np.testing.assert_allclose(dT, np.broadcast_to(want, (ny, nx)), rtol=1e-3, atol=1e-3 * np.abs(want).max())
    assert np.abs(want).max() > 1e-7


def test_advection_moves_a_temperature_wave_downstream():
    """Eq. 24's -u . grad T with the Eq. 27 gradient: a uniform flow U along
    x over T = T0 + eps sin(k x) (long wave, 64 columns).  The gradient of the
    wave is eps sin(k) cos(k x), so one step adds -eps U sin(k) cos(k x): the
    wave moves downstream.  Conduction and the psi-mediated source act in
    phase with sin(k x) (they change the amplitude, not the phase) and enter
    the cos(k x) part only at second order."""
    nx, ny, U = 64, 4, 0.02
    cfg = W.periodic_box(nx, ny, liquid_rows=ny, isothermal=False, init_noise=0.0)
    r = O.OracleRun(cfg)
    rho, T0 = cfg.rho_L, r.T[0, 0]
    eps = 1e-4 * T0
    k = 2 * np.pi / nx
    x = np.arange(nx)
    feq = O.inverse_moments(O.meq(rho, U, 0.0))
    r.set_f(np.broadcast_to(feq[:, None, None], (9, ny, nx)).copy())
    r.set_T(np.broadcast_to(T0 + eps * np.sin(k * x), (ny, nx)))
    r.step(1)
    dT = (r.T - T0).mean(axis=0)
    cos_part = 2.0 / nx * np.sum(dT * np.cos(k * x))
    assert cos_part == pytest.approx(-eps * U * np.sin(k), rel=2e-3)


def test_initial_state_layers_noise_rest_and_saturation():
    """Sec. 3.1's start: liquid below, vapour above, at rest, T = T_sat in
    fluid and heater.  Each site's density carries the relative noise
    A (2U - 1), U the counter-based draw of (seed, tag 1, step 0, site); the
    populations are the rest equilibrium w_i rho; rho_bar is the fluid mean."""
    nx, nf, lr, A = 24, 30, 11, 1e-3
    cfg = W.RunConfig(nx=nx, nf=nf, ns=5, liquid_rows=lr, init_noise=A, seed=17)
    r = O.OracleRun(cfg)
    rho, f = r.rho, r.f
    base = np.where(np.arange(nf)[:, None] < lr, cfg.rho_L, cfg.rho_V) * np.ones((1, nx))
    U = np.array([[O.uniform(17, 1, 0, y * nx + x) for x in range(nx)] for y in range(nf)])
    np.testing.assert_allclose(rho / base - 1.0, A * (2 * U - 1), rtol=0, atol=1e-15)
    assert np.all(np.abs(rho / base - 1.0) <= A)
    np.testing.assert_allclose(f.sum(axis=0), rho, rtol=1e-15)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    np.testing.assert_allclose(f, w[:, None, None] * rho[None], rtol=1e-15)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    assert np.abs(np.tensordot(ex, f, 1)).max() < 1e-15 and np.abs(np.tensordot(ey, f, 1)).max() < 1e-15
    np.testing.assert_allclose(r.T, 0.86 * r.Tc, rtol=1e-15)
    assert r.T.shape == (nf + 5, nx)
    assert r.rho_bar == pytest.approx(rho.mean(), rel=1e-14)


@pytest.mark.parametrize("scale", [1.0, 0.0])
def test_neutral_top_wall_keeps_saturated_vapour_at_rest(scale):
    """The lid's adhesion c_w_top (Eq. 14 on the top wall): uniform vapour at
    T_sat between the two walls, no gravity, no varpi term.  With
    c_w_top = c_w = -psi(rho_V, T_sat) both wall rows feel no net force and the
    vapour stays exactly at rest; without the lid's adhesion the top row
    moves."""
    nx, nf = 12, 10
    probe = W.RunConfig(nx=nx, nf=nf, ns=4, liquid_rows=0)
    psi_v, bad = O.psi(probe.rho_V, probe.T_sat_over_Tc * O.OracleRun(probe).Tc)
    assert not bad and psi_v > 0
    cfg = probe.replace(isothermal=True, g=0.0, init_noise=0.0, varpi=0.0, bc_mode="spots", spot_x=(),
                        c_w_spot=(), c_w_base=-psi_v, c_w_top=-scale * psi_v)
    r = O.OracleRun(cfg)
    f0 = r.f
    r.step(3)
    if scale == 1.0:
        np.testing.assert_allclose(r.f, f0, rtol=1e-13, atol=0)
        assert np.max(np.hypot(r.ux, r.uy)) < 1e-16
    else:
        assert np.max(np.abs(r.uy[-1])) > 1e-5 and np.max(np.abs(r.uy[0])) < 1e-16


def test_nucleate_spot_layout_and_adhesion_stencil():
    """One spot on column 0 with half width 1 (columns 23, 0, 1 of 24: it
    wraps), the rest of the wall neutral for the liquid (c_w = -psi(rho_L)).
    Eq. 14 reads c_w from the three solid neighbours x - 1, x, x + 1, so after
    one step the wall row moves vertically on columns 22 .. 2 only, and
    horizontally on 22, 23, 1, 2 with u_x mirror-antisymmetric about column
    0, where it vanishes; no other row moves yet."""
    nx, nf = 24, 8
    probe = W.RunConfig(nx=nx, nf=nf, ns=4, liquid_rows=nf)
    psi_l, _ = O.psi(probe.rho_L, probe.T_sat_over_Tc * O.OracleRun(probe).Tc)
    cfg = probe.replace(isothermal=True, g=0.0, init_noise=0.0, varpi=0.0, top_mode="outflow",
                        bc_mode="spots", spot_x=(0,), spot_half_width=1, c_w_spot=(-0.5 * psi_l,),
                        c_w_base=-psi_l)
    r = O.OracleRun(cfg)
    r.step(1)
    uy0, ux0 = r.uy[0], r.ux[0]
    moving = {22, 23, 0, 1, 2}
    for x in range(nx):
        if x in moving:
            assert abs(uy0[x]) > 1e-6, x
        else:
            assert uy0[x] == 0.0, x
    assert ux0[0] == 0.0
    assert abs(ux0[23]) > 1e-7 and ux0[1] == pytest.approx(-ux0[23], rel=1e-12)
    assert abs(ux0[22]) > 1e-7 and ux0[2] == pytest.approx(-ux0[22], rel=1e-12)
    assert all(ux0[x] == 0.0 for x in range(3, 22))
    assert np.abs(r.uy[1:]).max() == 0.0 and np.abs(r.ux[1:]).max() == 0.0
