"""Pins of the FP64 oracle against values the paper prints, closed forms,
textbook definitions and invariants (no GPU).  Each test states what a
plausible mistake in the oracle would break."""
import math

import numpy as np
import pytest

from oracle import oracle as O

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def feq_textbook(rho, u):
    """Second-order D2Q9 equilibrium (Qian, d'Humieres, Lallemand 1992)."""
    eu = E @ u
    return W * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u @ u))


def guo_force(u, F):
    """Guo, Zheng, Shi (2002) discrete force term without the (1 - 1/2tau) factor."""
    eu, eF = E @ u, E @ F
    return W * (3 * ((E - u) @ F) + 9 * eu * eF)


def test_velocity_set_and_transfer_matrix_match_eq2_eq6(golden):
    """Column j of M is M e_j; a transposed or reordered M, or a different
    velocity ordering, changes the moments of the unit populations."""
    Mg = np.array(golden["transfer_matrix"]["M"], float)
    Eg = np.array(golden["velocities"]["e"], float)
    assert np.array_equal(Eg, E)
    for j in range(9):
        unit = np.zeros(9)
        unit[j] = 1.0
        assert np.array_equal(O.moments(unit), Mg[:, j])
    # moments 3 and 5 are the momentum components of Eq. 10
    f = np.random.default_rng(0).random(9)
    m = O.moments(f)
    assert m[3] == pytest.approx(E[:, 0] @ f, abs=1e-15)
    assert m[5] == pytest.approx(E[:, 1] @ f, abs=1e-15)


def test_inverse_transform_round_trip():
    rng = np.random.default_rng(1)
    for _ in range(20):
        f = rng.normal(size=9)
        np.testing.assert_allclose(O.inverse_moments(O.moments(f)), f, rtol=0, atol=1e-14)
        m = rng.normal(size=9)
        np.testing.assert_allclose(O.moments(O.inverse_moments(m)), m, rtol=0, atol=1e-14)


def test_equilibrium_moments_are_moments_of_textbook_equilibrium():
    """Eq. 6's m_eq equals M f_eq of the standard D2Q9 equilibrium."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        rho = rng.uniform(0.3, 7.0)
        u = rng.uniform(-0.1, 0.1, size=2)
        np.testing.assert_allclose(O.meq(rho, u[0], u[1]), O.moments(feq_textbook(rho, u)),
                                   rtol=1e-13, atol=1e-14)


def test_forcing_term_is_moments_of_guo_force():
    """With varpi = 0, S-bar of Eq. 9 equals M S_Guo.  This fixes the sign of
    the last entry (u_x F_y + u_y F_x; the printed minus fails here)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        u = rng.uniform(-0.1, 0.1, size=2)
        F = rng.uniform(-0.01, 0.01, size=2)
        S = O.source(u[0], u[1], F[0], F[1], varpi=0.0)
        np.testing.assert_allclose(S, O.moments(guo_force(u, F)), rtol=1e-12, atol=1e-16)


def test_collision_reduces_to_bgk_with_guo_forcing():
    """With every rate equal to 1/tau and varpi = 0, Eq. 7 is the BGK collision
    with Guo forcing: f* = f - (f - f_eq(rho, u)) / tau + (1 - 1/(2 tau)) S_Guo,
    u = (sum e f + F/2) / rho."""
    rng = np.random.default_rng(4)
    for tau in (0.7, 1.0, 1.3):
        s = np.full(9, 1.0 / tau)
        for _ in range(10):
            rho = rng.uniform(0.3, 7.0)
            f = feq_textbook(rho, rng.uniform(-0.05, 0.05, 2)) + rng.normal(scale=1e-3, size=9)
            F = rng.uniform(-0.01, 0.01, size=2)
            u = (E.T @ f + F / 2) / f.sum()
            ref = f - (f - feq_textbook(f.sum(), u)) / tau + (1 - 0.5 / tau) * guo_force(u, F)
            got = O.collide_site(f, F[0], F[1], s=s, varpi=0.0)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_collision_conserves_mass_and_adds_force_to_momentum():
    """Whatever the rates and the epsilon term: sum f* = sum f and
    sum e f* = sum e f + F (the forcing of Eq. 7 and Eq. 10)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        f = rng.uniform(0.01, 1.0, size=9)
        F = rng.uniform(-0.01, 0.01, size=2)
        Fm = rng.uniform(-0.01, 0.01, size=2)
        s = rng.uniform(0.6, 1.9, size=9)
        out = O.collide_site(f, F[0], F[1], Fm[0], Fm[1], psi_=1.3, varpi=0.11, s=s)
        assert out.sum() == pytest.approx(f.sum(), rel=1e-14)
        np.testing.assert_allclose(E.T @ out, E.T @ f + F, rtol=0, atol=1e-14)


def test_critical_temperature_reading(golden):
    g = golden["critical_temperature"]
    assert O.Tc(3 / 49, 2 / 21, 1.0) == pytest.approx(g["Tc"], abs=g["abs_tol"])
    # the printed a = 2/49 gives a critical temperature 2/3 as large
    assert O.Tc(2 / 49, 2 / 21, 1.0) == pytest.approx(O.Tc(3 / 49, 2 / 21, 1.0) * 2 / 3, rel=1e-14)


def test_pressure_has_a_critical_point_at_Tc():
    """At T = Tc the PR isotherm has an inflection with zero slope (to the
    rounding of the constants 0.45724 and 0.0778); below Tc the slope turns
    negative (van der Waals loop), above Tc it stays positive."""
    tc = O.Tc()
    rho = np.linspace(0.2, 6.0, 4000)
    h = 1e-5

    def slope(T):
        return (O.pressure(rho + h, T) - O.pressure(rho - h, T)) / (2 * h)

    s_c = slope(tc)
    p_scale = O.pressure(np.array([2.5]), tc)[0] / 2.5
    assert abs(s_c.min()) < 2e-3 * p_scale
    assert slope(0.95 * tc).min() < 0 < slope(1.05 * tc).min()


def test_dpdT_matches_finite_difference_of_pressure():
    tc = O.Tc()
    rng = np.random.default_rng(6)
    for _ in range(20):
        rho, T = rng.uniform(0.3, 7.0), rng.uniform(0.7, 1.3) * tc
        h = T * 1e-6
        fd = (O.pressure(rho, T + h) - O.pressure(rho, T - h)) / (2 * h)
        assert float(O.dpdT(rho, T)) == pytest.approx(float(fd), rel=1e-7)


def test_psi_reproduces_eos_pressure():
    """Eq. 12 is chosen so that the pseudopotential pressure rho/3 + G psi^2/2
    equals p_EOS; the radicand is positive at both coexistence densities."""
    tc = O.Tc()
    for rho in (0.38, 1.0, 3.0, 6.5):
        ps, bad = O.psi(rho, 0.86 * tc)
        assert not bad and ps > 0
        assert rho / 3 + (-1.0) * ps * ps / 2 == pytest.approx(float(O.pressure(rho, 0.86 * tc)), rel=1e-12)


def test_maxwell_construction_matches_paper(golden):
    g = golden["coexistence_0p86Tc"]
    rl, rv, ps = O.maxwell(g["T_over_Tc"])
    assert rl == pytest.approx(g["rho_L"], abs=g["abs_tol"])
    assert rv == pytest.approx(g["rho_V"], abs=g["abs_tol"])
    tc = O.Tc()
    # equal pressures at both roots
    assert float(O.pressure(rl, 0.86 * tc)) == pytest.approx(ps, rel=1e-9)
    assert float(O.pressure(rv, 0.86 * tc)) == pytest.approx(ps, rel=1e-9)


def test_latent_heat_matches_paper_reading(golden):
    g = golden["latent_heat"]
    h = O.latent_heat(g["T_over_Tc"], a=3 / 49)
    assert h == pytest.approx(g["h_LV"], rel=g["rel_tol"])


def test_splitmix64_reference_outputs(golden):
    g = golden["splitmix64"]
    assert O.splitmix64_sequence(0, 1)[0] == int(g["seed0_first"], 16)
    assert O.splitmix64_sequence(1234567, 3) == g["seed1234567_first3"]


def test_uniform_draws_are_uniform_and_counter_based():
    u = np.array([O.uniform(7, 2, 5, i) for i in range(20000)])
    assert (u >= 0).all() and (u < 1).all()
    assert u.mean() == pytest.approx(0.5, abs=0.01)
    assert u.var() == pytest.approx(1 / 12, abs=0.003)
    # depends on every counter, and only on the counters
    assert O.uniform(7, 2, 5, 3) == O.uniform(7, 2, 5, 3)
    others = {O.uniform(8, 2, 5, 3), O.uniform(7, 1, 5, 3), O.uniform(7, 2, 6, 3), O.uniform(7, 2, 5, 4)}
    assert O.uniform(7, 2, 5, 3) not in others and len(others) == 4


def test_isotropic_gradient_and_laplacian_closed_forms():
    """Eq. 27 is the central difference (phi(x+1) - phi(x-1)) / 2 along each
    axis for fields uniform in the other axis, exact on linear fields; Eq. 28
    is exact on quadratics; on a Fourier mode cos(k x) the Laplacian
    eigenvalue is 2 (cos k - 1) and the gradient of sin(k x) is sin k cos(k x)."""
    ny, nx = 12, 16
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    phi = 0.3 * x - 1.7 * y + 2.0
    gx, gy, lap = O.grad_lap(phi)
    inner = (slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(gx[inner], 0.3, atol=1e-13)
    np.testing.assert_allclose(gy[inner], -1.7, atol=1e-13)
    np.testing.assert_allclose(lap[inner], 0.0, atol=1e-12)
    q = 0.5 * x ** 2 + 0.25 * y ** 2 - 0.1 * x * y
    _, _, lap = O.grad_lap(q)
    np.testing.assert_allclose(lap[inner], 1.5, atol=1e-11)
    k = 2 * math.pi * 3 / nx
    gx, gy, lap = O.grad_lap(np.cos(k * x))
    np.testing.assert_allclose(lap, 2 * (math.cos(k) - 1) * np.cos(k * x), atol=1e-13)
    gx, gy, _ = O.grad_lap(np.sin(k * x))
    np.testing.assert_allclose(gx, math.sin(k) * np.cos(k * x), atol=1e-13)
    np.testing.assert_allclose(gy, 0.0, atol=1e-13)


@pytest.mark.parametrize("omega", [0.1, 0.2, 0.344, 0.5])
def test_peng_robinson_reproduces_its_acentric_factor(omega):
    """The kappa(omega) correlation of the PR EOS (Eq. 13) was fitted so that
    the EOS returns the acentric factor it is given: omega = -log10(p_sat at
    0.7 Tc / p_c) - 1, with p_c = 0.07780 R Tc / b the PR critical pressure.
    The oracle's Maxwell construction at 0.7 Tc recovers omega to 0.01 over a
    range of omega -- a check of kappa and of the PR form together."""
    import math
    a, b, R = 2.0 / 49.0, 2.0 / 21.0, 1.0
    rl, rv, ps = O.maxwell(0.7, a=a, b=b, R=R, omega=omega)
    pc = 0.07780 * R * O.Tc(a, b, R) / b
    assert -math.log10(ps / pc) - 1.0 == pytest.approx(omega, abs=0.01)
