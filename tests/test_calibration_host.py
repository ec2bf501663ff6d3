"""Host side of the wettability calibration (no GPU): the contact-angle
measurement against drops of known geometry, and the inversion."""
import math

import numpy as np
import pytest

from paper_1911_10747_gb300 import calibration as K
from paper_1911_10747_gb300 import workloads as W


def cap_field(theta_deg, R=40.0, nx=200, nf=100, width=2.0, rho_L=6.5, rho_V=0.38):
    """A circular drop of radius R cut by the wall line y = -1/2 at angle
    theta: centre at y_c = y_wall - R cos(theta)."""
    yc = K.WALL_Y - R * math.cos(math.radians(theta_deg))
    y, x = np.mgrid[0:nf, 0:nx].astype(float)
    r = np.hypot(x - nx / 2.0, y - yc)
    return rho_V + 0.5 * (rho_L - rho_V) * (1.0 - np.tanh(2.0 * (r - R) / width))


@pytest.mark.parametrize("theta", [40.0, 55.0, 90.0, 105.0, 125.0, 140.0])
def test_contact_angle_of_a_circular_cap(theta):
    m = K.contact_angle(cap_field(theta), 6.5, 0.38)
    assert m["theta_deg"] == pytest.approx(theta, abs=0.5)
    assert m["radius"] == pytest.approx(40.0, rel=0.01)
    assert m["x_c"] == pytest.approx(100.0, abs=0.05)


def test_fit_circle_recovers_exact_points():
    t = np.linspace(0.3, 2.8, 40)
    pts = np.column_stack([7.0 + 12.0 * np.cos(t), -3.0 + 12.0 * np.sin(t)])
    xc, yc, R = K.fit_circle(pts)
    assert (xc, yc, R) == pytest.approx((7.0, -3.0, 12.0), abs=1e-10)


def test_drop_state_is_at_rest_with_the_drop_mass():
    cfg = K.drop_config(-1.2, nx=64, nf=40)
    f, T = K.drop_state(cfg, 12.0)
    rho = f.sum(axis=0)
    np.testing.assert_allclose(rho, K.drop_density(cfg, 12.0), rtol=1e-15)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    assert np.abs(np.tensordot(ex, f, 1)).max() < 1e-14
    assert np.abs(np.tensordot(ey, f, 1)).max() < 1e-14
    assert T.shape == (cfg.t_rows, cfg.nx)
    assert rho[0, 32] == pytest.approx(cfg.rho_L, rel=1e-6) and rho[-1, 0] == pytest.approx(cfg.rho_V, rel=1e-6)


def test_invert_interpolates_and_rejects_non_monotonic_tables():
    table = [{"c_w": c, "theta_deg": 90.0 + 60.0 * (c + 1.2)} for c in (-2.0, -1.6, -1.2, -0.8)]
    inv = K.invert(table, (55.0, 105.0))
    assert inv[55.0] == pytest.approx(-1.2 - 35.0 / 60.0)
    assert inv[105.0] == pytest.approx(-1.2 + 15.0 / 60.0)
    with pytest.raises(ValueError):
        K.invert(table + [{"c_w": -0.7, "theta_deg": 10.0}], (55.0,))
    with pytest.raises(ValueError):
        K.invert(table, (170.0,))
