"""Wettability calibration: contact angle theta -> wall coefficient c_w.

The paper prescribes contact angles (55 deg for the heater, 105 / 115 / 125
deg for the nucleate spots, Sec. 3.1 and 4.1) and says they are set through
G_w of Eq. 14, but prints no G_w.  This module measures theta(c_w) with the
library's own kernels -- isothermal sessile drops at T_sat on the bottom wall,
no gravity -- and inverts the curve.  Host code only: the drops are stepped
by the CUDA path through lbm.Batch; this file builds the initial states and
reads the angle off the density field.

Geometry: fluid row y has its centre at height y; the halfway bounce-back
wall lies at y = -1/2.  A drop's interface is the level set
rho = (rho_L + rho_V) / 2; a circle fitted to it (algebraic least squares)
gives the angle through cos(theta) = (y_wall - y_centre) / radius.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W

WALL_Y = -0.5
_WL = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def drop_config(c_w: float, nx: int = 200, nf: int = 100, precision: str = "fp32", **kw) -> W.RunConfig:
    """An isothermal, gravity-free run whose bottom wall has coefficient c_w
    everywhere (no spots).  The heater rows only hold T_sat."""
    base = dict(nx=nx, nf=nf, ns=3, liquid_rows=0, bc_mode="spots", spot_x=(), c_w_spot=(),
                c_w_base=float(c_w), isothermal=True, g=0.0, init_noise=0.0, T_b_over_Tc=0.86,
                precision=precision)
    base.update(kw)
    return W.RunConfig(**base)


def drop_density(cfg: W.RunConfig, radius: float, width: float = 2.0, theta0_deg: float = 90.0) -> np.ndarray:
    """rho[nf, nx] of a liquid disc of the given radius cut by the wall line
    at the angle theta0 (90 deg: a half disc resting on the wall), centred at
    x = nx / 2, with a tanh interface of the given width between rho_L and
    rho_V."""
    y, x = np.mgrid[0:cfg.nf, 0:cfg.nx].astype(float)
    yc = WALL_Y - radius * math.cos(math.radians(theta0_deg))
    r = np.hypot(x - cfg.nx / 2.0, y - yc)
    return cfg.rho_V + 0.5 * (cfg.rho_L - cfg.rho_V) * (1.0 - np.tanh(2.0 * (r - radius) / width))


def drop_state(cfg: W.RunConfig, radius: float, **shape):
    """(f, T) for Run.set_state: populations at rest, f_i = w_i rho (the
    equilibrium of Eq. 3 at u = 0), and T = T_sat everywhere."""
    rho = drop_density(cfg, radius, **shape)
    f = _WL[:, None, None] * rho[None, :, :]
    tc = (0.0778 * cfg.a) / (0.45724 * cfg.b * cfg.R)
    T = np.full((cfg.t_rows, cfg.nx), cfg.T_sat_over_Tc * tc)
    return f, T


def interface_points(rho: np.ndarray, level: float, y_min: float = 2.0):
    """Points of the level set rho = level of one drop, by linear
    interpolation between neighbouring sites: the left and right crossing of
    every row y >= y_min, and the top crossing of every column."""
    nf, nx = rho.shape
    pts = []
    for y in range(nf):
        if y < y_min:
            continue
        row = rho[y]
        inside = np.nonzero(row > level)[0]
        if inside.size == 0:
            continue
        i0, i1 = inside[0], inside[-1]
        if i0 > 0:
            a, b = row[i0 - 1], row[i0]
            pts.append((i0 - 1 + (level - a) / (b - a), y))
        if i1 < nx - 1:
            a, b = row[i1], row[i1 + 1]
            pts.append((i1 + (level - a) / (b - a), y))
    for x in range(nx):
        col = rho[:, x]
        inside = np.nonzero(col > level)[0]
        if inside.size == 0:
            continue
        j = inside[-1]
        if j < nf - 1 and j >= y_min:
            a, b = col[j], col[j + 1]
            pts.append((x, j + (level - a) / (b - a)))
    return np.array(pts, dtype=float)


def fit_circle(pts: np.ndarray):
    """Algebraic (Kasa) least-squares circle x^2 + y^2 + D x + E y + F = 0:
    returns (x_c, y_c, radius)."""
    x, y = pts[:, 0], pts[:, 1]
    A = np.column_stack([x, y, np.ones_like(x)])
    D, E, F = np.linalg.lstsq(A, -(x * x + y * y), rcond=None)[0]
    xc, yc = -D / 2.0, -E / 2.0
    return xc, yc, math.sqrt(max(xc * xc + yc * yc - F, 0.0))


def contact_angle(rho: np.ndarray, rho_L: float, rho_V: float) -> dict:
    """Contact angle (degrees) of the single drop in rho[nf, nx], with the
    fitted circle, the drop height above the wall and its base width."""
    level = 0.5 * (rho_L + rho_V)
    pts = interface_points(rho, level)
    xc, yc, R = fit_circle(pts)
    # a drop whose circle clears the wall by more than a lattice spacing has
    # left it (non-wetting): no contact angle
    detached = yc - R > WALL_Y + 1.0
    c = (WALL_Y - yc) / R
    theta = math.degrees(math.acos(max(-1.0, min(1.0, c))))
    return {"theta_deg": theta, "detached": bool(detached), "x_c": xc, "y_c": yc, "radius": R,
            "height": yc + R - WALL_Y, "points": int(len(pts))}


def measure(c_w_values, steps: int = 30000, radius: float = 30.0, precision: str = "fp32",
            nx: int = 200, nf: int = 100, reading: str = "stated", **shape) -> list:
    """Step one drop per c_w together (one lbm.Batch) and return the
    measured contact angle of each, with the drop's mass drift.  reading:
    "stated" (a = 2/49) or "paper_tc" (a = 3/49, the printed Tc)."""
    from . import lbm
    cfgs = [drop_config(c, nx=nx, nf=nf, precision=precision) for c in c_w_values]
    if reading == "paper_tc":
        cfgs = [W.paper_tc_reading(c) for c in cfgs]
    runs = []
    for cfg in cfgs:
        r = lbm.Run(cfg)
        f, T = drop_state(cfg, radius, **shape)
        r.set_state(f, T, step=0)
        runs.append(r)
    m0 = [float(np.sum(drop_density(c, radius, **shape))) for c in cfgs]
    batch = lbm.Batch(runs)
    batch.step(steps)
    try:
        batch.sync()
    except lbm.LbmError:
        pass  # a run that faulted is reported below; the others are valid
    out = []
    for c, cfg, r, m in zip(c_w_values, cfgs, runs, m0):
        try:
            r.sync()
        except lbm.LbmError as e:
            out.append({"c_w": float(c), "theta_deg": None, "error": str(e)})
            continue
        fl = r.fields(("rho", "ux", "uy"))
        res = contact_angle(fl["rho"], cfg.rho_L, cfg.rho_V)
        res.update(c_w=float(c), mass_drift=float(fl["rho"].sum() / m - 1.0),
                   max_u=float(np.max(np.hypot(fl["ux"], fl["uy"]))))
        out.append(res)
    batch.close()
    return out


def invert(table: list, targets_deg) -> dict:
    """c_w for each target angle by linear interpolation of the measured
    theta(c_w), which rises monotonically with c_w (less attraction, less
    wetting)."""
    t = sorted((r for r in table if r.get("theta_deg") is not None and not r.get("detached")),
               key=lambda r: r["c_w"])
    cw = np.array([r["c_w"] for r in t])
    th = np.array([r["theta_deg"] for r in t])
    if not np.all(np.diff(th) > 0):
        raise ValueError("measured contact angle is not monotonic in c_w: %s" % list(zip(cw, th)))
    res = {}
    for a in targets_deg:
        if not th[0] <= a <= th[-1]:
            raise ValueError(f"target {a} deg outside the measured range {th[0]:.1f}..{th[-1]:.1f}")
        res[float(a)] = float(np.interp(a, th, cw))
    return res


if __name__ == "__main__":  # python -m paper_1911_10747_gb300.calibration
    import json
    import sys
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 30000
    grid = [round(v, 3) for v in np.arange(-1.8, -0.95, 0.05)]
    table = measure(grid, steps=steps)
    for row in table:
        if row["theta_deg"] is None:
            print(f"c_w {row['c_w']:6.2f}  {row['error']}")
            continue
        if row["detached"]:
            print(f"c_w {row['c_w']:6.2f}  drop left the wall")
            continue
        print(f"c_w {row['c_w']:6.2f}  theta {row['theta_deg']:6.1f} deg  radius {row['radius']:5.1f}  "
              f"height {row['height']:5.1f}  mass drift {row['mass_drift']:.1e}  max|u| {row['max_u']:.1e}")
    inv = invert(table, (105.0, 115.0, 125.0))
    print(json.dumps({"steps": steps, "table": table, "c_w_for_theta": inv}))
