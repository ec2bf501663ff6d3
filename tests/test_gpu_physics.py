"""Physical properties of the method checked directly on the CUDA paths (the
FP32 path that the benchmark times, and the FP64 path): the same cases that
pin the oracle, with the GPU's own runs as the measurement."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


def _tsat(cfg):
    return cfg.T_sat_over_Tc * O.OracleRun(cfg).Tc


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_shear_wave_decays_at_the_phase_viscosity(precision, phase):
    """Eq. 4-5: a shear wave in a uniform periodic box decays as
    exp(-nu k^2 t), nu = 0.1 in the liquid and 1/6 in the vapour."""
    nx, ny, U = 4, 64, 5e-3
    cfg = W.periodic_box(nx, ny, liquid_rows=ny if phase == "liquid" else 0, init_noise=0.0,
                         precision=precision)
    rho = cfg.rho_L if phase == "liquid" else cfg.rho_V
    nu = cfg.nu_L if phase == "liquid" else cfg.nu_V
    k = 2 * np.pi / ny
    y = np.arange(ny)
    f = np.zeros((9, ny, nx))
    for j in range(ny):
        f[:, j, :] = O.inverse_moments(O.meq(rho, U * np.sin(k * y[j]), 0.0))[:, None]
    g = lbm.Run(cfg)
    g.set_state(f, np.full((g.nt, nx), _tsat(cfg)), step=0)

    def amplitude():
        return 2.0 / ny * float(np.sum(g.fields(("ux",))["ux"].mean(axis=1) * np.sin(k * y)))

    g.step(20)
    a0 = amplitude()
    g.step(300)
    a1 = amplitude()
    rate = -np.log(a1 / a0) / (300 * k * k)
    assert rate == pytest.approx(nu, rel=5e-3), rate


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_neutral_wall_adhesion_keeps_the_liquid_at_rest(precision):
    """c_w = -psi(rho_L, T_sat) cancels the psi force the wall row lacks
    (Eq. 11, 14): without the varpi term the liquid stays at rest; a wall 20 %
    more attractive sets the wall row in motion."""
    nx, nf = 64, 24
    base = W.RunConfig(nx=nx, nf=nf, ns=4, liquid_rows=nf, top_mode="outflow", isothermal=True, g=0.0,
                       init_noise=0.0, bc_mode="spots", spot_x=(), c_w_spot=(), varpi=0.0,
                       precision=precision)
    psi_l, bad = O.psi(base.rho_L, _tsat(base))
    assert not bad
    umax = {}
    for scale in (1.0, 1.2):
        g = lbm.Run(base.replace(c_w_base=-scale * psi_l))
        g.step(20)
        fl = g.fields(("ux", "uy"))
        umax[scale] = float(np.max(np.hypot(fl["ux"], fl["uy"])))
    assert umax[1.0] < (1e-14 if precision == "fp64" else 1e-6), umax
    assert umax[1.2] > 1e-3, umax


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_momentum_changes_by_the_total_gravity_force(precision):
    """Doubly periodic box: one step changes the population momentum by
    -g (M - N rho_bar) in y and by nothing in x (the psi-psi force cancels
    pairwise; Eq. 10, 11, 15), with rho_bar set away from the true mean."""
    nx, ny, gv = 64, 48, 3e-4
    probe = W.periodic_box(nx, ny, liquid_rows=16, init_noise=1e-2, precision=precision)
    r = lbm.Run(probe)
    m0 = r.mass()
    rho_bar = m0 / (nx * ny) + 0.05
    g = lbm.Run(probe.replace(g=gv, rho_mean=rho_bar))
    g.step(5)
    f0 = g.fields(("f",))["f"]
    g.step(1)
    f1 = g.fields(("f",))["f"]
    M = f0.sum()
    djx = float(np.tensordot(EX, f1, 1).sum() - np.tensordot(EX, f0, 1).sum())
    djy = float(np.tensordot(EY, f1, 1).sum() - np.tensordot(EY, f0, 1).sum())
    want = -gv * (M - nx * ny * rho_bar)
    tol = 1e-10 if precision == "fp64" else 2e-2
    assert djy == pytest.approx(want, rel=tol), (djy, want)
    assert abs(djx) < tol * abs(want), djx
