"""The allocation-free diagnostics entry point (lbm_diagnostics_static).

It serves callers that cannot call cudaMalloc or cudaFree (their device
memory belongs to another allocator, or they must not risk the implicit
synchronisation of those calls): its scratch is a static device array.  Its
four values must match the library's regular per-step diagnostics of the
same state, on two calls in a row (the second call reuses the static array
the first one filled).  This file sorts last so a failure here does not stop
the other GPU tests."""
import numpy as np
import pytest

from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


CASES = {
    # heater rows under the fluid (model B)
    "heater": lambda: W.small_parity().replace(bc_mode="noise", spot_x=(), c_w_spot=(), rho_mean=2.42),
    # no heater (model A): T has one wall row below the fluid; both flux
    # slots carry the wall flux
    "model_a": lambda: W.small_parity().replace(nx=48, nf=40, ns=0, liquid_rows=13, bc_mode="noise", spot_x=(),
                                                c_w_spot=(), rho_mean=2.42),
    # periodic in y: no wall, both fluxes zero
    "periodic": lambda: W.periodic_box(40, 30, liquid_rows=10, init_noise=1e-3, isothermal=False),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_static_diagnostics_match_the_step_diagnostics_twice(case):
    torch = pytest.importorskip("torch")
    cfg = CASES[case]()
    run = lbm.Run(cfg)
    dev = torch.device("cuda", 0)
    rho = torch.empty((cfg.nf, cfg.nx), dtype=torch.float64, device=dev)
    nt = cfg.nf + (1 if cfg.model_a else cfg.ns)
    T = torch.empty((nt, cfg.nx), dtype=torch.float64, device=dev)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device=dev)
    for steps in (7, 25):
        run.step(steps)
        run.fields_device({"rho": rho.data_ptr(), "T": T.data_ptr()})
        want = run.series(run.step_count - 1, 1)[0]
        torch.cuda.synchronize(dev)
        lbm.diagnostics_static(rho.data_ptr(), T.data_ptr(), cfg, out.data_ptr())
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=TOL, atol=1e-15)
        assert 0.0 < got[2] < 1.0
        if case == "periodic":
            assert got[0] == 0.0 and got[1] == 0.0
        else:
            assert got[0] != 0.0 and got[1] != 0.0
        if case == "model_a":
            assert got[0] == got[1]


def test_static_diagnostics_reject_heater_rows_the_library_does_not_build():
    pytest.importorskip("torch")
    for ns in (1, 2):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.diagnostics_static(1, 1, W.small_parity().replace(ns=ns), 1)
        assert ei.value.code == lbm.LBM_E_INVAL


def test_static_diagnostics_reject_sizes_beyond_the_capacity():
    pytest.importorskip("torch")
    cfg = W.small_parity().replace(nx=8192, nf=4096)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.diagnostics_static(1, 1, cfg, 1)
    assert ei.value.code == lbm.LBM_E_INVAL
    assert "capacity" in str(ei.value)
