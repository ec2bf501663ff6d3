"""FP32 path with the phase-change source of Eq. 24 in double-float
arithmetic (precision "fp32_dfsrc") against the FP64 oracle, next to the
all-FP32 path on the same heat-kernel shape: the comparison isolates the
error of the source term from that of FP32 storage and arithmetic."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

from gpu_util import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


def _run(cfg, steps, heat):
    g = lbm.Run(cfg)
    v = g.variants()
    g.select_variants(0, v["heat"].index(heat))
    g.step(steps)
    g.sync()
    return g


@pytest.mark.parametrize("shape", ["heatrows_64x8x4", "heatrows_64x6x5"])
def test_double_float_source_against_the_oracle_beside_fp32(shape):
    cfg = W.small_parity(precision="fp32").replace(rho_mean=2.42)
    o = O.OracleRun(cfg)
    o.step(200)
    e32 = field_errors(_run(cfg, 200, shape), o)
    edf = field_errors(_run(cfg.replace(precision="fp32_dfsrc"), 200, shape + "_dfsrc"), o)
    print(shape, "fp32", e32, "dfsrc", edf)
    for e in (e32, edf):
        assert e["rho"] < 1e-3 and e["T"] < 1e-5, e


def test_double_float_source_model_a_outflow_and_noise():
    """Model A with the sine bottom, and an open top with the noisy bottom:
    the source coefficients off the fluid rows are zero in both forms."""
    for kw in (dict(nx=48, nf=40, ns=0, liquid_rows=13, bc_mode="sine", spot_x=(), c_w_spot=(), sine_t0=5,
                    sine_t1=50, sine_wavelength=24.0),
               dict(nx=40, nf=33, ns=4, liquid_rows=11, top_mode="outflow", bc_mode="noise", spot_x=(), c_w_spot=())):
        cfg = W.small_parity(precision="fp32_dfsrc").replace(rho_mean=2.3, **kw)
        o = O.OracleRun(cfg)
        o.step(60)
        g = lbm.Run(cfg)
        g.step(60)
        g.sync()
        e = field_errors(g, o)
        assert e["rho"] < 1e-4 and e["T"] < 1e-5, (kw, e)


def test_double_float_source_full_size_two_steps():
    cfg = W.large(precision="fp32_dfsrc").replace(rho_mean=2.41)
    o = O.OracleRun(cfg)
    o.step(2)
    g = lbm.Run(cfg)
    g.autotune(2)
    g.step(2)
    g.sync()
    e = field_errors(g, o)
    assert e["rho"] < 1e-5 and e["T"] < 1e-6, e
