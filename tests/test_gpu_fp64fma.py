"""FP64 path compiled with fused multiply-add contraction ("fp64_fma")
against the oracle: the contracted products round differently from the
oracle's separate products and sums, so results are not bit-identical, but
they must stay within a relative 1e-12 per site (u relative to max |u|)
over 200 steps of the 64 x 96 case, and on ragged, model-A, open-top and
full-size domains."""
import pytest

from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

from gpu_util import field_errors, run_both

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


def test_fp64_fma_200_steps_within_1e_12():
    cfg = W.small_parity(precision="fp64_fma")
    g, o = run_both(cfg, 200)
    e = field_errors(g, o)
    print("fp64_fma 200-step errors", e)
    assert max(e.values()) <= TOL, e
    assert g.mass() == pytest.approx(o.diagnostics()["mass"], rel=1e-13)


@pytest.mark.parametrize("kw", [
    dict(nx=70, nf=45, ns=5, liquid_rows=15, spot_x=(3, 40, 69), spot_half_width=2),
    dict(nx=48, nf=40, ns=0, liquid_rows=13, bc_mode="sine", spot_x=(), c_w_spot=(), sine_t0=5, sine_t1=50,
         sine_wavelength=24.0),
    dict(nx=40, nf=33, ns=4, liquid_rows=11, top_mode="outflow", bc_mode="noise", spot_x=(), c_w_spot=()),
])
def test_fp64_fma_edge_domains_within_1e_12(kw):
    cfg = W.small_parity(precision="fp64_fma").replace(rho_mean=2.3, **kw)
    g, o = run_both(cfg, 100)
    e = field_errors(g, o)
    assert max(e.values()) <= TOL, (kw, e)


def test_fp64_fma_full_size_two_steps():
    cfg = W.large(precision="fp64_fma").replace(rho_mean=2.41)
    g, o = run_both(cfg, 2)
    e = field_errors(g, o)
    assert max(e.values()) <= TOL, e
