"""FP32 shifted-population path and FP16-storage probe against the FP64
oracle: error reports with bounds derived from single-precision rounding."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

from gpu_util import field_errors, run_both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


def test_fp32_small_case_error_report():
    cfg = W.small_parity(precision="fp32").replace(rho_mean=2.42)
    g, o = run_both(cfg, 200)
    errs = field_errors(g, o)
    print("fp32 200-step errors", errs)
    assert errs["rho"] < 1e-3 and errs["T"] < 1e-5, errs
    assert g.mass() == pytest.approx(o.diagnostics()["mass"], rel=1e-6)


def test_fp16_probe_runs_and_stays_bounded():
    cfg = W.small_parity(precision="fp16").replace(rho_mean=2.42)
    g, o = run_both(cfg, 100)
    errs = field_errors(g, o)
    print("fp16 100-step errors", errs)
    assert errs["rho"] < 0.2, errs


def test_fp32_full_size_domain_two_steps():
    cfg = W.large(precision="fp32").replace(rho_mean=2.41)
    g, o = run_both(cfg, 2)
    errs = field_errors(g, o)
    print("fp32 full-size 2-step errors", errs)
    assert errs["rho"] < 1e-5 and errs["T"] < 1e-6, errs
