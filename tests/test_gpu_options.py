"""Run options of lbm_opts_t on the GPU: the caller's device allocator
(PyTorch's caching allocator through the dev_alloc / dev_free callbacks) and
the step-by-step checking mode."""
import numpy as np
import pytest

from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


def test_torch_caching_allocator_holds_the_run_and_results_match():
    import torch
    cfg = W.small_parity(precision="fp32").replace(rho_mean=2.42)
    a = lbm.Run(cfg)
    a.step(50)
    want = a.fields(("rho", "T", "f"))
    a.close()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated(0)
    b = lbm.Run(cfg, allocator="torch")
    held = torch.cuda.memory_allocated(0) - before
    assert held >= 0.5 * lbm.device_bytes(cfg), (held, lbm.device_bytes(cfg))
    b.step(50)
    got = b.fields(("rho", "T", "f"))
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    b.close()
    assert torch.cuda.memory_allocated(0) == before


def test_bounds_check_mode_matches_and_reports_the_faulting_step():
    cfg = W.small_parity()  # FP64
    a = lbm.Run(cfg)
    a.step(12)
    want = a.fields(("rho", "T"))
    b = lbm.Run(cfg, bounds_check=True)
    b.step(12)
    got = b.fields(("rho", "T"))
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    c = lbm.Run(cfg, bounds_check=True)
    f = c.fields(("f",))["f"]
    f[:, 10, 10] = np.nan
    c.set_state(f, None, step=0)
    with pytest.raises(lbm.LbmError) as ei:
        c.step(5)  # the call itself reports the fault ...
    assert ei.value.code == lbm.LBM_E_NUMERIC
    assert c.step_count == 1  # ... at the step that caused it
