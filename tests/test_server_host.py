"""Host-side logic of the request loop and the memory estimate (no GPU: a
server only touches the device in lbm_server_tick)."""
import pytest

from paper_1911_10747_gb300 import build as B
from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    lbm.load()


def test_device_bytes_estimate_scales_with_size_and_precision():
    small = W.small_parity(precision="fp32")
    b32 = lbm.device_bytes(small)
    b64 = lbm.device_bytes(small.replace(precision="fp64"))
    b16 = lbm.device_bytes(small.replace(precision="fp16"))
    nfl, ntl = small.fluid_sites, small.temperature_sites
    # populations and temperature in two buffers, moments for each step parity
    assert b32 >= 2 * 9 * nfl * 4 + 2 * ntl * 4 + 6 * nfl * 4
    assert b64 >= 2 * 9 * nfl * 8 + 2 * ntl * 8 + 6 * nfl * 8
    assert b16 < b32 < b64
    big = lbm.device_bytes(W.large())
    assert 2 * 9 * 2048 * 2048 * 4 < big < 1.2e9


def test_server_queues_and_validates_without_touching_the_device():
    s = lbm.Server(hbm_budget_bytes=10**9, max_active=2, chunk_steps=5)
    ids = [s.submit(W.small_parity(precision="fp32", seed=k), 10) for k in range(3)]
    assert ids == sorted(ids) and len(set(ids)) == 3
    assert s.counts() == (3, 0, 0)
    st, times = s.status(ids[1])
    assert st == 0 and times[0] >= 0.0
    with pytest.raises(lbm.LbmError):
        s.submit(W.small_parity(), 0)  # zero steps
    with pytest.raises(lbm.LbmError):
        s.status(12345)
    s.close()


def test_server_rejects_requests_larger_than_the_budget():
    s = lbm.Server(hbm_budget_bytes=10**6, max_active=2, chunk_steps=5)
    with pytest.raises(lbm.LbmError) as ei:
        s.submit(W.small_parity(), 10)
    assert ei.value.code == lbm.LBM_E_INVAL and "budget" in str(ei.value)
    with pytest.raises(lbm.LbmError):
        lbm.Server(hbm_budget_bytes=0)
    s.close()
