"""Continuous batching: requests that arrive while others run are admitted
as slots and memory free up, the budget and slot limit hold at every tick,
each request's result is the same alone and in the mix (bitwise; FP32 and
FP16 runs alone on the multi-run kernels the batches use), and the FP64
requests' results match the oracle."""
import time

import numpy as np
import pytest

from oracle import oracle as O

from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


def requests():
    base = W.small_parity()
    return [
        (base.replace(precision="fp32"), 23),
        (base.replace(precision="fp64", rho_mean=2.42), 17),
        (base.replace(precision="fp32", nx=70, nf=45, ns=5, liquid_rows=15, spot_x=(3, 40, 69), bc_mode="noise"), 31),
        (base.replace(precision="fp32", seed=5, T_b_over_Tc=1.0), 12),
        (base.replace(precision="fp16", top_mode="outflow"), 20),
        (base.replace(precision="fp64", nx=40, nf=30, liquid_rows=10, spot_x=(5, 20, 35)), 9),
    ]


def alone(cfg, steps):
    """The request stepped by itself.  The request loop steps its runs in
    batches, and a batch steps FP32 and FP16 runs with the multi-run kernels,
    so the run alone uses those kernels too (its "multi" launch shapes)."""
    from gpu_util import select_multi
    r = select_multi(lbm.Run(cfg))
    r.step(steps)
    f = r.fields(("rho", "T"))
    return r.series(steps - 1, 1)[0], f["rho"], f["T"]


def test_requests_give_the_same_results_alone_and_in_the_mix():
    reqs = requests()
    budget = 2 * max(lbm.device_bytes(c) for c, _ in reqs) + 1
    srv = lbm.Server(hbm_budget_bytes=budget, max_active=3, chunk_steps=7)
    ids = [srv.submit(c, n, keep_fields=True) for c, n in reqs[:3]]
    for _ in range(2):
        srv.tick()
        q, a, used = srv.counts()
        assert a <= 3 and used <= budget
    ids += [srv.submit(c, n, keep_fields=True) for c, n in reqs[3:]]
    late_admitted_while_others_ran = False
    for _ in range(200):
        srv.tick()
        q, a, used = srv.counts()
        assert a <= 3 and used <= budget
        states = [srv.status(i)[0] for i in ids]
        if states[3] >= 1 and states[0] == 1:
            late_admitted_while_others_ran = True
        if all(st >= 2 for st in states):
            break
    assert all(srv.status(i)[0] == 2 for i in ids)
    assert late_admitted_while_others_ran or srv.status(ids[3])[1][1] < srv.status(ids[2])[1][2]
    for i, (c, n) in zip(ids, reqs):
        diag, rho, T = srv.result(i, fields=True)
        d0, r0, t0 = alone(c, n)
        assert np.array_equal(diag, d0), i
        assert np.array_equal(rho, r0) and np.array_equal(T, t0), i
        st, (ts, t1, t2) = srv.status(i)
        assert ts <= t1 <= t2
        if c.precision == "fp64":
            # the served FP64 run against the oracle (1e-12 per site; the two
            # sides sum the initial densities in different orders)
            o = O.OracleRun(c)
            o.step(n)
            assert np.max(np.abs(rho - o.rho) / np.abs(o.rho)) <= 1e-12, i
            assert np.max(np.abs(T - o.T) / np.abs(o.T)) <= 1e-12, i
            od = o.diagnostics()
            want = [od["q_bottom"], od["q_top"], od["vapour_fraction"], od["mass"]]
            np.testing.assert_allclose(diag, want, rtol=1e-11, atol=1e-16)
    srv.close()


def test_poll_admits_arrivals_while_a_chunk_runs():
    """lbm_server_poll does not wait for the chunk in flight: a request that
    arrives during a long chunk is admitted (its run created on its own
    stream) by the next poll, which returns long before the chunk ends; the
    request joins at the next chunk, and every result equals the run alone."""
    big = W.small_parity(precision="fp64").replace(nx=512, nf=512, ns=8, liquid_rows=170,
                                                    spot_x=W.scaled_spots(512), rho_mean=2.4)
    small = W.small_parity(precision="fp32").replace(rho_mean=2.42)
    srv = lbm.Server(hbm_budget_bytes=10**10, max_active=4, chunk_steps=400)
    a = srv.submit(big, 800, keep_fields=True)
    srv.poll()                                    # admits a, launches its first chunk
    assert srv.status(a)[0] == 1
    b = srv.submit(small, 30, keep_fields=True)
    t0 = time.perf_counter()
    srv.poll()                                    # admits b while a's chunk runs
    dt = time.perf_counter() - t0
    q, active, _ = srv.counts()
    assert srv.status(b)[0] == 1 and active == 2 and q == 0
    print("poll during a chunk took", dt, "s")
    assert dt < 0.2, dt
    deadline = time.perf_counter() + 120
    while any(srv.status(i)[0] < 2 for i in (a, b)):
        assert time.perf_counter() < deadline
        if srv.poll() == 0:
            time.sleep(0.001)
    for i, (c, n) in ((a, (big, 800)), (b, (small, 30))):
        diag, rho, T = srv.result(i, fields=True)
        d0, r0, t0_ = alone(*(c, n))
        assert np.array_equal(diag, d0) and np.array_equal(rho, r0) and np.array_equal(T, t0_), i
    srv.close()


def test_model_a_request_keeps_its_whole_temperature_field():
    """Model A (no heater): T has the heated wall's row and the fluid rows,
    NF + 1 of them; the kept fields of a served request are those of the
    same run stepped alone."""
    cfg = W.small_parity().replace(precision="fp32", ns=0)
    srv = lbm.Server(hbm_budget_bytes=4 * lbm.device_bytes(cfg), max_active=2, chunk_steps=5)
    rid = srv.submit(cfg, 12, keep_fields=True)
    for _ in range(50):
        srv.tick()
        if srv.status(rid)[0] >= 2:
            break
    diag, rho, T = srv.result(rid, fields=True)
    d0, rho0, T0 = alone(cfg, 12)
    assert T.shape == (cfg.nf + 1, cfg.nx)
    assert np.array_equal(rho, rho0) and np.array_equal(T, T0)
    assert np.array_equal(diag, d0)
    srv.close()
