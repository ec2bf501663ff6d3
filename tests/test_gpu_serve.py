"""Continuous batching: requests that arrive while others run are admitted
as slots and memory free up, the budget and slot limit hold at every tick,
and each request's result is the same alone and in the mix (bitwise)."""
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
    r = lbm.Run(cfg)
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
