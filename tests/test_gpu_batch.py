"""Batches of runs: every run's result is the same alone and inside a mixed
batch (different sizes, precisions and bottom modes), bitwise; the FP64
members, a sweep-drawn one among them, match the oracle."""
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


def mixed_configs():
    base = W.small_parity()
    return [
        base.replace(rho_mean=2.42),
        base.replace(precision="fp32", nx=70, nf=45, ns=5, liquid_rows=15, spot_x=(3, 40, 69), rho_mean=2.3),
        base.replace(precision="fp32", bc_mode="noise", spot_x=(), c_w_spot=(), seed=9),
        W.sweep(3, seed=11)[0].replace(nf=96, liquid_rows=32),
        base.replace(precision="fp16", top_mode="outflow"),
        W.sweep(3, seed=12)[1].replace(nf=90, liquid_rows=30, precision="fp64"),
    ]


def test_results_alone_and_in_a_batch_are_identical():
    cfgs = mixed_configs()
    alone = []
    for c in cfgs:
        r = lbm.Run(c)
        r.step(21)
        alone.append(r.fields(("rho", "ux", "uy", "T", "f")))
    runs = [lbm.Run(c) for c in cfgs]
    runs[1].step(1)                 # odd parity on entry
    batch = lbm.Batch(runs)
    batch.step(13)
    runs[2].step(3)                 # interleaved single-run work stays ordered
    batch.step(4)
    batch.sync()
    # every run has now taken 17 batch steps plus its own extra ones; top all
    # up to 21 below and compare with the runs stepped alone
    for i, r in enumerate(runs):
        extra = (1 if i == 1 else 0) + (3 if i == 2 else 0)
        assert r.step_count == 17 + extra, (i, r.step_count)
        r.step(4 - extra)
        got = r.fields(("rho", "ux", "uy", "T", "f"))
        for k in got:
            assert np.array_equal(got[k], alone[i][k]), (i, k)
        if cfgs[i].precision == "fp64":
            o = O.OracleRun(cfgs[i])
            o.step(21)
            umax = max(np.abs(o.ux).max(), np.abs(o.uy).max())
            assert np.max(np.abs(got["rho"] - o.rho) / np.abs(o.rho)) <= 1e-12, i
            assert np.max(np.abs(got["T"] - o.T) / np.abs(o.T)) <= 1e-12, i
            assert np.max(np.abs(got["ux"] - o.ux)) <= 1e-12 * umax, i
    batch.close()


def test_batch_recaptures_after_variant_change():
    cfgs = [W.small_parity(precision="fp32"), W.small_parity(precision="fp32", seed=3)]
    runs = [lbm.Run(c) for c in cfgs]
    ref = [lbm.Run(c) for c in cfgs]
    b = lbm.Batch(runs)
    b.step(4)
    runs[0].select_variants(1, 1)
    ref[0].select_variants(1, 1)
    b.step(6)
    for r in ref:
        r.step(10)
    for r, q in zip(runs, ref):
        a, c = r.fields(("rho", "T")), q.fields(("rho", "T"))
        assert np.array_equal(a["rho"], c["rho"]) and np.array_equal(a["T"], c["T"])
