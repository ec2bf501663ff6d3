"""Batches of runs: every run's result is the same alone and inside a mixed
batch (different sizes, precisions and bottom modes), bitwise; the FP64
members, a sweep-drawn one among them, match the oracle.  A batch steps its
FP32 and FP16 runs with the multi-run kernels (one launch per kernel kind
over a work list of (run, tile), the FP32 runs whose width is a multiple of
64 with the wavefront flow over (run, unit)); a run stepped alone with
those kernels (the "multi" launch-shape variants) gives bit for bit the
same."""
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


def multi(run):
    from gpu_util import select_multi
    return select_multi(run)


def test_results_alone_and_in_a_batch_are_identical():
    cfgs = mixed_configs()
    alone = []
    for c in cfgs:
        r = multi(lbm.Run(c))
        r.step(21)
        alone.append(r.fields(("rho", "ux", "uy", "T", "f")))
    runs = [multi(lbm.Run(c)) for c in cfgs]
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


def test_batch_steps_its_fp32_runs_with_the_multi_run_kernels_whatever_their_variants():
    """A variant change on a run between batch steps re-captures the batch
    graph; the batch still steps its FP32 runs with the multi-run kernels,
    so they match runs stepped alone with the multi variants, bitwise, over
    even and odd step counts."""
    cfgs = [W.small_parity(precision="fp32"), W.small_parity(precision="fp32", seed=3).replace(nx=40, nf=30, liquid_rows=10, spot_x=(5, 20, 35))]
    runs = [lbm.Run(c) for c in cfgs]
    ref = [multi(lbm.Run(c)) for c in cfgs]
    b = lbm.Batch(runs)
    b.step(4)
    runs[0].select_variants(1, 1)
    b.step(7)
    b.sync()
    for r in ref:
        r.step(11)
    for r, q in zip(runs, ref):
        a, c = r.fields(("rho", "T", "f")), q.fields(("rho", "T", "f"))
        for k in a:
            assert np.array_equal(a[k], c[k]), k
        assert np.array_equal(r.series(0, 11), q.series(0, 11))
    b.close()


def test_multi_run_variants_agree_with_the_single_run_kernels_and_the_oracle():
    """The multi-run kernels do the single-run kernels' per-site arithmetic:
    against the oracle within the FP32 bounds, on a ragged domain, model A
    with the sine bottom, an open top with the noisy bottom and a doubly
    periodic box with heat, with the tiles and (widths of 128 and more in
    strips of 64) with the wavefront units."""
    from gpu_util import field_errors
    cases = [W.small_parity(precision="fp32").replace(nx=70, nf=45, ns=5, liquid_rows=15, spot_x=(3, 40, 69),
                                                       spot_half_width=2, rho_mean=2.3),
             W.small_parity(precision="fp32").replace(nx=48, nf=40, ns=0, liquid_rows=13, bc_mode="sine", spot_x=(),
                                                       c_w_spot=(), sine_t0=5, sine_t1=50, sine_wavelength=24.0,
                                                       rho_mean=2.3),
             W.small_parity(precision="fp32").replace(nx=40, nf=33, ns=4, liquid_rows=11, top_mode="outflow",
                                                       bc_mode="noise", spot_x=(), c_w_spot=(), rho_mean=2.3),
             W.periodic_box(64, 40, liquid_rows=13, init_noise=1e-3, isothermal=False, precision="fp32"),
             # wavefront units: several strips, spots on a strip edge, the
             # segment ends of a 45-row domain; an open top; a periodic box
             W.small_parity(precision="fp32").replace(nx=192, nf=45, ns=5, liquid_rows=15, spot_x=(3, 64, 191),
                                                       spot_half_width=2, rho_mean=2.3),
             W.small_parity(precision="fp32").replace(nx=128, nf=37, ns=4, liquid_rows=12, top_mode="outflow",
                                                       bc_mode="noise", spot_x=(), c_w_spot=(), rho_mean=2.3),
             W.periodic_box(128, 30, liquid_rows=10, init_noise=1e-3, isothermal=False, precision="fp32")]
    for cfg in cases:
        o = O.OracleRun(cfg)
        o.step(60)
        g = multi(lbm.Run(cfg))
        g.step(60)
        g.sync()
        e = field_errors(g, o)
        assert e["rho"] < 1e-4 and e["T"] < 1e-5, (cfg, e)


def test_fresh_batches_take_odd_steps_at_once():
    """A new batch whose first call is a single step fills its run
    descriptors and launches at once (the descriptors must land before the
    kernels read them); repeated with fresh batches of several sizes, the
    runs match the same runs stepped alone with the multi variants."""
    cfgs = [c.replace(nf=96, liquid_rows=32) for c in W.sweep(6, seed=21)]
    runs = [lbm.Run(c) for c in cfgs]
    ref = [multi(lbm.Run(c)) for c in cfgs]
    total = 0
    for k in (1, 3, 1, 2, 5):
        b = lbm.Batch(runs[: 2 + (total % 5)])
        b.step(k)
        b.sync()
        b.close()
        total += 1
    for r, q in zip(runs, ref):
        q.step(r.step_count)
        a, c = r.fields(("rho", "T")), q.fields(("rho", "T"))
        assert np.array_equal(a["rho"], c["rho"]) and np.array_equal(a["T"], c["T"])


def test_batch_of_more_runs_than_the_wavefront_lookup_table():
    """More than 256 wavefront-capable runs in one batch: the multi-run
    wavefront flow then takes each run's units in turn (no shared-memory
    prefix tables); the per-run unit numbering is the same, so members agree
    bitwise with the same runs stepped alone with the multi-run kernels."""
    base = W.small_parity(precision="fp32").replace(nx=128, ns=4, spot_x=(3, 64, 127), rho_mean=2.3)
    cfgs = [base.replace(nf=20 + (i % 13), liquid_rows=7 + (i % 5), seed=100 + i) for i in range(260)]
    runs = [multi(lbm.Run(c)) for c in cfgs]
    batch = lbm.Batch(runs)
    batch.step(6)
    batch.sync()
    for i in (0, 1, 137, 255, 256, 259):
        r = multi(lbm.Run(cfgs[i]))
        r.step(6)
        want = r.fields(("rho", "T", "f"))
        got = runs[i].fields(("rho", "T", "f"))
        for k in want:
            assert np.array_equal(got[k], want[k]), (i, k)
        r.close()
    batch.close()
    for r in runs:
        r.close()
