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


def test_fp32_full_size_in_the_benchmarked_launch_configuration():
    """The bench's workload (2048 x 2048 fluid + 64 heater rows, seed 3) as
    the bench runs it: on a stream of its own, autotuned with the bench's
    call, stepped through the captured CUDA graphs; two steps against the
    oracle.  Then every heat variant with the chosen flow variant and every
    flow variant with the chosen heat variant, so that whichever the
    autotuner picks on a given GPU has met the oracle at full size."""
    import torch
    cfg = W.large(precision="fp32", seed=3)
    o = O.OracleRun(cfg)
    o.step(2)
    stream = torch.cuda.Stream()
    g = lbm.Run(cfg, stream=stream.cuda_stream)
    g.autotune(20)
    v = g.variants()
    fv, hv0 = v["selected"]
    g.step(2)
    g.sync()
    errs = field_errors(g, o)
    print("benchmarked pair", v["flow"][fv], v["heat"][hv0], errs)
    assert errs["rho"] < 1e-5 and errs["T"] < 1e-6, errs
    g.close()
    pairs = [(fv, hv) for hv in range(len(v["heat"])) if hv != hv0]
    pairs += [(f, hv0) for f in range(len(v["flow"])) if f != fv]
    for f, hv in pairs:
        g = lbm.Run(cfg, stream=stream.cuda_stream)
        g.select_variants(f, hv)
        g.step(2)
        g.sync()
        errs = field_errors(g, o)
        g.close()
        assert errs["rho"] < 1e-5 and errs["T"] < 1e-6, (v["flow"][f], v["heat"][hv], errs)


def test_fp32_variants_agree_are_deterministic_and_autotune_keeps_state():
    """Every launch-shape variant does the same per-site arithmetic (up to the
    compiler's FMA contraction choices per instantiation): fields agree to
    FP32 rounding, each variant is run-to-run deterministic, and the
    autotuner leaves the run's state untouched."""
    cfg = W.small_parity(precision="fp32").replace(nx=70, nf=45, ns=5, liquid_rows=15, rho_mean=2.3,
                                                   spot_x=(3, 40, 69), spot_half_width=2)
    names = lbm.Run(cfg).variants()

    def run(fv, hv, n=12, tune_after=None):
        r = lbm.Run(cfg)
        r.select_variants(fv, hv)
        if tune_after is None:
            r.step(n)
        else:
            r.step(tune_after)
            r.autotune(2)
            r.select_variants(fv, hv)
            r.step(n - tune_after)
        return r.fields(("rho", "ux", "uy", "T", "f"))

    want = run(0, 0)
    for fv in range(len(names["flow"])):
        for hv in range(len(names["heat"])):
            a, b = run(fv, hv), run(fv, hv)
            for k in want:
                assert np.array_equal(a[k], b[k]), ("nondeterministic", names["flow"][fv], names["heat"][hv], k)
                scale = np.abs(want[k]).max()
                assert np.max(np.abs(a[k] - want[k])) <= 1e-4 * scale, (names["flow"][fv], names["heat"][hv], k)
    tuned = run(1, 1, tune_after=5)
    plain = run(1, 1)
    for k in plain:
        assert np.array_equal(tuned[k], plain[k]), k


def test_fp32_outflow_ragged_top_tile():
    cfg = W.small_parity(precision="fp32").replace(nx=70, nf=33, ns=3, liquid_rows=11, top_mode="outflow",
                                                   rho_mean=2.3, spot_x=(3, 40, 69), spot_half_width=2)
    g, o = run_both(cfg, 60)
    errs = field_errors(g, o)
    print("fp32 outflow errors", errs)
    assert errs["rho"] < 1e-4 and errs["T"] < 1e-5, errs


def test_fp32_model_a_error_report():
    """Model A (no heater) through the FP32 kernels, against the oracle."""
    cfg = W.small_parity(precision="fp32").replace(ns=0, rho_mean=2.42)
    g, o = run_both(cfg, 200)
    errs = field_errors(g, o)
    print("fp32 model A 200-step errors", errs)
    assert errs["rho"] < 1e-3 and errs["T"] < 1e-5, errs
    d = o.diagnostics()
    assert g.wall_heat_flux() == pytest.approx(d["q_bottom"], rel=1e-3)


@pytest.mark.parametrize("tb", [0.96, 1.0])
def test_fp32_long_run_statistics_match_fp64(tb):
    """20,000 steps of the 64 x 96 boiling case: the time averages of the
    heater-bottom flux and the vapour fraction over the second half agree
    between the FP32 path and the FP64 path (which matches the oracle) to
    2 %; the FP32 mass drifts by less than 1e-5."""
    n = 20000
    cfg = W.small_parity().replace(rho_mean=2.42, T_b_over_Tc=tb)
    out = {}
    for prec in ("fp64", "fp32"):
        r = lbm.Run(cfg.replace(precision=prec), series_capacity=n + 8)
        r.step(n)
        r.sync()
        s = r.series(0, n)
        out[prec] = s
    h64, h32 = out["fp64"][n // 2:], out["fp32"][n // 2:]
    for col in (0, 2):
        assert h32[:, col].mean() == pytest.approx(h64[:, col].mean(), rel=0.02)
    m = out["fp32"][:, 3]
    assert abs(m[-1] / m[0] - 1) < 1e-5
    assert np.array_equal(out["fp64"][:, 3], np.full(n, out["fp64"][0, 3])) or \
        np.max(np.abs(out["fp64"][:, 3] / out["fp64"][0, 3] - 1)) < 1e-11


def test_fp16_storage_rounds_without_bias():
    """FP16 population stores round stochastically.  On the film-boiling case
    (Sec. 3.2, c_w = -1.2, to t* = 60) round-to-nearest storage drifted the
    mass by 4.6 % and doubled Nu; unbiased rounding keeps the drift under
    2e-3 and Nu within 20 % of the FP32 path (which is within 0.1 % of
    FP64)."""
    from paper_1911_10747_gb300 import validation as V
    s32 = V.film_boiling(0.06316, precision="fp32", c_w=-1.2)
    s16 = V.film_boiling(0.06316, precision="fp16", c_w=-1.2)
    print("fp16 film", s16["mass_drift"], s16["nu_lbm_surface"], "fp32", s32["nu_lbm_surface"])
    assert abs(s16["mass_drift"]) < 2e-3
    assert s16["nu_lbm_surface"] == pytest.approx(s32["nu_lbm_surface"], rel=0.2)


@pytest.mark.parametrize("kw", [
    dict(nx=192, nf=45, ns=5, liquid_rows=15, spot_x=(3, 100, 191), spot_half_width=2),
    dict(nx=128, nf=37, ns=4, liquid_rows=12, top_mode="outflow", bc_mode="noise", spot_x=(), c_w_spot=()),
])
def test_fp32_bulk_copy_flow_variants_against_the_oracle(kw):
    """The flow kernels that stage tiles with bulk asynchronous copies (nx a
    multiple of 64): several tiles across, the periodic x edges, a ragged top
    tile and both top boundaries, against the oracle."""
    cfg = W.small_parity(precision="fp32").replace(rho_mean=2.3, **kw)
    names = lbm.Run(cfg).variants()["flow"]
    tma = [i for i, n in enumerate(names) if n.startswith("flowtma_")]
    assert tma
    o = O.OracleRun(cfg)
    o.step(60)
    for fv in tma:
        g = lbm.Run(cfg)
        g.select_variants(fv, 0)
        g.step(60)
        g.sync()
        errs = field_errors(g, o)
        assert errs["rho"] < 1e-4 and errs["T"] < 1e-5, (names[fv], errs)


def test_fp32_bulk_copy_flow_in_a_periodic_box():
    """Periodic in y with a box lower than one tile plus its halo rows."""
    cfg = W.periodic_box(64, 6, liquid_rows=3, init_noise=1e-3, precision="fp32")
    names = lbm.Run(cfg).variants()["flow"]
    o = O.OracleRun(cfg)
    o.step(40)
    for fv in [i for i, n in enumerate(names) if n.startswith("flowtma_")]:
        g = lbm.Run(cfg)
        g.select_variants(fv, 0)
        g.step(40)
        g.sync()
        errs = field_errors(g, o)
        assert errs["rho"] < 1e-4, (names[fv], errs)


@pytest.mark.parametrize("kw", [
    dict(nx=150, nf=45, ns=5, liquid_rows=15, spot_x=(3, 80, 149), spot_half_width=2),
    dict(nx=40, nf=33, ns=4, liquid_rows=11, top_mode="outflow", bc_mode="noise", spot_x=(), c_w_spot=()),
    dict(nx=96, nf=40, ns=0, liquid_rows=13, bc_mode="sine", spot_x=(), c_w_spot=()),
    dict(nx=192, nf=45, ns=5, liquid_rows=15, spot_x=(3, 100, 191), spot_half_width=2),
    dict(nx=128, nf=37, ns=4, liquid_rows=12, top_mode="outflow", bc_mode="noise", spot_x=(), c_w_spot=()),
])
def test_fp32_paired_column_and_wavefront_heat_variants_against_the_oracle(kw):
    """The heat kernels that hold two columns per thread as packed pairs (with
    4-byte or whole-row 16-byte staging) and the row-wavefront kernels (one
    warp per column strip): several tiles or strips across with a ragged
    last one, a domain narrower than one tile or strip (columns wrap inside
    it), model A, heater rows, an open top, each bottom mode."""
    cfg = W.small_parity(precision="fp32").replace(rho_mean=2.3, **kw)
    if cfg.bc_mode == "sine":
        cfg = cfg.replace(sine_t0=5, sine_t1=50, sine_wavelength=48.0)
    names = lbm.Run(cfg).variants()["heat"]
    pair = [i for i, n in enumerate(names) if n.startswith(("heatpair_", "heatpair16_", "heatwave_"))]
    assert pair
    o = O.OracleRun(cfg)
    o.step(60)
    for hv in pair:
        g = lbm.Run(cfg)
        g.select_variants(0, hv)
        g.step(60)
        g.sync()
        errs = field_errors(g, o)
        assert errs["rho"] < 1e-4 and errs["T"] < 1e-5, (names[hv], errs)


@pytest.mark.parametrize("nx", [70, 128])
def test_fp16_storage_heat_variants_agree(nx):
    """The heat kernels read float T, rho and u whatever the population
    storage: with FP16 storage every heat variant follows the same run (the
    flow kernel's stochastic rounding is keyed by site and step, so it draws
    the same dither in every run; values that land next to a rounding step
    can still differ by one half ulp).  128 columns: the row-staged kernels
    stage whole rows (nx a multiple of 4)."""
    cfg = W.small_parity(precision="fp16").replace(nx=nx, nf=45, ns=5, liquid_rows=15, rho_mean=2.3,
                                                   spot_x=(3, 40, nx - 1), spot_half_width=2)
    names = lbm.Run(cfg).variants()["heat"]

    def run(hv):
        r = lbm.Run(cfg)
        r.select_variants(0, hv)
        r.step(8)
        return r.fields(("rho", "T"))

    want = run(0)
    for hv in range(1, len(names)):
        got = run(hv)
        for k in want:
            assert np.max(np.abs(got[k] - want[k])) <= 1e-2 * np.abs(want[k]).max(), (names[hv], k)


@pytest.mark.parametrize("ny", [40, 100])
def test_fp32_heat_variants_in_a_periodic_box_with_heat(ny):
    """Doubly periodic box with the energy equation on: rows wrap inside the
    heat tiles (40 rows: fewer than the tallest tile holds; 100 rows: several
    tiles), for every heat variant, against the oracle."""
    cfg = W.periodic_box(64, ny, liquid_rows=ny // 3, init_noise=1e-3, isothermal=False, precision="fp32")
    names = lbm.Run(cfg).variants()["heat"]
    o = O.OracleRun(cfg)
    o.step(40)
    for hv, name in enumerate(names):
        g = lbm.Run(cfg)
        g.select_variants(0, hv)
        g.step(40)
        g.sync()
        errs = field_errors(g, o)
        assert errs["rho"] < 1e-4 and errs["T"] < 1e-5, (name, errs)


@pytest.mark.parametrize("kw", [
    dict(nx=192, nf=45, ns=5, liquid_rows=15, spot_x=(3, 100, 191), spot_half_width=2),
    dict(nx=128, nf=37, ns=4, liquid_rows=12, top_mode="outflow", bc_mode="noise", spot_x=(), c_w_spot=()),
    dict(nx=128, nf=40, ns=0, liquid_rows=13, bc_mode="sine", spot_x=(), c_w_spot=()),
    dict(nx=64, nf=200, ns=3, liquid_rows=60, spot_x=(0, 31, 63), spot_half_width=1),
    dict(nx=256, nf=45, ns=5, liquid_rows=15, spot_x=(0, 127, 200), spot_half_width=2),
    dict(nx=256, nf=37, ns=4, liquid_rows=12, top_mode="outflow", bc_mode="noise", spot_x=(), c_w_spot=()),
])
def test_fp32_wavefront_flow_variants_against_the_oracle(kw):
    """The flow kernels in which each warp sweeps a 64-column strip up a
    segment of rows (nx a multiple of 64): several strips across with the
    periodic x edges, nucleate spots on a strip edge, an open top, model A
    with the sine bottom, and a tall single-strip domain cut into many
    segments, against the oracle; and the wavefront shapes agree."""
    cfg = W.small_parity(precision="fp32").replace(rho_mean=2.3, **kw)
    if cfg.bc_mode == "sine":
        cfg = cfg.replace(sine_t0=5, sine_t1=50, sine_wavelength=48.0)
    names = lbm.Run(cfg).variants()["flow"]
    wave = [i for i, n in enumerate(names) if n.startswith("flowwave_")]
    assert len(wave) >= 2
    o = O.OracleRun(cfg)
    o.step(60)
    got = []
    for fv in wave:
        g = lbm.Run(cfg)
        g.select_variants(fv, 0)
        g.step(60)
        g.sync()
        errs = field_errors(g, o)
        assert errs["rho"] < 1e-4 and errs["T"] < 1e-5, (names[fv], errs)
        assert g.mass() == pytest.approx(o.diagnostics()["mass"], rel=1e-6), names[fv]
        got.append(g.fields(("rho", "f")))
    for other in got[1:]:   # same per-site arithmetic whatever the launch shape
        for k in got[0]:
            assert np.max(np.abs(got[0][k] - other[k])) <= 1e-5 * np.abs(got[0][k]).max(), k


def test_fp32_wavefront_flow_long_and_short_units():
    """A domain wide enough (2048 columns, 32 strips) that the wavefront
    shapes cut it into long units below a band of short ones, with 700 rows
    so that the last long segment is ragged (shapes with 16-row units: 92
    rows below the short band); three steps against the oracle for every
    wavefront shape, and the shapes agree."""
    cfg = W.large(precision="fp32").replace(nf=700, ns=16, liquid_rows=233, rho_mean=2.41)
    names = lbm.Run(cfg).variants()["flow"]
    o = O.OracleRun(cfg)
    o.step(3)
    for fv in [i for i, n in enumerate(names) if n.startswith("flowwave_")]:
        g = lbm.Run(cfg)
        g.select_variants(fv, 0)
        g.step(3)
        g.sync()
        errs = field_errors(g, o)
        g.close()
        assert errs["rho"] < 1e-5 and errs["T"] < 1e-6 and errs["f"] < 1e-5, (names[fv], errs)


@pytest.mark.parametrize("nx,ny", [(128, 6), (128, 70), (256, 40)])
def test_fp32_wavefront_flow_in_a_periodic_box(nx, ny):
    """Periodic in y: the sweep's first and last rows wrap (6 rows: fewer
    than one segment), against the oracle, on one and on several strips."""
    cfg = W.periodic_box(nx, ny, liquid_rows=max(1, ny // 3), init_noise=1e-3, precision="fp32")
    names = lbm.Run(cfg).variants()["flow"]
    o = O.OracleRun(cfg)
    o.step(40)
    for fv in [i for i, n in enumerate(names) if n.startswith("flowwave_")]:
        g = lbm.Run(cfg)
        g.select_variants(fv, 0)
        g.step(40)
        g.sync()
        errs = field_errors(g, o)
        assert errs["rho"] < 1e-4, (names[fv], errs)
