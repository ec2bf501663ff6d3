"""GPU path (C ABI) against the FP64 oracle on the same seeded inputs.

FP64 path: every field within 1e-12 relative per site (u relative to its
maximum) after the steps run, and the per-step diagnostics series within
1e-12.  The sizes span several tiles of both kernels and ragged tails."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

from gpu_util import field_errors, rel_err, run_both

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1911_10747_gb300 import build
    build.build()
    lbm.load()


def check_fp64(g, o, steps):
    errs = field_errors(g, o)
    assert all(v <= TOL64 for v in errs.values()), errs
    ser = g.series(0, steps)
    d = o.diagnostics()
    last = ser[-1]
    assert last[0] == pytest.approx(d["q_bottom"], rel=TOL64, abs=1e-15)
    assert last[1] == pytest.approx(d["q_top"], rel=TOL64, abs=1e-15)
    assert last[2] == pytest.approx(d["vapour_fraction"], abs=1e-15)
    assert last[3] == pytest.approx(d["mass"], rel=TOL64)
    return errs


def test_fp64_parity_small_boiling_case_200_steps():
    """64 x 96 fluid over 8 heater rows, three nucleate spots, 200 steps."""
    cfg = W.small_parity().replace(rho_mean=2.42)
    g, o = run_both(cfg, 200)
    errs = check_fp64(g, o, 200)
    print("fp64 200-step errors", errs)
    # the flow really moved and the heater really heated
    assert np.abs(o.uy).max() > 1e-4
    assert o.diagnostics()["q_bottom"] != 0.0


def test_fp64_series_matches_every_step():
    cfg = W.small_parity().replace(rho_mean=2.42)
    g = lbm.Run(cfg)
    o = O.OracleRun(cfg)
    ser = []
    for _ in range(30):
        o.step(1)
        d = o.diagnostics()
        ser.append([d["q_bottom"], d["q_top"], d["vapour_fraction"], d["mass"]])
    g.step(30)
    got = g.series(0, 30)
    np.testing.assert_allclose(got, np.array(ser), rtol=TOL64, atol=1e-15)


def test_fp64_parity_computed_mean_density():
    """rho_mean left to each side (its own reduction of the initial density)."""
    cfg = W.small_parity()
    g, o = run_both(cfg, 50)
    check_fp64(g, o, 50)


@pytest.mark.parametrize("kw", [
    dict(nx=37, nf=45, ns=5, liquid_rows=15, bc_mode="noise", spot_x=(), c_w_spot=()),
    dict(nx=70, nf=33, ns=3, liquid_rows=11, bc_mode="spots", spot_x=(3, 40, 69), spot_half_width=2,
         c_w_spot=(-0.9, -0.8, -0.7), top_mode="outflow"),
    dict(nx=33, nf=40, ns=9, liquid_rows=12, bc_mode="sine", sine_t0=3, sine_t1=40, sine_wavelength=33.0,
         spot_x=(), c_w_spot=()),
    # model A (Fig. 1a): no heater, T_b on the wall row
    dict(ns=0),
    dict(nx=45, nf=40, ns=0, liquid_rows=13, bc_mode="noise", spot_x=(), c_w_spot=(), T_b_over_Tc=1.0),
])
def test_fp64_parity_ragged_domains_and_bc_modes(kw):
    cfg = W.small_parity().replace(rho_mean=2.3, **kw)
    g, o = run_both(cfg, 60)
    check_fp64(g, o, 60)


def test_fp64_parity_periodic_box_and_test_modes():
    cfg = W.periodic_box(24, 40, liquid_rows=20, init_noise=1e-3)
    g, o = run_both(cfg, 80)
    errs = field_errors(g, o)
    assert all(v <= TOL64 for v in errs.values()), errs
    cfg = W.periodic_box(16, 8, liquid_rows=8, isothermal=False, frozen_flow=True, init_noise=1e-3)
    g, o = run_both(cfg, 20)
    errs = field_errors(g, o)
    assert all(v <= TOL64 for v in errs.values()), errs


def test_fp64_frozen_flow_conduction_mode():
    cfg = W.small_parity().replace(frozen_flow=True, rho_mean=2.42)
    g, o = run_both(cfg, 40)
    check_fp64(g, o, 40)


def test_graph_replay_is_bitwise_identical_to_plain_launches():
    cfg = W.small_parity().replace(bc_mode="noise", spot_x=(), c_w_spot=())
    a = lbm.Run(cfg, use_graphs=True).step(21)
    b = lbm.Run(cfg, use_graphs=False).step(21)
    fa, fb = a.fields(("rho", "ux", "uy", "T", "f")), b.fields(("rho", "ux", "uy", "T", "f"))
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.array_equal(a.series(0, 21), b.series(0, 21))


def test_set_state_round_trip_and_restart_is_exact():
    cfg = W.small_parity().replace(bc_mode="noise", spot_x=(), c_w_spot=(), rho_mean=2.42)
    a = lbm.Run(cfg).step(10)
    st = a.fields(("f", "T"))
    a.step(10)
    b = lbm.Run(cfg)
    b.set_state(st["f"], st["T"], step=10)
    back = b.fields(("f", "T"))
    assert np.array_equal(back["f"], st["f"]) and np.array_equal(back["T"], st["T"])
    b.step(10)
    fa, fb = a.fields(("rho", "T", "f")), b.fields(("rho", "T", "f"))
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("pinned", [False, True])
def test_float32_state_import_equals_the_same_values_as_float64(precision, pinned):
    """lbm_set_state_f32 widens its float32 arrays before converting them to
    the run's storage: the same values given as float64 to lbm_set_state give
    the same state and the same next steps, bit for bit, from pageable and
    from page-locked host memory."""
    torch = pytest.importorskip("torch")
    cfg = W.small_parity(precision=precision).replace(bc_mode="noise", spot_x=(), c_w_spot=(), rho_mean=2.42)
    a = lbm.Run(cfg).step(7)
    st = a.fields(("f", "T"))
    f32, T32 = st["f"].astype(np.float32), st["T"].astype(np.float32)
    b, c = lbm.Run(cfg), lbm.Run(cfg)
    b.set_state(f32.astype(np.float64), T32.astype(np.float64), step=7)
    if pinned:
        hf = torch.from_numpy(f32.reshape(-1)).pin_memory()
        hT = torch.from_numpy(T32.reshape(-1)).pin_memory()
        c.set_state_f32(hf.data_ptr(), hT.data_ptr(), step=7)
    else:
        c.set_state_f32(f32, T32, step=7)
    for r in (b, c):
        r.step(5)
    fb, fc = b.fields(("rho", "T", "f")), c.fields(("rho", "T", "f"))
    for k in fb:
        assert np.array_equal(fb[k], fc[k]), k
    assert np.array_equal(b.series(7, 5), c.series(7, 5))


def test_get_state_checkpoint_restarts_bit_for_bit():
    """lbm_get_state returns what lbm_set_state takes back: a run restarted
    from the checkpoint (populations, temperature, step counter that keys
    the noisy bottom) continues exactly as the original."""
    cfg = W.small_parity().replace(bc_mode="noise", spot_x=(), c_w_spot=(), rho_mean=2.42)
    a = lbm.Run(cfg).step(13)
    f, T, step = a.get_state()
    assert step == 13 and f.shape == (9, cfg.nf, cfg.nx) and T.shape == (cfg.t_rows, cfg.nx)
    st = a.fields(("f", "T"))
    assert np.array_equal(st["f"], f) and np.array_equal(st["T"], T)
    a.step(11)
    b = lbm.Run(cfg)
    b.set_state(f, T, step=step)
    b.step(11)
    fa, fb = a.fields(("rho", "T", "f")), b.fields(("rho", "T", "f"))
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_full_size_domain_fp64_against_oracle():
    """The 2048 x 2048 + 64 domain of the throughput run, two steps, FP64."""
    cfg = W.large(precision="fp64").replace(rho_mean=2.41)
    g, o = run_both(cfg, 2)
    errs = field_errors(g, o)
    assert all(v <= TOL64 for v in errs.values()), errs


def test_numerical_fault_is_reported():
    """A non-finite population (host input) makes the density and the EOS
    radicand non-finite: the kernels latch it in the error word and the next
    synchronising call returns LBM_E_NUMERIC; the context stays usable."""
    cfg = W.small_parity()
    g = lbm.Run(cfg)
    f = g.fields(("f",))["f"]
    f[:, 10, 10] = np.nan
    g.set_state(f, None, step=0)
    g.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        g.sync()
    assert ei.value.code == lbm.LBM_E_NUMERIC
    # a fresh run on the same device still works
    h = lbm.Run(cfg).step(2)
    h.sync()


def test_fp64_parity_sessile_drop_from_set_state():
    """The wettability-calibration setting: an isothermal, gravity-free drop
    on the bottom wall, loaded through lbm_set_state on both sides."""
    from paper_1911_10747_gb300 import calibration as K
    cfg = K.drop_config(-1.1, nx=72, nf=40, precision="fp64")
    f, T = K.drop_state(cfg, 14.0)
    g = lbm.Run(cfg)
    g.set_state(f, T, step=0)
    o = O.OracleRun(cfg)
    o.set_f(f)
    o.set_T(T)
    g.step(120)
    g.sync()
    o.step(120)
    errs = field_errors(g, o)
    assert all(v <= TOL64 for v in errs.values()), errs


@pytest.mark.parametrize("variant", ["flowtma_64x4x2_b3", "flowwave_w4_b4_u8"])
def test_staged_copy_wait_that_runs_out_is_reported_and_the_context_survives(monkeypatch, variant):
    """The flow kernels that stage rows or tiles by tensor copies bound their
    waits on the copy barriers.  The test hook makes each stage expect 16
    bytes more than its copies deliver, so every wait runs out (after
    100 ms): the step must report LBM_E_TIMEOUT, and a new run on the same
    context must work."""
    cfg = W.small_parity(precision="fp32").replace(nx=128, nf=40, ns=4, liquid_rows=12, rho_mean=2.3,
                                                   spot_x=(), c_w_spot=())
    monkeypatch.setenv("LBM_TEST_TX_PAD", "16")
    g = lbm.Run(cfg)
    monkeypatch.delenv("LBM_TEST_TX_PAD")
    names = g.variants()["flow"]
    g.select_variants(names.index(variant), 0)
    g.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        g.sync()
    assert "LBM_E_TIMEOUT" in str(ei.value)
    del g
    ok = lbm.Run(cfg)
    ok.select_variants(names.index(variant), 0)
    ok.step(3)
    ok.sync()
    assert ok.step_count == 3


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_set_state_from_page_locked_memory_equals_the_staged_path(precision):
    """lbm_set_state reads page-locked host arrays directly (import kernel
    over the host link) and stages pageable ones: both give the same state."""
    import torch
    cfg = W.small_parity(precision=precision).replace(bc_mode="noise", spot_x=(), c_w_spot=(), rho_mean=2.42)
    a = lbm.Run(cfg).step(7)
    st = a.fields(("f", "T"))
    pf = torch.from_numpy(st["f"].copy()).pin_memory()
    pT = torch.from_numpy(st["T"].copy()).pin_memory()
    b, c = lbm.Run(cfg), lbm.Run(cfg)
    b.set_state(pf.data_ptr(), pT.data_ptr(), step=7)
    c.set_state(st["f"], st["T"], step=7)
    fb, fc = b.fields(("f", "T")), c.fields(("f", "T"))
    for k in fb:
        assert np.array_equal(fb[k], fc[k]), k
    b.step(5)
    c.step(5)
    assert np.array_equal(b.fields(("rho",))["rho"], c.fields(("rho",))["rho"])


@pytest.mark.parametrize("kw", [
    dict(nx=1, nf=12, ns=3, liquid_rows=4, spot_x=(), c_w_spot=()),              # one column
    dict(nx=5, nf=2, ns=3, liquid_rows=1, spot_x=(), c_w_spot=()),               # two fluid rows
    dict(nx=1, nf=3, ns=0, liquid_rows=1, spot_x=(), c_w_spot=(), bc_mode="noise"),  # model A, one column
])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_degenerate_domains(kw, precision):
    """Smallest domains the ABI accepts: every neighbour wraps onto the site
    itself or its column, the bottom and top walls touch."""
    cfg = W.small_parity(precision=precision).replace(rho_mean=2.42, **kw)
    g, o = run_both(cfg, 30)
    errs = field_errors(g, o)
    tol = TOL64 if precision == "fp64" else 1e-4
    assert all(v <= tol for v in errs.values()), errs


@pytest.mark.parametrize("bc", ["spots", "noise"])
def test_paper_scale_domain_against_oracle(bc):
    """The 400 x 600 + 30 paper-scale domain, 20 steps: FP64 to 1e-12 per
    site, FP32 within its rounding bound."""
    cfg = W.paper_scale(0.1, bc, precision="fp64").replace(rho_mean=2.42)
    g, o = run_both(cfg, 20)
    errs = field_errors(g, o)
    assert all(v <= TOL64 for v in errs.values()), errs
    g32 = lbm.Run(cfg.replace(precision="fp32")).step(20)
    g32.sync()
    errs32 = field_errors(g32, o)
    assert errs32["rho"] < 1e-5 and errs32["T"] < 1e-6, errs32
