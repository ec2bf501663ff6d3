"""The oracle's optional threaded per-site loops (OpenMP over rows) give
results bit-identical to the serial oracle: each loop iteration writes only
its own sites, the arithmetic and its order per site are unchanged, and the
diagnostics sums stay serial.  The serial oracle remains the parity checker;
the threaded one serves the CPU baseline timing."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1911_10747_gb300 import workloads as W

CASES = {
    "spots": lambda: W.small_parity().replace(nx=40, nf=30, ns=4, liquid_rows=10, spot_x=(3, 20, 37),
                                              spot_half_width=1),
    "noise_outflow": lambda: W.small_parity().replace(nx=33, nf=27, ns=3, liquid_rows=9, top_mode="outflow",
                                                      bc_mode="noise", spot_x=(), c_w_spot=()),
    "model_a": lambda: W.small_parity().replace(nx=32, nf=24, ns=0, liquid_rows=8, bc_mode="sine", spot_x=(),
                                                c_w_spot=(), sine_t0=2, sine_t1=20, sine_wavelength=16.0),
    "periodic": lambda: W.periodic_box(36, 30, liquid_rows=10, init_noise=1e-3, isothermal=False),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_threaded_oracle_is_bit_identical_to_the_serial_oracle(case):
    cfg = CASES[case]()
    runs = {}
    try:
        for nthreads in (1, 4):
            O.set_threads(nthreads)
            o = O.OracleRun(cfg)
            o.step(25)
            runs[nthreads] = ({"f": o.f, "T": o.T, "rho": o.rho, "ux": o.ux, "uy": o.uy, "q_top": o.q_top},
                              o.diagnostics())
            assert o.err == 0
    finally:
        O.set_threads(1)
    (f1, d1), (f4, d4) = runs[1], runs[4]
    for k in f1:
        assert np.array_equal(f1[k], f4[k]), k
    for k in d1:
        assert np.array_equal(np.asarray(d1[k]), np.asarray(d4[k])), k


def test_thread_count_round_trips_and_defaults_to_serial():
    assert O.threads() == 1
    O.set_threads(3)
    try:
        assert O.threads() == 3
    finally:
        O.set_threads(1)
    assert O.threads() == 1
