"""Helpers shared by the GPU parity tests: run the same configuration on the
CUDA library and on the oracle, and compare fields."""
import numpy as np

from oracle import oracle as O
from paper_1911_10747_gb300 import lbm


def run_both(cfg, steps, use_graphs=True):
    g = lbm.Run(cfg, use_graphs=use_graphs)
    g.step(steps)
    g.sync()
    o = O.OracleRun(cfg)
    o.step(steps)
    return g, o


def rel_err(a, b, scale=None):
    a, b = np.asarray(a), np.asarray(b)
    if scale is None:
        scale = np.maximum(np.abs(b), 1e-300)
    return float(np.max(np.abs(a - b) / scale)) if a.size else 0.0


def field_errors(g, o):
    """Max relative error per field: rho and T pointwise relative, u relative
    to max |u| (it passes through zero), f relative to max |f| of its plane."""
    fg = g.fields(("rho", "ux", "uy", "T", "f"))
    umax = max(np.abs(o.ux).max(), np.abs(o.uy).max(), 1e-300)
    fo = o.f
    fscale = np.abs(fo).max(axis=(1, 2), keepdims=True)
    return {
        "rho": rel_err(fg["rho"], o.rho),
        "ux": rel_err(fg["ux"], o.ux, umax),
        "uy": rel_err(fg["uy"], o.uy, umax),
        "T": rel_err(fg["T"], o.T),
        "f": rel_err(fg["f"], fo, fscale),
    }


def select_multi(run):
    """Select the multi-run kernels as the run's own launch shapes: the
    kernels a batch steps it with (FP32 and FP16 storage; the wavefront flow
    variant takes runs whose width is a multiple of 64, at least 128, and
    runs the tiles otherwise, as a batch does).  Other precisions keep
    theirs."""
    v = run.variants()
    for name in ("flowwavemulti_w4_b4", "flowmulti_32x8x2"):
        if name in v["flow"]:
            run.select_variants(v["flow"].index(name), v["heat"].index("heatmulti_64x12x4"))
            break
    return run

