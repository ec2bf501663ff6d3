"""GB300-native hot path of the hybrid pseudopotential phase-change lattice
Boltzmann method with conjugate heat transfer (arXiv:1911.10747).

The compute path lives in the CUDA library ``csrc/`` (C ABI in
``include/lbm.h``); :mod:`.lbm` is its ctypes binding and :mod:`.workloads`
holds the run configurations.  Importing the package loads nothing native.

Typical use (one GB300)::

    from paper_1911_10747_gb300 import build, lbm, workloads as W
    build.build()                                # in-tree liblbm_gb300.so for sm_103a
    run = lbm.Run(W.paper_scale(0.1, "spots", precision="fp32"), series_capacity=20000)
    run.autotune(20)                             # launch shapes for this domain and GPU
    run.step(20000)                              # asynchronous, replayed CUDA graphs
    q_bottom, q_top = run.wall_heat_flux(local=True)   # Eq. 36 / 39 and the local flux
    fields = run.fields(("rho", "ux", "uy", "T"))      # float64 numpy arrays
    history = run.series(0, 20000)               # per step: fluxes, vapour fraction, mass

Many independent runs step together with :class:`.lbm.Batch` (one
concurrent graph); :class:`.lbm.Server` admits runs as they arrive under an
HBM budget (continuous batching).  Model A is ``ns=0``; the bottom
condition is ``bc_mode`` = ``"spots"``, ``"noise"`` or ``"sine"``;
``precision`` = ``"fp64"``, ``"fp64_fma"``, ``"fp32"``, ``"fp32_dfsrc"`` or ``"fp16"`` (storage).
"""
__all__ = ["lbm", "workloads"]
