"""ctypes binding of the C ABI in ``include/lbm.h`` (liblbm_gb300.so).

Argument marshalling only: every step of the method runs in the CUDA
kernels of the library.  There is no CPU fallback: if the library cannot be
loaded, :func:`load` raises.

Low-level names mirror the C functions (``lbm_create``, ``lbm_step``,
``lbm_fields``, ``lbm_wall_heat_flux`` ...); :class:`Run` wraps one handle
for a :class:`~paper_1911_10747_gb300.workloads.RunConfig`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm_gb300.so")

LBM_OK, LBM_E_INVAL, LBM_E_NOMEM, LBM_E_CUDA, LBM_E_NUMERIC, LBM_E_TIMEOUT, LBM_E_STATE = range(7)
LBM_TOP_WALL, LBM_TOP_OUTFLOW = 0, 1
LBM_BC_SPOTS, LBM_BC_NOISE, LBM_BC_SINE = 0, 1, 2
LBM_FP64, LBM_FP32, LBM_FP16, LBM_FP32_DFSRC, LBM_FP64_FMA = 0, 1, 2, 3, 4
LBM_PERIODIC_Y, LBM_ISOTHERMAL, LBM_FROZEN_FLOW = 1, 2, 4
LBM_FIELD_RHO, LBM_FIELD_UX, LBM_FIELD_UY, LBM_FIELD_T, LBM_FIELD_F = 1, 2, 4, 8, 16

#: every entry point declared in include/lbm.h
EXPORTS = ("lbm_create", "lbm_destroy", "lbm_step", "lbm_sync", "lbm_step_count", "lbm_fields",
           "lbm_set_state", "lbm_set_state_f32", "lbm_get_state", "lbm_wall_heat_flux", "lbm_vapour_fraction", "lbm_mass", "lbm_series",
           "lbm_set_timing", "lbm_kernel_times", "lbm_kernels_per_step", "lbm_variants",
           "lbm_variant_name", "lbm_select_variants", "lbm_autotune", "lbm_diagnostics_static",
           "lbm_batch_create", "lbm_batch_step", "lbm_batch_sync", "lbm_batch_destroy",
           "lbm_batch_last_error", "lbm_batch_query", "lbm_device_bytes", "lbm_server_create", "lbm_server_submit",
           "lbm_server_tick", "lbm_server_poll", "lbm_server_status", "lbm_server_result", "lbm_server_counts",
           "lbm_server_destroy", "lbm_server_last_error", "lbm_peak_fma",
           "lbm_last_error",
           "lbm_status_string")


class lbm_domain_t(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny_fluid", C.c_int32), ("liquid_rows", C.c_int32),
                ("top_mode", C.c_int32), ("flags", C.c_int32), ("pad0", C.c_int32),
                ("g", C.c_double), ("nu_L", C.c_double), ("nu_V", C.c_double), ("c_v", C.c_double),
                ("cv_chi", C.c_double), ("s", C.c_double * 9), ("varpi", C.c_double),
                ("sign_eps", C.c_double), ("init_noise", C.c_double), ("rho_mean", C.c_double),
                ("seed", C.c_uint64)]


class lbm_heater_t(C.Structure):
    _fields_ = [("ny_solid", C.c_int32), ("pad0", C.c_int32), ("lambda_s", C.c_double),
                ("rho_c_s", C.c_double)]


class lbm_eos_t(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("omega", C.c_double),
                ("G", C.c_double), ("T_sat_over_Tc", C.c_double), ("rho_L", C.c_double),
                ("rho_V", C.c_double)]


class lbm_bc_t(C.Structure):
    _fields_ = [("mode", C.c_int32), ("n_spots", C.c_int32), ("T_b_over_Tc", C.c_double),
                ("noise_amp", C.c_double), ("sine_amp_over_Tc", C.c_double),
                ("sine_wavelength", C.c_double), ("sine_t0", C.c_int64), ("sine_t1", C.c_int64),
                ("spot_x", C.c_int32 * 8), ("spot_half_width", C.c_int32), ("pad0", C.c_int32),
                ("c_w_base", C.c_double), ("c_w_spot", C.c_double * 8), ("c_w_top", C.c_double)]


#: lbm_opts_t.dev_alloc / dev_free
DEV_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbm_opts_t(C.Structure):
    _fields_ = [("precision", C.c_int32), ("use_graphs", C.c_int32), ("stream", C.c_void_p),
                ("rho_shift", C.c_double), ("series_capacity", C.c_int32), ("device", C.c_int32),
                ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN), ("alloc_ctx", C.c_void_p),
                ("bounds_check", C.c_int32), ("pad1", C.c_int32)]


def torch_allocator(device: int = 0):
    """(dev_alloc, dev_free) callbacks that take the run's device memory from
    PyTorch's caching allocator on `device` (keep them referenced while the
    run lives: lbm.Run does)."""
    import torch

    def alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device)
        except RuntimeError:
            return None  # -> LBM_E_NOMEM

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return DEV_ALLOC_FN(alloc), DEV_FREE_FN(free)


_lib = None
_D = C.POINTER(C.c_double)


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {_status_name(code)}: {msg}")
        self.code = code


def _status_name(code):
    names = {0: "LBM_OK", 1: "LBM_E_INVAL", 2: "LBM_E_NOMEM", 3: "LBM_E_CUDA", 4: "LBM_E_NUMERIC",
             5: "LBM_E_TIMEOUT", 6: "LBM_E_STATE"}
    return names.get(code, str(code))


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_1911_10747_gb300.build.build() "
                          "(the CUDA library is required; there is no CPU path)")
    L = C.CDLL(path)
    L.lbm_create.argtypes = [C.POINTER(lbm_domain_t), C.POINTER(lbm_heater_t), C.POINTER(lbm_eos_t),
                             C.POINTER(lbm_bc_t), C.POINTER(lbm_opts_t), C.POINTER(C.c_void_p)]
    L.lbm_destroy.argtypes = [C.c_void_p]
    L.lbm_step.argtypes = [C.c_void_p, C.c_int64]
    L.lbm_sync.argtypes = [C.c_void_p]
    L.lbm_step_count.argtypes = [C.c_void_p]
    L.lbm_step_count.restype = C.c_int64
    L.lbm_fields.argtypes = [C.c_void_p, C.c_uint, C.POINTER(C.c_void_p), C.c_int]
    L.lbm_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int]
    L.lbm_set_state_f32.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int]
    L.lbm_get_state.argtypes = [C.c_void_p, _D, _D, C.POINTER(C.c_int64), C.c_int]
    L.lbm_wall_heat_flux.argtypes = [C.c_void_p, _D, _D]
    L.lbm_vapour_fraction.argtypes = [C.c_void_p, _D]
    L.lbm_mass.argtypes = [C.c_void_p, _D]
    L.lbm_series.argtypes = [C.c_void_p, C.c_int64, C.c_int64, _D]
    L.lbm_set_timing.argtypes = [C.c_void_p, C.c_int]
    L.lbm_kernel_times.argtypes = [C.c_void_p, _D, C.POINTER(C.c_int64)]
    L.lbm_kernels_per_step.argtypes = [C.c_void_p]
    L.lbm_variants.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lbm_variant_name.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.lbm_variant_name.restype = C.c_char_p
    L.lbm_select_variants.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.lbm_autotune.argtypes = [C.c_void_p, C.c_int, _D]
    L.lbm_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]
    L.lbm_batch_step.argtypes = [C.c_void_p, C.c_int64]
    L.lbm_batch_sync.argtypes = [C.c_void_p]
    L.lbm_batch_query.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.lbm_batch_destroy.argtypes = [C.c_void_p]
    L.lbm_batch_last_error.argtypes = [C.c_void_p]
    L.lbm_batch_last_error.restype = C.c_char_p
    L.lbm_device_bytes.argtypes = [C.POINTER(lbm_domain_t), C.POINTER(lbm_heater_t), C.POINTER(lbm_opts_t),
                                   C.POINTER(C.c_uint64)]
    L.lbm_server_create.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]
    L.lbm_server_submit.argtypes = [C.c_void_p, C.POINTER(lbm_domain_t), C.POINTER(lbm_heater_t),
                                    C.POINTER(lbm_eos_t), C.POINTER(lbm_bc_t), C.POINTER(lbm_opts_t),
                                    C.c_int64, C.c_int32, C.POINTER(C.c_int64)]
    L.lbm_server_tick.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.lbm_server_poll.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.lbm_server_status.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), _D]
    L.lbm_server_result.argtypes = [C.c_void_p, C.c_int64, _D, _D, _D]
    L.lbm_server_counts.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_uint64)]
    L.lbm_server_destroy.argtypes = [C.c_void_p]
    L.lbm_server_last_error.argtypes = [C.c_void_p]
    L.lbm_server_last_error.restype = C.c_char_p
    L.lbm_diagnostics_static.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                         C.c_void_p]
    L.lbm_peak_fma.argtypes = [C.c_int32, C.c_int32, C.c_int32, _D]
    L.lbm_last_error.argtypes = [C.c_void_p]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_status_string.argtypes = [C.c_int]
    L.lbm_status_string.restype = C.c_char_p
    _lib = L
    return L


def _check(rc: int, h, where: str):
    if rc != LBM_OK:
        msg = load().lbm_last_error(h)
        raise LbmError(rc, where, msg.decode() if msg else "")


def structs_from_config(cfg, stream=None, use_graphs=True, series_capacity=0, device=0, allocator=None,
                        bounds_check=False):
    """Fill the five ABI structs from a RunConfig.  allocator: None
    (cudaMalloc) or a (dev_alloc, dev_free) pair of ctypes callbacks."""
    d = lbm_domain_t()
    d.nx, d.ny_fluid, d.liquid_rows = cfg.nx, cfg.nf, cfg.liquid_rows
    d.top_mode = {"wall": LBM_TOP_WALL, "outflow": LBM_TOP_OUTFLOW}[cfg.top_mode]
    d.flags = ((LBM_PERIODIC_Y if cfg.periodic_y else 0) | (LBM_ISOTHERMAL if cfg.isothermal else 0)
               | (LBM_FROZEN_FLOW if cfg.frozen_flow else 0))
    d.g, d.nu_L, d.nu_V, d.c_v, d.cv_chi = cfg.g, cfg.nu_L, cfg.nu_V, cfg.c_v, cfg.cv_chi
    for k in range(9):
        d.s[k] = cfg.s[k]
    d.varpi, d.sign_eps, d.init_noise, d.rho_mean = cfg.varpi, cfg.sign_eps, cfg.init_noise, cfg.rho_mean
    d.seed = cfg.seed
    ht = lbm_heater_t(ny_solid=cfg.ns, lambda_s=cfg.lambda_s, rho_c_s=cfg.rho_c_s)
    eo = lbm_eos_t(a=cfg.a, b=cfg.b, R=cfg.R, omega=cfg.omega, G=cfg.G, T_sat_over_Tc=cfg.T_sat_over_Tc,
                   rho_L=cfg.rho_L, rho_V=cfg.rho_V)
    bc = lbm_bc_t()
    bc.mode = {"spots": LBM_BC_SPOTS, "noise": LBM_BC_NOISE, "sine": LBM_BC_SINE}[cfg.bc_mode]
    if len(cfg.spot_x) > 8 or len(cfg.c_w_spot) < len(cfg.spot_x):
        raise ValueError("at most 8 spots, each with a c_w value")
    bc.n_spots = len(cfg.spot_x)
    for k, x in enumerate(cfg.spot_x):
        bc.spot_x[k] = int(x)
        bc.c_w_spot[k] = float(cfg.c_w_spot[k])
    bc.T_b_over_Tc, bc.noise_amp = cfg.T_b_over_Tc, cfg.bc_noise
    bc.sine_amp_over_Tc, bc.sine_wavelength = cfg.sine_amp_over_Tc, cfg.sine_wavelength
    bc.sine_t0, bc.sine_t1 = cfg.sine_t0, cfg.sine_t1
    bc.spot_half_width, bc.c_w_base, bc.c_w_top = cfg.spot_half_width, cfg.c_w_base, cfg.c_w_top
    op = lbm_opts_t()
    op.precision = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP16, "fp32_dfsrc": LBM_FP32_DFSRC,
                    "fp64_fma": LBM_FP64_FMA}[cfg.precision]
    op.use_graphs = 1 if use_graphs else 0
    op.stream = stream
    op.rho_shift = cfg.rho_shift
    op.series_capacity = series_capacity
    op.device = device
    if allocator is not None:
        op.dev_alloc, op.dev_free = allocator
    op.bounds_check = 1 if bounds_check else 0
    return d, ht, eo, bc, op


class Run:
    """One boiling run on the GPU (a handle of the C library)."""

    def __init__(self, cfg, stream=None, use_graphs=True, series_capacity=0, device=0, allocator=None,
                 bounds_check=False):
        """allocator: None (the library's cudaMalloc), "torch" (PyTorch's
        caching allocator) or a (dev_alloc, dev_free) pair of callbacks;
        bounds_check: step one step at a time and report faults at once."""
        L = load()
        self.cfg = cfg
        if allocator == "torch":
            allocator = torch_allocator(device)
        self._allocator = allocator  # the callbacks must outlive the handle
        self._structs = structs_from_config(cfg, stream, use_graphs, series_capacity, device, allocator,
                                            bounds_check)
        h = C.c_void_p()
        rc = L.lbm_create(*[C.byref(s) for s in self._structs], C.byref(h))
        _check(rc, None, "lbm_create")
        self._h = h
        self.nx, self.nf, self.nt = cfg.nx, cfg.nf, cfg.t_rows

    def close(self):
        if getattr(self, "_h", None):
            load().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def step(self, n: int = 1):
        _check(load().lbm_step(self._h, int(n)), self._h, "lbm_step")
        return self

    def sync(self):
        _check(load().lbm_sync(self._h), self._h, "lbm_sync")

    @property
    def step_count(self) -> int:
        return int(load().lbm_step_count(self._h))

    def fields(self, names=("rho", "ux", "uy", "T")) -> dict:
        """Host float64 copies of the requested fields (rho, ux, uy, T, f)."""
        bits = {"rho": LBM_FIELD_RHO, "ux": LBM_FIELD_UX, "uy": LBM_FIELD_UY, "T": LBM_FIELD_T,
                "f": LBM_FIELD_F}
        shapes = {"rho": (self.nf, self.nx), "ux": (self.nf, self.nx), "uy": (self.nf, self.nx),
                  "T": (self.nt, self.nx), "f": (9, self.nf, self.nx)}
        order = [k for k in ("rho", "ux", "uy", "T", "f") if k in names]
        out = {k: np.empty(shapes[k], dtype=np.float64) for k in order}
        mask = 0
        for k in order:
            mask |= bits[k]
        ptrs = (C.c_void_p * len(order))(*[out[k].ctypes.data for k in order])
        _check(load().lbm_fields(self._h, mask, ptrs, 0), self._h, "lbm_fields")
        return out

    def fields_device(self, ptrs: dict):
        """Export into device float64 buffers: ptrs maps field name -> device pointer."""
        bits = {"rho": LBM_FIELD_RHO, "ux": LBM_FIELD_UX, "uy": LBM_FIELD_UY, "T": LBM_FIELD_T,
                "f": LBM_FIELD_F}
        order = [k for k in ("rho", "ux", "uy", "T", "f") if k in ptrs]
        mask = 0
        for k in order:
            mask |= bits[k]
        arr = (C.c_void_p * len(order))(*[ptrs[k] for k in order])
        _check(load().lbm_fields(self._h, mask, arr, 1), self._h, "lbm_fields")

    def set_state(self, f=None, T=None, step: int = 0, src_is_device: bool = False):
        """Replace post-stream populations / temperature (float64 host arrays or
        device pointers when src_is_device)."""
        if src_is_device or isinstance(f, int) or isinstance(T, int):
            # raw pointers (device memory when src_is_device, else host memory)
            fp, tp = f, T
            keep = None
        else:
            fa = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
            ta = None if T is None else np.ascontiguousarray(T, dtype=np.float64)
            if fa is not None and fa.size != 9 * self.nf * self.nx:
                raise ValueError("f must have 9 * nf * nx values")
            if ta is not None and ta.size != self.nt * self.nx:
                raise ValueError("T must have t_rows * nx values")
            fp = None if fa is None else fa.ctypes.data
            tp = None if ta is None else ta.ctypes.data
            keep = (fa, ta)
        _check(load().lbm_set_state(self._h, fp, tp, int(step), 1 if src_is_device else 0), self._h,
               "lbm_set_state")
        del keep

    def set_state_f32(self, f=None, T=None, step: int = 0, src_is_device: bool = False):
        """lbm_set_state_f32: as set_state with float32 arrays (or raw pointers
        to float32 data)."""
        if src_is_device or isinstance(f, int) or isinstance(T, int):
            fp, tp = f, T
            keep = None
        else:
            fa = None if f is None else np.ascontiguousarray(f, dtype=np.float32)
            ta = None if T is None else np.ascontiguousarray(T, dtype=np.float32)
            if fa is not None and fa.size != 9 * self.nf * self.nx:
                raise ValueError("f must have 9 * nf * nx values")
            if ta is not None and ta.size != self.nt * self.nx:
                raise ValueError("T must have t_rows * nx values")
            fp = None if fa is None else fa.ctypes.data
            tp = None if ta is None else ta.ctypes.data
            keep = (fa, ta)
        _check(load().lbm_set_state_f32(self._h, fp, tp, int(step), 1 if src_is_device else 0), self._h,
               "lbm_set_state_f32")
        del keep

    def get_state(self):
        """Checkpoint (lbm_get_state): (f [9, nf, nx], T [nt, nx], step), float64."""
        f = np.empty((9, self.nf, self.nx))
        T = np.empty((self.nt, self.nx))
        step = C.c_int64()
        _check(load().lbm_get_state(self._h, f.ctypes.data_as(_D), T.ctypes.data_as(_D), C.byref(step), 0),
               self._h, "lbm_get_state")
        return f, T, int(step.value)

    def wall_heat_flux(self, local: bool = False):
        qb = C.c_double()
        qt = np.empty(self.nx, dtype=np.float64) if local else None
        _check(load().lbm_wall_heat_flux(self._h, C.byref(qb), None if qt is None else qt.ctypes.data_as(_D)),
               self._h, "lbm_wall_heat_flux")
        return (qb.value, qt) if local else qb.value

    def vapour_fraction(self) -> float:
        v = C.c_double()
        _check(load().lbm_vapour_fraction(self._h, C.byref(v)), self._h, "lbm_vapour_fraction")
        return v.value

    def mass(self) -> float:
        v = C.c_double()
        _check(load().lbm_mass(self._h, C.byref(v)), self._h, "lbm_mass")
        return v.value

    def series(self, first: int, count: int) -> np.ndarray:
        out = np.empty((count, 4), dtype=np.float64)
        _check(load().lbm_series(self._h, int(first), int(count), out.ctypes.data_as(_D)), self._h,
               "lbm_series")
        return out

    def set_timing(self, enable: bool):
        _check(load().lbm_set_timing(self._h, 1 if enable else 0), self._h, "lbm_set_timing")

    def kernel_times(self):
        ms = (C.c_double * 3)()
        n = C.c_int64()
        _check(load().lbm_kernel_times(self._h, ms, C.byref(n)), self._h, "lbm_kernel_times")
        return list(ms), int(n.value)

    def kernels_per_step(self) -> int:
        return int(load().lbm_kernels_per_step(self._h))

    def variants(self) -> dict:
        """{'flow': [names], 'heat': [names], 'selected': (flow, heat)}"""
        L = load()
        out = {}
        sel = []
        for kind, key in ((0, "flow"), (1, "heat")):
            n, cur = C.c_int(), C.c_int()
            _check(L.lbm_variants(self._h, kind, C.byref(n), C.byref(cur)), self._h, "lbm_variants")
            out[key] = [L.lbm_variant_name(self._h, kind, i).decode() for i in range(n.value)]
            sel.append(cur.value)
        out["selected"] = tuple(sel)
        return out

    def select_variants(self, flow: int, heat: int):
        _check(load().lbm_select_variants(self._h, int(flow), int(heat)), self._h, "lbm_select_variants")

    def autotune(self, iters: int = 5):
        ms = (C.c_double * 2)()
        _check(load().lbm_autotune(self._h, int(iters), ms), self._h, "lbm_autotune")
        return list(ms)


def diagnostics_static(rho_ptr: int, T_ptr: int, cfg, out_ptr: int, stream=None):
    """Allocation-free diagnostics of a state held in float64 device arrays
    (see lbm_diagnostics_static in include/lbm.h); out_ptr receives 4 doubles."""
    flags = LBM_PERIODIC_Y if cfg.periodic_y else 0
    rc = load().lbm_diagnostics_static(rho_ptr, T_ptr, cfg.nx, cfg.nf, cfg.ns, flags, cfg.lambda_s, cfg.cv_chi,
                                       cfg.rho_L, cfg.rho_V, out_ptr, stream)
    _check(rc, None, "lbm_diagnostics_static")


def peak_fma(bits: int, iters: int = 4096, device: int = -1) -> float:
    """Measured FMA throughput (TFLOP/s) in float (bits = 32) or double
    (bits = 64): lbm_peak_fma in include/lbm.h."""
    v = C.c_double()
    rc = load().lbm_peak_fma(device, bits, iters, C.byref(v))
    _check(rc, None, "lbm_peak_fma")
    return v.value


class Batch:
    """Steps several runs together through one concurrent CUDA graph
    (lbm_batch_* in include/lbm.h).  Keeps references to its runs."""

    def __init__(self, runs):
        L = load()
        self.runs = list(runs)
        arr = (C.c_void_p * len(self.runs))(*[r.handle for r in self.runs])
        b = C.c_void_p()
        rc = L.lbm_batch_create(arr, len(self.runs), C.byref(b))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_batch_create", L.lbm_batch_last_error(None).decode())
        self._b = b

    def _check(self, rc, where):
        if rc != LBM_OK:
            raise LbmError(rc, where, load().lbm_batch_last_error(self._b).decode())

    def step(self, n: int = 1):
        self._check(load().lbm_batch_step(self._b, int(n)), "lbm_batch_step")
        return self

    def sync(self):
        self._check(load().lbm_batch_sync(self._b), "lbm_batch_sync")

    def done(self) -> bool:
        """Non-blocking: has all queued work of the batch finished?"""
        d = C.c_int32()
        self._check(load().lbm_batch_query(self._b, C.byref(d)), "lbm_batch_query")
        return bool(d.value)

    def close(self):
        if getattr(self, "_b", None):
            load().lbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_bytes(cfg) -> int:
    d, ht, _, _, op = structs_from_config(cfg)
    out = C.c_uint64()
    _check(load().lbm_device_bytes(C.byref(d), C.byref(ht), C.byref(op), C.byref(out)), None, "lbm_device_bytes")
    return int(out.value)


class Server:
    """Continuous-batching request loop (lbm_server_* in include/lbm.h)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, chunk_steps: int = 200, device: int = 0):
        L = load()
        s = C.c_void_p()
        rc = L.lbm_server_create(int(hbm_budget_bytes), int(max_active), int(chunk_steps), int(device), C.byref(s))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_server_create", L.lbm_last_error(None).decode())
        self._s = s
        self._cfg = {}

    def _check(self, rc, where):
        if rc != LBM_OK:
            raise LbmError(rc, where, load().lbm_server_last_error(self._s).decode())

    def submit(self, cfg, steps: int, keep_fields: bool = False) -> int:
        d, ht, eo, bc, op = structs_from_config(cfg)
        rid = C.c_int64()
        self._check(load().lbm_server_submit(self._s, C.byref(d), C.byref(ht), C.byref(eo), C.byref(bc),
                                             C.byref(op), int(steps), 1 if keep_fields else 0, C.byref(rid)),
                    "lbm_server_submit")
        self._cfg[rid.value] = cfg
        return int(rid.value)

    def tick(self) -> int:
        """Advance by one whole chunk (waits for it); returns requests finished."""
        n = C.c_int32()
        self._check(load().lbm_server_tick(self._s, C.byref(n)), "lbm_server_tick")
        return int(n.value)

    def poll(self) -> int:
        """Non-blocking tick: retire a finished chunk, admit arrivals, launch
        the next chunk; returns requests finished."""
        n = C.c_int32()
        self._check(load().lbm_server_poll(self._s, C.byref(n)), "lbm_server_poll")
        return int(n.value)

    def status(self, rid: int):
        st = C.c_int32()
        t = (C.c_double * 3)()
        self._check(load().lbm_server_status(self._s, int(rid), C.byref(st), t), "lbm_server_status")
        return int(st.value), tuple(t)

    def result(self, rid: int, fields: bool = False):
        cfg = self._cfg[rid]
        diag = np.zeros(4)
        rho = np.empty((cfg.nf, cfg.nx)) if fields else None
        T = np.empty((cfg.t_rows, cfg.nx)) if fields else None
        self._check(load().lbm_server_result(self._s, int(rid), diag.ctypes.data_as(_D),
                                             None if rho is None else rho.ctypes.data_as(_D),
                                             None if T is None else T.ctypes.data_as(_D)), "lbm_server_result")
        return (diag, rho, T) if fields else diag

    def counts(self):
        q, a, b = C.c_int32(), C.c_int32(), C.c_uint64()
        self._check(load().lbm_server_counts(self._s, C.byref(q), C.byref(a), C.byref(b)), "lbm_server_counts")
        return int(q.value), int(a.value), int(b.value)

    def close(self):
        if getattr(self, "_s", None):
            load().lbm_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

