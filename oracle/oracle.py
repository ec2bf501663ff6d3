"""Python handle on the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and nothing here imports the CUDA library.

Also holds the thermodynamic utilities that pin the equation of state:
the Maxwell equal-area construction and the Clausius-Clapeyron latent heat.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 and no FMA contraction, with OpenMP
    for the optional threaded per-site loops (without it if the compiler has
    no OpenMP runtime: the loops then run serially whatever the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp,
                _SRC, "-lm"]
        try:
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Threads for the oracle's per-site loops (1: serial).  Results are
    bit-identical for every count; the diagnostics sums stay serial."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_threads())


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("nf", C.c_int), ("ns", C.c_int), ("liquid_rows", C.c_int),
        ("top_mode", C.c_int), ("flags", C.c_int), ("bc_mode", C.c_int), ("n_spots", C.c_int),
        ("spot_x", C.c_int * 8), ("spot_half_width", C.c_int), ("pad0", C.c_int),
        ("c_w_base", C.c_double), ("c_w_top", C.c_double), ("c_w_spot", C.c_double * 8),
        ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("omega", C.c_double),
        ("G", C.c_double), ("T_sat_over_Tc", C.c_double), ("T_b_over_Tc", C.c_double),
        ("rho_L", C.c_double), ("rho_V", C.c_double), ("rho_mean", C.c_double),
        ("g", C.c_double), ("nu_L", C.c_double), ("nu_V", C.c_double), ("c_v", C.c_double),
        ("cv_chi", C.c_double), ("lambda_s", C.c_double), ("rho_c_s", C.c_double),
        ("s", C.c_double * 9), ("varpi", C.c_double), ("sign_eps", C.c_double),
        ("init_noise", C.c_double), ("bc_noise", C.c_double), ("sine_amp_over_Tc", C.c_double),
        ("sine_wavelength", C.c_double), ("sine_t0", C.c_longlong), ("sine_t1", C.c_longlong),
        ("seed", C.c_ulonglong),
    ]


_lib = None
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Params)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_longlong]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_threads.restype = C.c_int
        for name in ("orc_f", "orc_T", "orc_rho", "orc_ux", "orc_uy", "orc_q_top", "orc_diag"):
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [C.c_void_p]
        L.orc_get_step.restype = C.c_longlong
        L.orc_get_step.argtypes = [C.c_void_p]
        L.orc_set_step.argtypes = [C.c_void_p, C.c_longlong]
        L.orc_err.restype = C.c_uint
        L.orc_err.argtypes = [C.c_void_p]
        L.orc_rho_bar.restype = C.c_double
        L.orc_rho_bar.argtypes = [C.c_void_p]
        L.orc_run_Tc.restype = C.c_double
        L.orc_run_Tc.argtypes = [C.c_void_p]
        L.orc_set_rho_bar.argtypes = [C.c_void_p, C.c_double]
        L.orc_params_size.restype = C.c_int
        L.orc_uniform.restype = C.c_double
        L.orc_uniform.argtypes = [C.c_ulonglong] * 4
        L.orc_Tc.restype = C.c_double
        L.orc_Tc.argtypes = [C.c_double] * 3
        L.orc_kappa.restype = C.c_double
        L.orc_kappa.argtypes = [C.c_double]
        for name in ("orc_pressure", "orc_dpdT"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double] * 7
        L.orc_psi.restype = C.c_double
        L.orc_psi.argtypes = [C.c_double] * 8 + [C.POINTER(C.c_int)]
        L.orc_moments.argtypes = [_D, _D]
        L.orc_inverse_moments.argtypes = [_D, _D]
        L.orc_meq.argtypes = [C.c_double] * 3 + [_D]
        L.orc_source_vec.argtypes = [C.c_double] * 11 + [_D]
        L.orc_collide_site.argtypes = [_D] + [C.c_double] * 6 + [_D, C.c_double, _D]
        L.orc_grad_lap.argtypes = [_D, C.c_int, C.c_int, _D, _D, _D]
        L.orc_splitmix64_next.restype = C.c_ulonglong
        L.orc_splitmix64_next.argtypes = [C.POINTER(C.c_ulonglong)]
        assert L.orc_params_size() == C.sizeof(_Params), "oracle parameter struct mismatch"
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _params(cfg) -> _Params:
    p = _Params()
    # Model A (no heater): row 0 of T is the wall's Dirichlet row
    p.nx, p.nf, p.ns, p.liquid_rows = cfg.nx, cfg.nf, cfg.t_rows - cfg.nf, cfg.liquid_rows
    p.top_mode = {"wall": 0, "outflow": 1}[cfg.top_mode]
    p.flags = ((1 if cfg.periodic_y else 0) | (2 if cfg.isothermal else 0) | (4 if cfg.frozen_flow else 0)
               | (8 if cfg.model_a else 0))
    p.bc_mode = {"spots": 0, "noise": 1, "sine": 2}[cfg.bc_mode]
    if len(cfg.spot_x) > 8 or len(cfg.c_w_spot) < len(cfg.spot_x):
        raise ValueError("at most 8 spots, each with a c_w value")
    p.n_spots = len(cfg.spot_x)
    for k, x in enumerate(cfg.spot_x):
        p.spot_x[k] = int(x)
        p.c_w_spot[k] = float(cfg.c_w_spot[k])
    p.spot_half_width = cfg.spot_half_width
    p.c_w_base, p.c_w_top = cfg.c_w_base, cfg.c_w_top
    for name in ("a", "b", "R", "omega", "G", "T_sat_over_Tc", "T_b_over_Tc", "rho_L", "rho_V",
                 "rho_mean", "g", "nu_L", "nu_V", "c_v", "cv_chi", "lambda_s", "rho_c_s", "varpi",
                 "sign_eps", "init_noise", "bc_noise", "sine_amp_over_Tc", "sine_wavelength"):
        setattr(p, name, float(getattr(cfg, name)))
    for k in range(9):
        p.s[k] = float(cfg.s[k])
    p.sine_t0, p.sine_t1 = int(cfg.sine_t0), int(cfg.sine_t1)
    p.seed = int(cfg.seed)
    return p


class OracleRun:
    """One boiling run advanced by the oracle.  Arrays are returned as copies:
    f[9, nf, nx], T[t_rows, nx] (ns + nf rows; Model A: 1 + nf), rho/ux/uy[nf, nx] (the moments of the last
    step, i.e. rho^n and the force-corrected u^n used by the collision)."""

    def __init__(self, cfg):
        self.cfg = cfg
        self._p = _params(cfg)
        self._h = lib().orc_create(C.byref(self._p))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self.nx, self.nf, self.nt = cfg.nx, cfg.nf, cfg.t_rows

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def _arr(self, name, shape):
        ptr = getattr(lib(), name)(self._h)
        n = int(np.prod(shape))
        return np.ctypeslib.as_array(ptr, shape=(n,)).reshape(shape)

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))
        return self

    @property
    def step_count(self) -> int:
        return int(lib().orc_get_step(self._h))

    @property
    def f(self):
        return self._arr("orc_f", (9, self.nf, self.nx)).copy()

    @property
    def T(self):
        return self._arr("orc_T", (self.nt, self.nx)).copy()

    @property
    def rho(self):
        return self._arr("orc_rho", (self.nf, self.nx)).copy()

    @property
    def ux(self):
        return self._arr("orc_ux", (self.nf, self.nx)).copy()

    @property
    def uy(self):
        return self._arr("orc_uy", (self.nf, self.nx)).copy()

    @property
    def q_top(self):
        return self._arr("orc_q_top", (self.nx,)).copy()

    def diagnostics(self) -> dict:
        d = self._arr("orc_diag", (4,))
        return {"q_bottom": float(d[0]), "q_top": float(d[1]), "vapour_fraction": float(d[2]),
                "mass": float(d[3])}

    @property
    def err(self) -> int:
        return int(lib().orc_err(self._h))

    @property
    def rho_bar(self) -> float:
        return float(lib().orc_rho_bar(self._h))

    @property
    def Tc(self) -> float:
        return float(lib().orc_run_Tc(self._h))

    def set_f(self, f):
        self._arr("orc_f", (9, self.nf, self.nx))[...] = np.asarray(f, dtype=np.float64)

    def set_T(self, T):
        self._arr("orc_T", (self.nt, self.nx))[...] = np.asarray(T, dtype=np.float64)

    def set_rho_bar(self, v: float):
        lib().orc_set_rho_bar(self._h, float(v))


# ---- pointwise functions ----------------------------------------------------

def Tc(a=2.0 / 49.0, b=2.0 / 21.0, R=1.0) -> float:
    return lib().orc_Tc(a, b, R)


def kappa(omega=0.344) -> float:
    return lib().orc_kappa(omega)


def pressure(rho, T, a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344):
    L = lib()
    tc, k = L.orc_Tc(a, b, R), L.orc_kappa(omega)
    return np.vectorize(lambda r, t: L.orc_pressure(r, t, a, b, R, k, tc))(rho, T)


def dpdT(rho, T, a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344):
    L = lib()
    tc, k = L.orc_Tc(a, b, R), L.orc_kappa(omega)
    return np.vectorize(lambda r, t: L.orc_dpdT(r, t, a, b, R, k, tc))(rho, T)


def psi(rho, T, a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344, G=-1.0):
    L = lib()
    tc, k = L.orc_Tc(a, b, R), L.orc_kappa(omega)
    bad = C.c_int(0)
    return L.orc_psi(rho, T, a, b, R, k, tc, G, C.byref(bad)), bool(bad.value)


def uniform(seed, tag, step, idx) -> float:
    return lib().orc_uniform(seed, tag, step, idx)


def splitmix64_sequence(seed: int, n: int):
    st = C.c_ulonglong(seed)
    return [int(lib().orc_splitmix64_next(C.byref(st))) for _ in range(n)]


def moments(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    m = np.zeros(9)
    lib().orc_moments(_dp(f), _dp(m))
    return m


def inverse_moments(m):
    m = np.ascontiguousarray(m, dtype=np.float64)
    f = np.zeros(9)
    lib().orc_inverse_moments(_dp(m), _dp(f))
    return f


def meq(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_meq(rho, ux, uy, _dp(out))
    return out


def source(ux, uy, Fx, Fy, Fmx=0.0, Fmy=0.0, psi_=1.0, varpi=0.0, tau_e=1.25, tau_s=1.25,
           sign_eps=-1.0):
    out = np.zeros(9)
    lib().orc_source_vec(ux, uy, Fx, Fy, Fmx, Fmy, psi_, varpi, tau_e, tau_s, sign_eps, _dp(out))
    return out


def collide_site(f, Fx, Fy, Fmx=0.0, Fmy=0.0, psi_=1.0, varpi=0.0, s=None, sign_eps=-1.0):
    f = np.ascontiguousarray(f, dtype=np.float64)
    s = np.ascontiguousarray(s if s is not None else [1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0],
                             dtype=np.float64)
    out = np.zeros(9)
    lib().orc_collide_site(_dp(f), Fx, Fy, Fmx, Fmy, psi_, varpi, _dp(s), sign_eps, _dp(out))
    return out


def grad_lap(phi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape
    gx, gy, lap = np.zeros_like(phi), np.zeros_like(phi), np.zeros_like(phi)
    lib().orc_grad_lap(_dp(phi), nx, ny, _dp(gx), _dp(gy), _dp(lap))
    return gx, gy, lap


# ---- thermodynamics ---------------------------------------------------------

def maxwell(T_over_Tc=0.86, a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344):
    """Coexistence densities (rho_L, rho_V) and saturation pressure of the PR
    EOS (Eq. 13) by the equal-area rule: p(rho_V) = p(rho_L) = p_s and
    int_{rho_V}^{rho_L} (p_s - p(rho)) / rho^2 d rho = 0 (equal areas in the
    specific-volume plane).  The spinodal interval brackets the roots."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    T = T_over_Tc * Tc(a, b, R)
    L = lib()
    tc, k = L.orc_Tc(a, b, R), L.orc_kappa(omega)

    def p(r):
        return L.orc_pressure(r, T, a, b, R, k, tc)

    def dp(r, h=1e-6):
        return (p(r + h) - p(r - h)) / (2 * h)

    grid = np.linspace(1e-3, 0.999 / b, 20000)
    dps = np.array([dp(r) for r in grid])
    neg = np.where(dps < 0)[0]
    if len(neg) == 0:
        raise ValueError("supercritical: no spinodal")
    r_sv, r_sl = grid[neg[0]], grid[neg[-1]]  # vapour and liquid spinodals
    p_lo, p_hi = max(p(r_sl), 1e-12), p(r_sv)

    def roots(ps):
        rv = brentq(lambda r: p(r) - ps, 0.0, r_sv)
        rl = brentq(lambda r: p(r) - ps, r_sl, 0.999 / b)
        return rv, rl

    def area(ps):
        rv, rl = roots(ps)
        val, _ = quad(lambda r: (ps - p(r)) / (r * r), rv, rl, limit=200, epsabs=1e-14, epsrel=1e-12)
        return val

    ps = brentq(area, p_lo * (1 + 1e-9), p_hi * (1 - 1e-9), xtol=1e-15, rtol=1e-14)
    rv, rl = roots(ps)
    return rl, rv, ps


def latent_heat(T_over_Tc=0.86, a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344, dT_rel=1e-4):
    """Specific latent heat h_fg = T (1/rho_V - 1/rho_L) dp_s/dT (Clausius-
    Clapeyron), with dp_s/dT from Maxwell constructions at T (1 +- dT_rel)."""
    rl, rv, _ = maxwell(T_over_Tc, a, b, R, omega)
    _, _, p_hi = maxwell(T_over_Tc * (1 + dT_rel), a, b, R, omega)
    _, _, p_lo = maxwell(T_over_Tc * (1 - dT_rel), a, b, R, omega)
    T = T_over_Tc * Tc(a, b, R)
    dps = (p_hi - p_lo) / (2 * T * dT_rel)
    return T * (1.0 / rv - 1.0 / rl) * dps
