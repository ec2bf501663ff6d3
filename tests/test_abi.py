"""The C-ABI library builds for sm_103a, loads, exports every entry point
declared in include/lbm.h, its structs match the binding, and the host-side
configuration checks reject bad input before touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1911_10747_gb300 import build as B
from paper_1911_10747_gb300 import lbm
from paper_1911_10747_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.check_output(["nm", "-D", "--defined-only", B.LIB]).decode()
    exported = set(re.findall(r" T (lbm_[a-z0-9_]+)", out))
    assert set(names) <= exported, set(names) - exported
    assert set(names) == set(lbm.EXPORTS)
    for n in names:
        getattr(lib, n)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "lbm.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(lbm_domain_t),sizeof(lbm_heater_t),sizeof(lbm_eos_t),sizeof(lbm_bc_t),sizeof(lbm_opts_t),'
                   'offsetof(lbm_domain_t, seed),offsetof(lbm_bc_t, c_w_top));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(lbm.lbm_domain_t), C.sizeof(lbm.lbm_heater_t), C.sizeof(lbm.lbm_eos_t),
            C.sizeof(lbm.lbm_bc_t), C.sizeof(lbm.lbm_opts_t), lbm.lbm_domain_t.seed.offset,
            lbm.lbm_bc_t.c_w_top.offset]
    assert got == want


@pytest.mark.parametrize("change, field", [
    (dict(nf=1), "ny_fluid"),
    (dict(ns=1), "ny_solid"),
    (dict(G=1.0), "eos.G"),
    (dict(s=(1.0, 0.8, 0.8, 1.0, 2.5, 1.0, 1.1, 1.0, 1.0)), "MRT"),
    (dict(periodic_y=True), "periodic"),
    (dict(rho_V=7.0), "rho_L > rho_V"),
    (dict(nx=0), "domain.nx"),
    (dict(ns=2), "ny_solid"),
    (dict(liquid_rows=200), "liquid_rows"),
    (dict(nx=1 << 20, nf=1 << 12), "too large"),  # 4.3e9 sites: rejected before any allocation
])
def test_invalid_configuration_is_rejected_on_the_host(lib, change, field):
    cfg = W.small_parity().replace(**change)
    structs = lbm.structs_from_config(cfg)
    h = C.c_void_p()
    rc = lib.lbm_create(*[C.byref(s) for s in structs], C.byref(h))
    assert rc == lbm.LBM_E_INVAL
    assert not h.value
    assert field in lib.lbm_last_error(None).decode()


def test_status_strings(lib):
    assert lib.lbm_status_string(0) == b"LBM_OK"
    assert lib.lbm_status_string(4) == b"LBM_E_NUMERIC"


def test_null_arguments(lib):
    assert lib.lbm_destroy(None) == lbm.LBM_OK
    assert lib.lbm_step(None, 1) == lbm.LBM_E_INVAL
    assert lib.lbm_step_count(None) == -1


@pytest.mark.parametrize("bits, iters", [(16, 64), (64, 0), (32, (1 << 24) + 1)])
def test_fma_probe_rejects_bad_arguments_on_the_host(lib, bits, iters):
    v = C.c_double(-1.0)
    assert lib.lbm_peak_fma(-1, bits, iters, C.byref(v)) == lbm.LBM_E_INVAL
    assert "lbm_peak_fma" in lib.lbm_last_error(None).decode()
    assert v.value == -1.0
    assert lib.lbm_peak_fma(-1, 32, 64, None) == lbm.LBM_E_INVAL


def test_allocator_callbacks_must_come_in_pairs(lib):
    """opts.dev_alloc without opts.dev_free (or the reverse) is rejected on
    the host, before any device work."""
    cfg = W.small_parity()
    for half in ("dev_alloc", "dev_free"):
        structs = lbm.structs_from_config(cfg)
        op = structs[4]
        if half == "dev_alloc":
            op.dev_alloc = lbm.DEV_ALLOC_FN(lambda n, ctx: None)
        else:
            op.dev_free = lbm.DEV_FREE_FN(lambda p, ctx: None)
        h = C.c_void_p()
        assert lib.lbm_create(*[C.byref(s) for s in structs], C.byref(h)) == lbm.LBM_E_INVAL
        assert not h.value
        assert "dev_alloc" in lib.lbm_last_error(None).decode()


def test_get_state_without_a_run_is_rejected(lib):
    step = C.c_int64(-7)
    assert lib.lbm_get_state(None, None, None, C.byref(step), 0) == lbm.LBM_E_INVAL
    assert step.value == -7


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without the CUDA library the binding raises instead
    of computing anything, for a direct load and for a run."""
    missing = str(tmp_path / "liblbm_gb300.so")
    monkeypatch.setattr(lbm, "_lib", None)
    with pytest.raises(ImportError, match="no CPU path"):
        lbm.load(missing)
    monkeypatch.setattr(lbm.load, "__defaults__", (missing,))
    with pytest.raises(ImportError, match="no CPU path"):
        lbm.Run(W.small_parity())
