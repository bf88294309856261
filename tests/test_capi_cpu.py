"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, exports every function include/kwgb.h declares, and validates grid
descriptors without touching the device."""

import ctypes
import os
import re

import numpy as np

import pytest

from paper_1408_4675_gb300 import build, kwgb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return kwgb.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kwgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kwgb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("kwgb_create", "kwgb_set_medium", "kwgb_add_source", "kwgb_add_sensor", "kwgb_step",
              "kwgb_read", "kwgb_set_allocator", "kwgb_last_error", "kwgb_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _desc(**kw):
    d = kwgb.GridDesc()
    d.nx, d.ny, d.nz = kw.get("n", (64, 32, 16))
    d.dx = d.dy = d.dz = 1e-4
    d.dt, d.c_ref = 2e-8, 1500.0
    for i in range(3):
        d.pml_size[i] = kw.get("pml", 4)
        d.pml_alpha[i] = 2.0
    d.flags = kw.get("flags", 3)
    d.alpha_power = kw.get("y", 1.5)
    return d


@pytest.mark.parametrize("kw,code", [
    (dict(), 0),
    (dict(n=(12, 16, 16)), -7),          # not a power of two
    (dict(n=(2048, 8, 8)), -7),          # too large
    (dict(n=(4, 8, 8)), -7),             # too small
    (dict(n=(0, 8, 8)), -1),
    (dict(pml=8, n=(16, 16, 16)), -1),   # PML leaves no interior
    (dict(y=1.0), -1),
    (dict(y=3.5), -1),
    (dict(flags=16), -1),                # unknown flag bit
    (dict(flags=3 | 4 | 8), -1),         # both tensor-core forms
    (dict(flags=3 | 8), 0),              # float16-split tensor-core form
    (dict(flags=3 | 4, n=(16, 8, 16), pml=2), -7),   # tensor-core form needs ny, nz >= 16
])
def test_create_validates_descriptor(lib, kw, code):
    h = ctypes.c_void_p()
    d = _desc(**kw)
    rc = lib.kwgb_create(ctypes.byref(d), ctypes.byref(h))
    assert rc == code, lib.kwgb_last_error(None)
    if rc == 0:
        assert lib.kwgb_steps_done(h) == 0
        assert lib.kwgb_device_bytes(h) == 0        # nothing allocated before set_medium
        lib.kwgb_destroy(h)
    else:
        assert h.value is None
        assert len(lib.kwgb_last_error(None)) > 0


def test_state_errors_without_device(lib):
    h = ctypes.c_void_p()
    assert lib.kwgb_create(ctypes.byref(_desc()), ctypes.byref(h)) == 0
    assert lib.kwgb_step(h, 1, None) == -6           # no medium yet
    assert lib.kwgb_step(h, -1, None) == -1
    assert b"n_steps" in lib.kwgb_last_error(h)
    lib.kwgb_destroy(h)
    lib.kwgb_destroy(None)


def test_snapshot_calls_without_device(lib):
    h = ctypes.c_void_p()
    assert lib.kwgb_create(ctypes.byref(_desc()), ctypes.byref(h)) == 0
    lib.kwgb_state_bytes.restype = ctypes.c_int64
    assert lib.kwgb_state_bytes(h) == 0                      # no medium yet
    buf = ctypes.create_string_buffer(64)
    assert lib.kwgb_save_state(h, buf, ctypes.c_int64(64)) == -6
    assert lib.kwgb_load_state(h, buf, ctypes.c_int64(64)) == -6
    assert lib.kwgb_save_state(None, buf, ctypes.c_int64(64)) == -1
    lib.kwgb_destroy(h)



def test_series_capacity_validation_without_device():
    sim = kwgb.Simulation((16, 16, 16), (1e-4,) * 3, 2e-8, 1500.0)
    L = sim.L
    sid = sim.add_sensor(np.array([1, 2, 3]), kwgb.P_SERIES)
    other = sim.add_sensor(np.array([1]), kwgb.P_MAX)
    assert L.kwgb_set_series_capacity(sim.h, sid, 0) == -1          # capacity must be >= 1
    assert L.kwgb_set_series_capacity(sim.h, 99, 3) == -1           # bad sensor id
    assert L.kwgb_set_series_capacity(sim.h, other, 3) == -1        # records no series
    assert L.kwgb_set_series_capacity(sim.h, sid, 3) == 0
    # outputs before any step: no device access needed
    assert sim.read(sid, kwgb.P_SERIES).shape == (0, 3)
    assert np.all(np.isneginf(sim.read(other, kwgb.P_MAX)))
    assert L.kwgb_add_sensor(sim.h, None, 0, 64, ctypes.byref(ctypes.c_int32())) == -1   # unknown record bit
    sim.close()


def test_static_gradient_validates_without_device(lib):
    """kwgb_gradient_static checks its arguments before any CUDA call: null
    pointers and non-finite steps are ARG, grids beyond its fixed scratch
    UNSUPPORTED, each with a message in the caller's buffer."""
    err = ctypes.create_string_buffer(128)
    x = ctypes.c_void_p(16)               # never dereferenced: validation fails first
    d = _desc(n=(16, 16, 16))
    assert lib.kwgb_gradient_static(ctypes.byref(d), kwgb.OP_GRAD_FWD, None, x, x, x, None, err, 128) == -1
    assert lib.kwgb_gradient_static(ctypes.byref(d), 7, x, x, x, x, None, err, 128) == -1
    d = _desc(n=(128, 16, 16))
    assert lib.kwgb_gradient_static(ctypes.byref(d), kwgb.OP_GRAD_FWD, x, x, x, x, None, err, 128) == -7
    assert b"[8, 64]" in err.value
    for field in ("dt", "c_ref"):
        d = _desc(n=(16, 16, 16))
        setattr(d, field, float("nan"))
        assert lib.kwgb_gradient_static(ctypes.byref(d), kwgb.OP_GRAD_BWD, x, x, x, x, None, err, 128) == -1
        assert b"finite" in err.value


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without libkwgb.so the binding raises instead of computing."""
    monkeypatch.setattr(kwgb, "LIB_PATH", str(tmp_path / "libkwgb.so"))
    monkeypatch.setattr(kwgb, "_lib", None)
    with pytest.raises(ImportError):
        kwgb.load()
    with pytest.raises(ImportError):
        kwgb.Simulation((8, 8, 8), (1e-4, 1e-4, 1e-4), 1e-8, 1500.0)


def test_product_package_does_not_reach_the_oracle():
    """The oracle is test infrastructure: nothing in the package imports or runs it."""
    pkg = os.path.join(ROOT, "paper_1408_4675_gb300")
    pat = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)|[\"']oracle/|import_module\([\"']oracle", re.M)
    for dirpath, dirnames, filenames in os.walk(pkg):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_", "."))]
        for fn in filenames:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not pat.search(src), os.path.join(dirpath, fn)


def header_constants():
    src = open(os.path.join(ROOT, "include", "kwgb.h")).read()
    out = {}
    for name, val in re.findall(r"#define\s+KWGB_([A-Z0-9_]+)\s+(-?(?:0x[0-9a-fA-F]+|\d+))u?\b", src):
        out[name] = int(val, 0)
    return out


def test_binding_constants_match_the_header():
    """Every flag, record, source mode, field and operator code of the Python
    binding has the value the C header defines."""
    h = header_constants()
    for name in ("NONLINEAR", "ABSORBING", "MIXED_BF16", "MIXED_F16", "P_MAX", "P_RMS", "I_AVG", "P_MIN",
                 "P_SERIES", "U_SERIES", "ADDITIVE_MASS", "FORCE_X", "FORCE_Y", "FORCE_Z", "DIRICHLET_P",
                 "SCALAR_C0", "SCALAR_RHO0", "SCALAR_BONA", "SCALAR_ALPHA0", "INPUT_DEVICE", "FIELD_P",
                 "FIELD_UX", "FIELD_UY", "FIELD_UZ", "FIELD_RHOX", "FIELD_RHOY", "FIELD_RHOZ", "OP_GRAD_FWD",
                 "OP_GRAD_BWD", "OP_ABS_TAU", "OP_ABS_ETA"):
        assert name in h, name
        assert getattr(kwgb, name) == h[name], (name, getattr(kwgb, name), h[name])
    assert kwgb.KWGB_OK == h["OK"]
    for code, short in kwgb.ERRORS.items():
        assert h["ERR_" + short] == code, short
