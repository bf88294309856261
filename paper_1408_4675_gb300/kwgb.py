"""Thin Python binding of the C ABI in include/kwgb.h (argument marshalling
only: every step of the time step runs in the CUDA library).

The library must have been built (``paper_1408_4675_gb300.build.build()``);
there is no CPU fallback: a missing or unloadable libkwgb.so raises.
PyTorch supplies device memory (its caching allocator backs the library's
allocations when CUDA is available) and streams.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkwgb.so")

KWGB_OK = 0
ERRORS = {-1: "ARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT", -6: "STATE",
          -7: "UNSUPPORTED"}

NONLINEAR, ABSORBING = 1, 2
MIXED_BF16, MIXED_F16 = 4, 8          # split-precision tensor-core y/z FFT stages (KWGB_MIXED_*)
P_MAX, P_RMS, I_AVG, P_MIN, P_SERIES, U_SERIES = 1, 2, 4, 8, 16, 32
ADDITIVE_MASS = 0
FORCE_X, FORCE_Y, FORCE_Z = 1, 2, 3
DIRICHLET_P = 4
SCALAR_C0, SCALAR_RHO0, SCALAR_BONA, SCALAR_ALPHA0 = 1, 2, 4, 8
INPUT_DEVICE = 0x80000000
FIELD_P, FIELD_UX, FIELD_UY, FIELD_UZ, FIELD_RHOX, FIELD_RHOY, FIELD_RHOZ = range(7)
OP_GRAD_FWD, OP_GRAD_BWD, OP_ABS_TAU, OP_ABS_ETA = range(4)
FIELDS = {"p": FIELD_P, "ux": FIELD_UX, "uy": FIELD_UY, "uz": FIELD_UZ,
          "rhox": FIELD_RHOX, "rhoy": FIELD_RHOY, "rhoz": FIELD_RHOZ}


class KwgbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("kwgb error %s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("c_ref", ctypes.c_double),
                ("pml_size", ctypes.c_int32 * 3), ("pml_alpha", ctypes.c_double * 3),
                ("flags", ctypes.c_uint32), ("alpha_power", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def load():
    """Load libkwgb.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libkwgb.so is not built; run paper_1408_4675_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    L.kwgb_create.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(vp)]
    L.kwgb_set_allocator.argtypes = [vp, ALLOC_FN, FREE_FN, vp]
    L.kwgb_set_medium.argtypes = [vp, vp, vp, vp, vp, u32]
    L.kwgb_set_initial_pressure.argtypes = [vp, vp]
    L.kwgb_add_source.argtypes = [vp, vp, i64, vp, i64, i64, ctypes.c_int, ctypes.POINTER(i32)]
    L.kwgb_add_sensor.argtypes = [vp, vp, i64, u32, ctypes.POINTER(i32)]
    L.kwgb_step.argtypes = [vp, i64, vp]
    L.kwgb_read.argtypes = [vp, i32, u32, vp, i64]
    L.kwgb_read_field.argtypes = [vp, ctypes.c_int, vp, i64]
    L.kwgb_apply_operator.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp]
    L.kwgb_steps_done.argtypes = [vp]
    L.kwgb_steps_done.restype = i64
    L.kwgb_status.argtypes = [vp]
    L.kwgb_device_bytes.argtypes = [vp]
    L.kwgb_device_bytes.restype = i64
    L.kwgb_last_error.argtypes = [vp]
    L.kwgb_last_error.restype = ctypes.c_char_p
    L.kwgb_launch_count.argtypes = [vp]
    L.kwgb_launch_count.restype = i64
    L.kwgb_step_profiled.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(i32)]
    L.kwgb_step_profiled.restype = ctypes.c_int
    L.kwgb_kernel_name.argtypes = [i32]
    L.kwgb_kernel_name.restype = ctypes.c_char_p
    L.kwgb_adjoint.argtypes = [vp, vp, i64, ctypes.c_int, i64, i64, ctypes.POINTER(ctypes.c_double), vp, i64, vp]
    L.kwgb_adjoint.restype = ctypes.c_int
    L.kwgb_adjoint_forward.argtypes = [vp, vp, i64, ctypes.c_int, i64, i64, ctypes.POINTER(ctypes.c_double), vp]
    L.kwgb_adjoint_forward.restype = ctypes.c_int
    L.kwgb_adjoint_backward.argtypes = [vp, vp, i64, vp]
    L.kwgb_adjoint_backward.restype = ctypes.c_int
    L.kwgb_set_series_capacity.argtypes = [vp, i32, i64]
    L.kwgb_set_series_capacity.restype = ctypes.c_int
    L.kwgb_state_bytes.argtypes = [vp]
    L.kwgb_state_bytes.restype = i64
    L.kwgb_save_state.argtypes = [vp, vp, i64]
    L.kwgb_save_state.restype = ctypes.c_int
    L.kwgb_load_state.argtypes = [vp, vp, i64]
    L.kwgb_load_state.restype = ctypes.c_int
    L.kwgb_debug_wait_fault.argtypes = [vp, ctypes.c_int]
    L.kwgb_debug_wait_fault.restype = ctypes.c_int
    L.kwgb_gradient_static.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int, vp, vp, vp, vp, vp,
                                       ctypes.c_char_p, ctypes.c_size_t]
    L.kwgb_gradient_static.restype = ctypes.c_int
    L.kwgb_gradient_static_status.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    L.kwgb_gradient_static_status.restype = ctypes.c_int
    L.kwgb_gradient_static_debug_wait_fault.argtypes = [ctypes.c_int]
    L.kwgb_gradient_static_debug_wait_fault.restype = ctypes.c_int
    L.kwgb_destroy.argtypes = [vp]
    L.kwgb_destroy.restype = None
    for name in ("kwgb_create", "kwgb_set_allocator", "kwgb_set_medium", "kwgb_set_initial_pressure",
                 "kwgb_add_source", "kwgb_add_sensor", "kwgb_step", "kwgb_read", "kwgb_read_field",
                 "kwgb_apply_operator", "kwgb_status"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _f32(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Simulation:
    """One simulation on the current CUDA device (see include/kwgb.h)."""

    def __init__(self, shape, spacing, dt, c_ref, pml_size=(0, 0, 0), pml_alpha=(0.0, 0.0, 0.0),
                 flags=0, alpha_power=1.5, use_torch_allocator=True):
        self.L = load()
        nz, ny, nx = shape
        d = GridDesc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.dx, d.dy, d.dz = spacing
        d.dt, d.c_ref = dt, c_ref
        for i in range(3):
            d.pml_size[i] = int(pml_size[i])
            d.pml_alpha[i] = float(pml_alpha[i])
        d.flags = int(flags)
        d.alpha_power = float(alpha_power)
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        h = ctypes.c_void_p()
        rc = self.L.kwgb_create(ctypes.byref(d), ctypes.byref(h))
        if rc != KWGB_OK:
            raise KwgbError(rc, self.L.kwgb_last_error(None).decode())
        self.h = h
        self._cb = None
        self._sensors = []
        self._caps = []
        self._src_shapes = []
        if use_torch_allocator:
            self._use_torch_allocator()

    def _use_torch_allocator(self):
        import torch
        if not torch.cuda.is_available():
            return
        dev = torch.cuda.current_device()

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(nbytes, dev)
            except Exception:
                return None

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
        self._check(self.L.kwgb_set_allocator(self.h, self._cb[0], self._cb[1], None))

    def _check(self, rc):
        if rc != KWGB_OK:
            raise KwgbError(rc, self.L.kwgb_last_error(self.h).decode())
        return rc

    # -- inputs ---------------------------------------------------------
    def set_medium(self, c0, rho0, bona=None, alpha0=None):
        """Each argument is a scalar, a host array of the grid's size, or a
        CUDA torch tensor (then all non-scalar arguments must be)."""
        mask = 0
        keep = []
        ptrs = []
        device = None
        for bit, v in ((SCALAR_C0, c0), (SCALAR_RHO0, rho0), (SCALAR_BONA, bona), (SCALAR_ALPHA0, alpha0)):
            if v is None:
                ptrs.append(None)
                continue
            if np.isscalar(v) or (isinstance(v, np.ndarray) and v.ndim == 0):
                a = np.array([v], dtype=np.float32)
                mask |= bit
                keep.append(a)
                ptrs.append(_ptr(a))
            elif hasattr(v, "is_cuda") and v.is_cuda:
                t = v.contiguous().float()
                if t.numel() != self.N:
                    raise ValueError("medium field has the wrong size")
                keep.append(t)
                ptrs.append(ctypes.c_void_p(t.data_ptr()))
                device = True
            else:
                a = _f32(v, self.N)
                keep.append(a)
                ptrs.append(_ptr(a))
                if device:
                    raise ValueError("mix of host and device medium arrays")
                device = False if device is None else device
        if device:
            mask |= INPUT_DEVICE
        self._check(self.L.kwgb_set_medium(self.h, *ptrs, mask))

    def set_initial_pressure(self, p0):
        a = _f32(p0, self.N)
        self._check(self.L.kwgb_set_initial_pressure(self.h, _ptr(a)))

    def add_source(self, idx, signal, mode=ADDITIVE_MASS):
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        sig = np.atleast_2d(_f32(signal))
        sid = ctypes.c_int32()
        self._check(self.L.kwgb_add_source(self.h, _ptr(idx), idx.size, _ptr(sig), sig.shape[0],
                                           sig.shape[1], mode, ctypes.byref(sid)))
        self._src_shapes.append(sig.shape)
        return sid.value

    def add_sensor(self, idx=None, record=P_MAX):
        sid = ctypes.c_int32()
        if idx is None:
            self._check(self.L.kwgb_add_sensor(self.h, None, 0, record, ctypes.byref(sid)))
            n = self.N
        else:
            idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
            self._check(self.L.kwgb_add_sensor(self.h, _ptr(idx), idx.size, record, ctypes.byref(sid)))
            n = idx.size
        self._sensors.append(n)
        self._caps.append(0)
        return sid.value

    def set_series_capacity(self, sensor_id, n_t):
        """Ring length of a P_SERIES / U_SERIES sensor (the last n_t steps are kept)."""
        self._check(self.L.kwgb_set_series_capacity(self.h, sensor_id, int(n_t)))
        self._caps[sensor_id] = int(n_t)

    # -- stepping and outputs -----------------------------------------------
    def step(self, n=1, stream=None):
        self._check(self.L.kwgb_step(self.h, int(n), _stream_ptr(stream)))

    @property
    def steps_done(self):
        return self.L.kwgb_steps_done(self.h)

    def save_state(self):
        """Snapshot of the run (fields, sensor accumulators, step index) as a
        bytes-like uint8 array (kwgb_save_state)."""
        n = self.L.kwgb_state_bytes(self.h)
        if n <= 0:
            raise KwgbError(-6, self.L.kwgb_last_error(self.h).decode())
        buf = np.empty(n, dtype=np.uint8)
        self._check(self.L.kwgb_save_state(self.h, _ptr(buf), n))
        return buf

    def load_state(self, buf):
        """Restore a snapshot from save_state (kwgb_load_state)."""
        buf = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if not isinstance(buf, np.ndarray) else buf,
                                   dtype=np.uint8)
        self._check(self.L.kwgb_load_state(self.h, _ptr(buf), buf.size))

    def read(self, sensor_id, which):
        """P_MAX / P_MIN / P_RMS: (n,); I_AVG: (3, n); P_SERIES: (m, n); U_SERIES:
        (m, 3, n) with m = min(steps taken, capacity), oldest sample first."""
        npts = self._sensors[sensor_id]
        m = min(self.steps_done, self._caps[sensor_id])
        shape = {I_AVG: (3, npts), P_SERIES: (m, npts), U_SERIES: (m, 3, npts)}.get(which, (npts,))
        out = np.empty(int(np.prod(shape)), dtype=np.float64)
        self._check(self.L.kwgb_read(self.h, sensor_id, which, _ptr(out), out.size))
        return out.reshape(shape)

    def read_field(self, name):
        out = np.empty(self.shape, dtype=np.float32)
        self._check(self.L.kwgb_read_field(self.h, FIELDS[name], _ptr(out), out.size))
        return out

    def apply_operator(self, op, field, outs, stream=None):
        """op on a CUDA float32 tensor `field` into CUDA tensors `outs`."""
        p = [ctypes.c_void_p(t.data_ptr()) for t in outs] + [None] * (3 - len(outs))
        self._check(self.L.kwgb_apply_operator(self.h, op, ctypes.c_void_p(field.data_ptr()),
                                               p[0], p[1], p[2], _stream_ptr(stream)))

    @property
    def launch_count(self):
        return self.L.kwgb_launch_count(self.h)

    def step_profiled(self, stream=None):
        """One step with per-launch CUDA-event timing: [(kernel name, ms), ...]."""
        cap = 64
        kinds = np.zeros(cap, dtype=np.int32)
        ms = np.zeros(cap, dtype=np.float32)
        n = ctypes.c_int32()
        self._check(self.L.kwgb_step_profiled(self.h, _stream_ptr(stream), _ptr(kinds), _ptr(ms),
                                              cap, ctypes.byref(n)))
        return [(self.L.kwgb_kernel_name(int(kinds[i])).decode(), float(ms[i])) for i in range(n.value)]

    def adjoint(self, obj_idx, n_steps, checkpoint_every=50, stream=None):
        """Run n_steps forward and the adjoint; returns (J, [dJ/dsignal per
        source, shaped (n_signals, n_t)]) for J = mean |p| over obj_idx."""
        obj = np.ascontiguousarray(np.asarray(obj_idx, dtype=np.int64))
        shapes = [tuple(s) for s in self._src_shapes]
        total = sum(a * b for a, b in shapes)
        g = np.zeros(max(total, 1), dtype=np.float64)
        J = ctypes.c_double()
        self._check(self.L.kwgb_adjoint(self.h, _ptr(obj), obj.size, 0, int(n_steps), int(checkpoint_every),
                                        ctypes.byref(J), _ptr(g), g.size, _stream_ptr(stream)))
        out, o = [], 0
        for a, b in shapes:
            out.append(g[o:o + a * b].reshape(a, b))
            o += a * b
        return J.value, out

    def adjoint_forward(self, obj_idx, n_steps, checkpoint_every=50, stream=None):
        """Run n_steps forward and return J = mean |p| over obj_idx.  With
        0 < checkpoint_every < n_steps the simulation keeps the checkpoints
        that adjoint_backward() recomputes from; with checkpoint_every >=
        n_steps it keeps every step's density fields (28 N bytes a step) and
        adjoint_backward() recomputes nothing; with 0 it computes J only."""
        obj = np.ascontiguousarray(np.asarray(obj_idx, dtype=np.int64))
        J = ctypes.c_double()
        self._check(self.L.kwgb_adjoint_forward(self.h, _ptr(obj), obj.size, 0, int(n_steps), int(checkpoint_every),
                                                ctypes.byref(J), _stream_ptr(stream)))
        return J.value

    def adjoint_backward(self, stream=None):
        """Reverse pass of the preceding adjoint_forward(); returns
        [dJ/dsignal per source, shaped (n_signals, n_t)]."""
        shapes = [tuple(s) for s in self._src_shapes]
        total = sum(a * b for a, b in shapes)
        g = np.zeros(max(total, 1), dtype=np.float64)
        self._check(self.L.kwgb_adjoint_backward(self.h, _ptr(g), g.size, _stream_ptr(stream)))
        out, o = [], 0
        for a, b in shapes:
            out.append(g[o:o + a * b].reshape(a, b))
            o += a * b
        return out

    def status(self):
        return self.L.kwgb_status(self.h)

    @property
    def device_bytes(self):
        return self.L.kwgb_device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            self.L.kwgb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_config(cfg, use_torch_allocator=True):
    """Build a Simulation from an inputs.make_config() dictionary."""
    sim = Simulation(cfg["shape"], cfg["d"], cfg["dt"], cfg["c_ref"], cfg["pml_size"],
                     cfg["pml_alpha"], cfg["flags"], cfg["alpha_power"],
                     use_torch_allocator=use_torch_allocator)
    sim.set_medium(cfg["c0"], cfg["rho0"], cfg["bona"], cfg["alpha0"])
    if cfg.get("p0") is not None:
        sim.set_initial_pressure(cfg["p0"])
    for src in cfg["sources"]:                     # (idx, signal) or (idx, signal, mode)
        sim.add_source(*src)
    ids = [sim.add_sensor(idx, rec) for idx, rec in cfg["sensors"]]
    for i, (idx, rec) in zip(ids, cfg["sensors"]):
        if rec & (P_SERIES | U_SERIES):
            sim.set_series_capacity(i, cfg.get("series_capacity", cfg["n_steps"]))
    return sim, ids
