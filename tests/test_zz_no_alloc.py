"""The allocation-free gradient entry point (kwgb_gradient_static) against the
allocating one (kwgb_apply_operator), through the C ABI.

kwgb_gradient_static exists for callers that cannot allocate device memory
(memory owned by another allocator or a fixed arena, or code that must not
allocate after start-up); it takes its scratch from a file-scope device array
instead.  This file is collected last so that a run that stops at the first
failure has already run every other test."""

import ctypes

import numpy as np
import pytest

from helpers import linf, rel_l2

pytestmark = pytest.mark.gpu


def _desc(kwgb, shape):
    nz, ny, nx = shape
    d = kwgb.GridDesc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.dx, d.dy, d.dz = 1e-4, 1.25e-4, 0.8e-4
    d.dt, d.c_ref = 2e-8, 1500.0
    return d


def test_static_gradient_matches_allocating_entry_point():
    import torch
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    L = kwgb.load()
    L.kwgb_gradient_static.argtypes = [ctypes.POINTER(kwgb.GridDesc), ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
    L.kwgb_gradient_static.restype = ctypes.c_int
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()
    # two calls in a row (different grids, operators and inputs) share the scratch
    for call, (shape, op) in enumerate((((16, 32, 64), kwgb.OP_GRAD_FWD), ((64, 8, 32), kwgb.OP_GRAD_BWD))):
        rng = np.random.default_rng(100 + call)
        f = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        ref = [torch.empty_like(f) for _ in range(3)]
        sim = kwgb.Simulation(shape, (1e-4, 1.25e-4, 0.8e-4), 2e-8, 1500.0)
        sim.set_medium(1500.0, 1000.0)
        sim.apply_operator(op, f, ref, stream=stream)
        got = [torch.full_like(f, float("nan")) for _ in range(3)]
        d = _desc(kwgb, shape)
        rc = L.kwgb_gradient_static(ctypes.byref(d), op, f.data_ptr(), got[0].data_ptr(), got[1].data_ptr(),
                                    got[2].data_ptr(), stream.cuda_stream, err, len(err))
        assert rc == 0, err.value
        torch.cuda.synchronize()
        for g_, r_ in zip(got, ref):
            a, b = g_.cpu().numpy(), r_.cpu().numpy()
            assert rel_l2(a, b) <= 1e-5 and linf(a, b) <= 5e-5, (call, rel_l2(a, b))
        sim.close()
    # sizes beyond the scratch are refused with a message, nothing is launched
    d = _desc(kwgb, (128, 64, 64))
    x = torch.zeros(8, device="cuda")
    rc = L.kwgb_gradient_static(ctypes.byref(d), kwgb.OP_GRAD_FWD, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                x.data_ptr(), None, err, len(err))
    assert rc == -7 and b"[8, 64]" in err.value
