"""The allocation-free gradient entry point (kwgb_gradient_static) against the
allocating one (kwgb_apply_operator), through the C ABI, and its failure
report (kwgb_gradient_static_status).

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

TIMEOUT = -5


def _lib():
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    return kwgb, kwgb.load()


def _desc(kwgb, shape):
    nz, ny, nx = shape
    d = kwgb.GridDesc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.dx, d.dy, d.dz = 1e-4, 1.25e-4, 0.8e-4
    d.dt, d.c_ref = 2e-8, 1500.0
    return d


def _reference(kwgb, f, op, stream):
    ref = [f.new_empty(f.shape) for _ in range(3)]
    sim = kwgb.Simulation(tuple(f.shape), (1e-4, 1.25e-4, 0.8e-4), 2e-8, 1500.0)
    sim.set_medium(1500.0, 1000.0)
    sim.apply_operator(op, f, ref, stream=stream)
    sim.close()
    return ref


def _static(L, kwgb, f, op, stream, err):
    import torch
    got = [torch.full_like(f, float("nan")) for _ in range(3)]
    d = _desc(kwgb, tuple(f.shape))
    rc = L.kwgb_gradient_static(ctypes.byref(d), op, f.data_ptr(), got[0].data_ptr(), got[1].data_ptr(),
                                got[2].data_ptr(), stream.cuda_stream, err, len(err))
    return rc, got


def _agree(got, ref):
    for g_, r_ in zip(got, ref):
        a, b = g_.cpu().numpy(), r_.cpu().numpy()
        assert rel_l2(a, b) <= 1e-5 and linf(a, b) <= 5e-5, rel_l2(a, b)


def test_static_gradient_matches_allocating_entry_point():
    import torch
    kwgb, L = _lib()
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()
    # two calls in a row (different grids, operators and inputs) share the scratch
    for call, (shape, op) in enumerate((((16, 32, 64), kwgb.OP_GRAD_FWD), ((64, 8, 32), kwgb.OP_GRAD_BWD))):
        rng = np.random.default_rng(100 + call)
        f = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        ref = _reference(kwgb, f, op, stream)
        rc, got = _static(L, kwgb, f, op, stream, err)
        assert rc == 0, err.value
        assert L.kwgb_gradient_static_status(stream.cuda_stream, err, len(err)) == 0, err.value
        _agree(got, ref)
    # sizes beyond the scratch, and a non-finite time step, are refused with a
    # message; nothing is launched
    d = _desc(kwgb, (128, 64, 64))
    x = torch.zeros(8, device="cuda")
    rc = L.kwgb_gradient_static(ctypes.byref(d), kwgb.OP_GRAD_FWD, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                x.data_ptr(), None, err, len(err))
    assert rc == -7 and b"[8, 64]" in err.value
    d = _desc(kwgb, (8, 8, 8))
    d.dt = float("inf")
    rc = L.kwgb_gradient_static(ctypes.byref(d), kwgb.OP_GRAD_FWD, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                x.data_ptr(), None, err, len(err))
    assert rc == -1 and b"finite" in err.value


def test_static_gradient_reports_a_wait_that_ran_out():
    """The test hook makes every tile load expect more bytes than arrive, so
    the kernels' bounded waits run out (no fault): the status query must
    report KWGB_ERR_TIMEOUT, and the next call without the hook computes
    normally on the same context."""
    import torch
    kwgb, L = _lib()
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()
    shape, op = (8, 16, 32), kwgb.OP_GRAD_FWD
    f = torch.from_numpy(np.random.default_rng(7).standard_normal(shape).astype(np.float32)).cuda()
    ref = _reference(kwgb, f, op, stream)
    L.kwgb_gradient_static_debug_wait_fault(1)
    try:
        rc, _ = _static(L, kwgb, f, op, stream, err)
        assert rc == 0, err.value
        assert L.kwgb_gradient_static_status(stream.cuda_stream, err, len(err)) == TIMEOUT
        assert b"wait" in err.value
    finally:
        L.kwgb_gradient_static_debug_wait_fault(0)
    rc, got = _static(L, kwgb, f, op, stream, err)
    assert rc == 0, err.value
    assert L.kwgb_gradient_static_status(stream.cuda_stream, err, len(err)) == 0, err.value
    _agree(got, ref)
