"""Failure detection without a GPU fault: a bounded wait that runs out
(test hook: the tile loads expect more bytes than arrive) is reported as
KWGB_ERR_TIMEOUT and the CUDA context stays usable; a pressure that
overflows is reported as KWGB_ERR_NONFINITE; an allocator that refuses
memory gives KWGB_ERR_OOM."""

import ctypes

import numpy as np
import pytest

from paper_1408_4675_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kw():
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    return kwgb


def _sim(kw, n=32):
    sim = kw.Simulation((n, n, n), (1e-4,) * 3, 2e-8, 1500.0, (2, 2, 2), (2.0, 2.0, 2.0),
                        flags=kw.ABSORBING, alpha_power=1.3)
    sim.set_medium(1500.0, 1000.0, 0.0, 1e-3)
    return sim


def test_bounded_wait_runs_out_and_context_survives(kw):
    import torch
    n = 32
    sim = _sim(kw, n)
    f = torch.randn(n, n, n, device="cuda")
    out = torch.empty_like(f)
    assert sim.L.kwgb_debug_wait_fault(sim.h, 1) == 0
    sim.apply_operator(kw.OP_ABS_TAU, f, [out])               # the y and z pass waits run out (2 s each)
    assert sim.status() == -5                                  # KWGB_ERR_TIMEOUT
    sim.close()
    # the context is still usable: a fresh simulation computes the same operator normally
    sim2 = _sim(kw, n)
    sim2.apply_operator(kw.OP_ABS_TAU, f, [out])
    torch.cuda.synchronize()
    assert sim2.status() == 0
    assert torch.isfinite(out).all()
    sim2.close()


def test_overflowing_pressure_is_reported(kw):
    cfg = inputs.make_config(2, n=32, n_steps=10)
    cfg["sources"] = [(np.array([5000, 5001]), np.full(10, 3e38, dtype=np.float32))]
    sim, _ = kw.from_config(cfg)
    sim.step(10)
    assert sim.status() == -4                                  # KWGB_ERR_NONFINITE
    sim.close()


def test_refusing_allocator_gives_oom(kw):
    sim = kw.Simulation((32, 32, 32), (1e-4,) * 3, 2e-8, 1500.0, use_torch_allocator=False)
    refuse = kw.ALLOC_FN(lambda nbytes, ctx: None)
    noop = kw.FREE_FN(lambda p, ctx: None)
    assert sim.L.kwgb_set_allocator(sim.h, refuse, noop, None) == 0
    c0 = np.full((32, 32, 32), 1500.0, np.float32)
    rho0 = np.full((32, 32, 32), 1000.0, np.float32)
    rc = sim.L.kwgb_set_medium(sim.h, c0.ctypes.data_as(ctypes.c_void_p), rho0.ctypes.data_as(ctypes.c_void_p),
                               None, None, 0)
    assert rc == -2                                            # KWGB_ERR_OOM
    sim.close()
