"""Edge cases of the GPU path against the FP64 oracle: the smallest grid, a
1024-point z axis through whole steps (z passes of 1024-point lines), empty
and degenerate sources and sensors (no points, no samples, signals shorter
than the run, repeated points), and a medium given entirely as scalars."""

import numpy as np
import pytest

from helpers import linf, oracle_from_config, rel_l2
from paper_1408_4675_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kw():
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    return kwgb


def _small_cfg(shape, pml, steps, seed=3):
    nz, ny, nx = shape
    d = (1e-4, 1.1e-4, 0.9e-4)
    cfg = inputs.make_config(2, n=32, n_steps=steps)
    cfg["shape"] = shape
    cfg["d"] = d
    for key, lo, hi, sd in (("c0", 1450, 1650, seed), ("rho0", 950, 1100, seed + 1), ("bona", 5, 9, seed + 2)):
        cfg[key] = inputs.smooth_random_field(shape, lo, hi, sd, 1.5)
    cfg["alpha0"] = inputs.db_to_neper(inputs.smooth_random_field(shape, 0.3, 1.0, seed + 3, 1.5), 1.1)
    cfg["c_ref"] = float(cfg["c0"].max())
    cfg["dt"] = 0.3 * min(d) / cfg["c_ref"]
    cfg["pml_size"] = pml
    cfg["p0"] = inputs.gaussian_ball(shape, 1.0, 1e5)
    cfg["sources"] = []
    cfg["sensors"] = [(None, 3)]
    return cfg


def _compare(kw, cfg, steps, tol=(1e-3, 5e-3)):
    gsim, gids = kw.from_config(cfg)
    osim, oids = oracle_from_config(cfg)
    gsim.step(steps)
    osim.step(steps)
    of = osim.fields()
    for name in ("p", "ux", "uy", "uz", "rhox", "rhoy", "rhoz"):
        got = gsim.read_field(name)
        assert rel_l2(got, of[name]) <= tol[0], (name, rel_l2(got, of[name]))
        assert linf(got, of[name]) <= tol[1], (name, linf(got, of[name]))
    for (idx, rec), gi, oi in zip(cfg["sensors"], gids, oids):
        for which in (1, 2, 4, 8):
            if rec & which:
                got, ref = gsim.read(gi, which), osim.read(oi, which)
                assert got.shape == ref.shape
                if ref.size:
                    assert rel_l2(got, ref) <= tol[0], (which, rel_l2(got, ref))
    assert gsim.status() == 0
    gsim.close()


def test_smallest_grid(kw):
    cfg = _small_cfg((8, 8, 8), (1, 1, 1), 30)
    cfg["sources"] = [(np.array([0, 511, 73]), inputs.cw(1e6, 1e4, cfg["dt"], 30))]
    cfg["sensors"] = [(None, 3), (np.array([0, 7, 56, 511]), 15)]
    _compare(kw, cfg, 30)


def test_1024_point_z_lines_in_a_step(kw):
    cfg = _small_cfg((1024, 8, 16), (2, 1, 20), 25)          # pml_size is (x, y, z)
    cfg["p0"] = inputs.gaussian_ball(cfg["shape"], 2.0, 1e5, (512, 4, 8))
    _compare(kw, cfg, 25)


@pytest.mark.parametrize("nz", [256, 512])
def test_256_and_512_point_z_lines_in_a_step(kw, nz):
    """The two-columns-per-thread z passes, with a ragged last column pair (nx = 32: 17 columns)."""
    cfg = _small_cfg((nz, 8, 32), (2, 1, 20), 25)
    cfg["p0"] = inputs.gaussian_ball(cfg["shape"], 2.0, 1e5, (nz // 2, 4, 16))
    _compare(kw, cfg, 25)


def test_1024_point_y_lines_in_a_step(kw):
    cfg = _small_cfg((8, 1024, 16), (2, 20, 1), 25)
    cfg["p0"] = inputs.gaussian_ball(cfg["shape"], 2.0, 1e5, (4, 512, 8))
    _compare(kw, cfg, 25)


def test_degenerate_sources_and_sensors(kw):
    cfg = _small_cfg((16, 16, 32), (2, 2, 2), 20)
    sig = inputs.cw(1e6, 2e4, cfg["dt"], 8)                   # shorter than the run
    cfg["sources"] = [
        (np.array([], dtype=np.int64), np.zeros(20)),         # no points
        (np.array([100, 101]), np.zeros((1, 0))),             # no samples
        (np.array([300, 300, 301, 300]), sig),                # repeated points add up
    ]
    cfg["sensors"] = [(np.array([], dtype=np.int64), 3),      # no points
                      (np.array([300, 300, 5000]), 15),       # repeated point
                      (None, 9)]
    _compare(kw, cfg, 20)


def test_scalar_medium(kw):
    cfg = _small_cfg((16, 32, 16), (2, 2, 2), 30)
    cfg["c0"], cfg["rho0"], cfg["bona"] = 1540.0, 1040.0, 7.0
    cfg["alpha0"] = float(inputs.db_to_neper(0.75, 1.1))
    cfg["c_ref"] = 1540.0
    cfg["sources"] = [(np.array([40, 41, 42]), inputs.tone_burst(1e6, 2, 3e4, cfg["dt"], 30))]
    _compare(kw, cfg, 30)


def test_device_medium_input_matches_host(kw):
    """The medium given as device arrays (CUDA tensors, KWGB_INPUT_DEVICE)
    steps bitwise like the same medium given as host arrays."""
    import torch
    cfg = _small_cfg((32, 16, 64), (4, 2, 4), 20)
    cfg["sources"] = [(np.arange(100, 900, 13), inputs.cw(1e6, 2e4, cfg["dt"], 20))]
    out = []
    for on_device in (False, True):
        sim = kw.Simulation(cfg["shape"], cfg["d"], cfg["dt"], cfg["c_ref"], cfg["pml_size"], cfg["pml_alpha"],
                            cfg["flags"], cfg["alpha_power"])
        med = [np.asarray(cfg[k], dtype=np.float32) for k in ("c0", "rho0", "bona", "alpha0")]
        if on_device:
            med = [torch.from_numpy(m).cuda() for m in med]
        sim.set_medium(*med)
        sim.set_initial_pressure(cfg["p0"])
        for idx, sig in cfg["sources"]:
            sim.add_source(idx, sig)
        sid = sim.add_sensor(None, 3)
        sim.step(20)
        out.append([sim.read_field(n) for n in ("p", "ux", "rhoz")] + [sim.read(sid, 1), sim.read(sid, 2)])
        assert sim.status() == 0
        sim.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
