"""Time-series sensor outputs on the GPU (p_min, p and u series in a device
ring buffer) against the FP64 oracle: every recorded sample, element by
element, including a ring shorter than the run (the last samples are kept,
oldest first) and a full-grid p_min."""

import numpy as np
import pytest

import oracle
from helpers import oracle_from_config, rel_l2
from paper_1408_4675_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kw():
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    return kwgb


def test_series_match_the_oracle(kw):
    steps = 40
    cfg = inputs.make_config(2, n=32, n_steps=steps)
    rng = np.random.default_rng(2)
    pts = np.sort(rng.choice(32 ** 3, 57, replace=False))
    rec = oracle.P_MAX | oracle.P_MIN | oracle.P_RMS | oracle.P_SERIES | oracle.U_SERIES
    cfg["sensors"] = [(pts, rec), (None, oracle.P_MAX | oracle.P_MIN), (pts[:5], oracle.P_SERIES)]
    gsim, gids = kw.from_config(cfg)
    gsim.set_series_capacity(gids[2], 7)                   # ring shorter than the run
    osim, oids = oracle_from_config(cfg)
    gsim.step(steps)
    osim.step(steps)
    for which in (oracle.P_MAX, oracle.P_MIN, oracle.P_RMS, oracle.P_SERIES, oracle.U_SERIES):
        got, ref = gsim.read(gids[0], which), osim.read(oids[0], which)
        assert got.shape == ref.shape, (which, got.shape, ref.shape)
        assert rel_l2(got, ref) <= 1e-3, (which, rel_l2(got, ref))
    assert rel_l2(gsim.read(gids[1], oracle.P_MIN), osim.read(oids[1], oracle.P_MIN)) <= 1e-3
    tail = gsim.read(gids[2], oracle.P_SERIES)
    assert tail.shape == (7, 5)
    np.testing.assert_array_equal(tail, gsim.read(gids[0], oracle.P_SERIES)[-7:, :5])
    gsim.close()


def test_series_before_stepping_and_errors(kw):
    cfg = inputs.make_config(2, n=32, n_steps=4)
    cfg["sensors"] = [(np.array([3, 4, 5]), oracle.P_SERIES | oracle.P_MIN)]
    cfg["series_capacity"] = 4
    gsim, gids = kw.from_config(cfg)
    assert gsim.read(gids[0], oracle.P_SERIES).shape == (0, 3)
    assert np.all(np.isposinf(gsim.read(gids[0], oracle.P_MIN)))
    gsim.close()
    cfg2 = dict(cfg)
    cfg2.pop("series_capacity")
    sim = kw.Simulation(cfg["shape"], cfg["d"], cfg["dt"], cfg["c_ref"], cfg["pml_size"], cfg["pml_alpha"],
                        cfg["flags"], cfg["alpha_power"])
    sim.set_medium(cfg["c0"], cfg["rho0"], cfg["bona"], cfg["alpha0"])
    sim.add_sensor(np.array([3]), oracle.U_SERIES)
    with pytest.raises(kw.KwgbError) as e:                 # no capacity set
        sim.step(1)
    assert e.value.code == -1
    sim.close()
