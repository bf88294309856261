"""Checkpoint / restart (kwgb_save_state / kwgb_load_state): a run stopped,
saved, restored into a fresh simulation set up the same way and continued is
bitwise identical to the uninterrupted run -- fields, p_max, p_rms and the
time-averaged intensity -- and a snapshot is refused by a simulation with a
different sensor layout."""

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


def _outputs(sim, ids, cfg):
    out = []
    for (idx, rec), i in zip(cfg["sensors"], ids):
        for which in (1, 2, 4):
            if rec & which:
                out.append(sim.read(i, which))
    for name in ("p", "ux", "uy", "uz", "rhox", "rhoy", "rhoz"):
        out.append(sim.read_field(name))
    return out


@pytest.mark.parametrize("cfgid,n,total,stop", [(3, 32, 40, 17), (2, 32, 30, 11), (5, 32, 25, 9)])
def test_restart_is_bitwise_identical(kw, cfgid, n, total, stop):
    cfg = inputs.make_config(cfgid, n=n, n_steps=total)
    a, ida = kw.from_config(cfg)
    a.step(total)
    ref = _outputs(a, ida, cfg)
    a.close()
    b, idb = kw.from_config(cfg)
    b.step(stop)
    snap = b.save_state()
    b.close()
    c, idc = kw.from_config(cfg)
    c.load_state(snap)
    assert c.steps_done == stop
    c.step(total - stop)
    got = _outputs(c, idc, cfg)
    assert c.status() == 0
    c.close()
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y)


def test_snapshot_needs_the_same_layout(kw):
    cfg = inputs.make_config(3, n=32, n_steps=5)
    b, _ = kw.from_config(cfg)
    b.step(3)
    snap = b.save_state()
    b.close()
    other = dict(cfg)
    other["sensors"] = cfg["sensors"][:1]
    c, _ = kw.from_config(other)
    with pytest.raises(kw.KwgbError) as e:
        c.load_state(snap)
    assert e.value.code == -1
    with pytest.raises(kw.KwgbError):
        c.load_state(np.zeros(16, np.uint8))
    c.close()
