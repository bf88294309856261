"""Host logic of bench.py that the reported numbers rest on: the algorithmic
byte model of each kernel (the roofline's numerator), the L2 note and the
clock record."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _cfg(n, flags, hetero=True, sensors=((np.arange(10), 7),)):
    field = np.zeros((1, 1, 1)) if hetero else 1500.0       # only the array-ness matters to the model
    return {"shape": (n, n, n), "flags": flags, "c0": field, "rho0": field, "bona": field, "alpha0": field,
            "sensors": list(sensors)}


def test_step_bytes_of_the_heterogeneous_nonlinear_absorbing_step():
    """Per step: 56 half-spectrum passes S and 20 real fields F (the 512^3 step's 40.9 GB)."""
    n = 512
    S = (n // 2 + 1) * 8 * n * n
    F = 4 * n ** 3
    b = bench.kernel_bytes(_cfg(n, 3))
    assert sum(b.values()) == 56 * S + 20 * F
    assert abs(sum(b.values()) / 1e9 - 40.92) < 0.01
    assert b["x_vel"] == 6 * S + 7 * F and b["x_dens"] == 5 * S + 8 * F
    assert b["z_div"] == 6 * S and b["z_grad"] == 4 * S and b["z_abs"] == 4 * S
    assert len(b) == 12


def test_byte_model_variants():
    n = 64
    S = (n // 2 + 1) * 8 * n * n
    F = 4 * n ** 3
    lossless = bench.kernel_bytes(_cfg(n, 0))               # 10 FFTs: no absorption passes, EOS in x_dens
    assert "x_eos" not in lossless and "z_abs" not in lossless
    assert lossless["x_dens"] == 4 * S + 6 * F + 2 * F      # rho0, c0 (linear: no B/A)
    scalar = bench.kernel_bytes(_cfg(n, 3, hetero=False))   # scalar medium values read nothing
    assert scalar["x_eos"] == 3 * S + F and scalar["x_vel"] == 6 * S + 6 * F
    full = bench.kernel_bytes(_cfg(n, 3, sensors=((None, 3),)))
    assert full["x_eos"] - bench.kernel_bytes(_cfg(n, 3))["x_eos"] == 24 * n ** 3


def test_l2_note_follows_the_field_size():
    assert "no flush needed" in bench.bench_config({**_cfg(512, 3), "shape": (512, 512, 512)}, 1)["l2"]
    assert "fit in the 129 MB L2" in bench.bench_config({**_cfg(128, 3), "shape": (128, 128, 128)}, 1)["l2"]


def test_clock_record_uses_the_timed_region(tmp_path):
    """The clocks object summarises the nvidia-smi samples taken while the
    timed steps ran (median SM clock under load, throttle reasons seen)."""
    import datetime
    import time
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.f = open(tmp_path / "clocks.csv", "w+")
    now = time.time()
    for k in range(10):
        ts = datetime.datetime.fromtimestamp(now + 0.05 * k).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        busy = 3 <= k <= 6
        c.f.write("%s, 0, %d, 2070, %.1f, 0x0, Not Active, Not Active, Not Active, %s\n"
                  % (ts, 2070 if busy else 1500, 800.0 if busy else 200.0, "Active" if k == 5 else "Not Active"))
    c.f.flush()

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass
    c.p = _Proc()
    c.region(now + 0.14, now + 0.31)
    out = c.stop()
    assert out["samples"] == 10 and out["samples_in_timed_region"] == 4
    assert out["sm_mhz"] == 2070.0 and out["power_w_max"] == 800.0
    assert out["reasons"] == ["sw_power_cap"]
