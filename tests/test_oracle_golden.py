"""Golden facts printed in the paper (fixtures under tests/golden/)."""

import os

import numpy as np

import oracle
from oracle import kspace as ks

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _counts():
    out = {}
    with open(os.path.join(GOLDEN, "fft_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, fw, inv = line.split()
                out[name] = (int(fw), int(inv))
    return out


def test_fft_count_per_step(monkeypatch):
    counts = _counts()
    for name, flags in (("nonlinear_absorbing", oracle.NONLINEAR | oracle.ABSORBING),
                        ("linear_lossless", 0)):
        g = oracle.Grid(8, 8, 8, 1e-4, 1e-4, 1e-4, 2e-8, 1500.0, flags=flags, alpha_power=1.1)
        sim = oracle.Simulation(g)
        sim.set_medium(1500.0, 1000.0, 5.0, 1e-10)
        sim.set_initial_pressure(np.ones(g.shape))
        seen = {"fw": 0, "inv": 0}
        ft, ift = ks._ft, ks._ift_real

        def cft(a):
            seen["fw"] += 1
            return ft(a)

        def cift(a):
            seen["inv"] += 1
            return ift(a)
        monkeypatch.setattr(ks, "_ft", cft)
        monkeypatch.setattr(ks, "_ift_real", cift)
        sim.step(1)
        monkeypatch.setattr(ks, "_ft", ft)
        monkeypatch.setattr(ks, "_ift_real", ift)
        assert (seen["fw"], seen["inv"]) == counts[name], name
