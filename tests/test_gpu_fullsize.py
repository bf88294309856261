"""Parity at the benchmark's sizes and launch configurations.

* 512^3 HIFU workload (the benchmark line): two steps against the FP64
  oracle, every field element by element and the sensor outputs.
* 1024-point x rows: the fused x kernels for nx = 1024 (the 1024^3 workload's
  instantiation) on a thin 8 x 8 x 1024 grid against the oracle.
* 1024^3: the oracle does not fit in reasonable time, so a property that holds
  at any size is checked on the GPU fields: the discrete energy
  sum p^2/(2 rho0 c0^2) + 1/2 sum rho0_sg u^{n-1/2} u^{n+1/2} of a lossless
  linear run without PML is exactly conserved by the scheme (pinned on the
  oracle in tests/test_oracle_pins.py)."""

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


def test_bench_workload_512_two_steps(kw):
    """Float32 form, float16-split (equal error) and bfloat16-split tensor-core
    forms of the benchmark workload against one FP64 oracle run."""
    steps = 2
    cfg = inputs.make_config(3, n_steps=steps + 4)
    osim, oids = oracle_from_config(cfg)
    osim.step(steps)
    of = osim.fields()
    for flags, tl2, tinf in ((cfg["flags"], 1e-4, 5e-4), (cfg["flags"] | 8, 1e-4, 5e-4),
                             (cfg["flags"] | 4, 1e-3, 5e-3)):
        c = dict(cfg)
        c["flags"] = flags
        gsim, gids = kw.from_config(c)
        gsim.step(steps)
        for name in ("p", "ux", "uy", "uz", "rhox", "rhoy", "rhoz"):
            got = gsim.read_field(name)
            assert rel_l2(got, of[name]) <= tl2, (flags, name, rel_l2(got, of[name]))
            assert linf(got, of[name]) <= tinf, (flags, name, linf(got, of[name]))
        for (idx, rec), gi, oi in zip(cfg["sensors"], gids, oids):
            for which in (1, 2):
                if rec & which:
                    assert rel_l2(gsim.read(gi, which), osim.read(oi, which)) <= tl2
        gsim.close()


@pytest.mark.parametrize("dirichlet", [False, True])
def test_fused_x_kernels_nx1024(kw, dirichlet):
    """Rows of 1024 reals (two-warp row teams): every fused x kernel, with the
    additive source, and in the second run Dirichlet points on the same rows
    (their instantiations of x_dens and x_eos)."""
    cfg = inputs.make_config(2, n=16, n_steps=30)
    shape = (8, 8, 1024)
    cfg["shape"] = shape
    cfg["d"] = (1e-4, 1e-4, 1e-4)
    for key, lo, hi, sd in (("c0", 1450, 1650, 1), ("rho0", 950, 1100, 2), ("bona", 5, 9, 3)):
        cfg[key] = inputs.smooth_random_field(shape, lo, hi, sd, 3.0)
    cfg["alpha0"] = inputs.db_to_neper(inputs.smooth_random_field(shape, 0.3, 1.0, 4, 3.0), 1.1)
    cfg["c_ref"] = float(cfg["c0"].max())
    cfg["dt"] = 0.3 * 1e-4 / cfg["c_ref"]
    cfg["pml_size"] = (20, 2, 2)
    cfg["p0"] = inputs.gaussian_ball(shape, 3.0, 5e5, (4, 4, 512))
    cfg["sources"] = [(np.arange(100, 900, 37) + 1024 * (8 * 4 + 3), inputs.cw(1e6, 3e5, cfg["dt"], 30))]
    if dirichlet:
        held = np.arange(120, 920, 41) + 1024 * (8 * 5 + 2)
        cfg["sources"].append((held, inputs.cw(1e6, 2e5, cfg["dt"], 25), kw.DIRICHLET_P))
    cfg["sensors"] = [(None, 3)]
    gsim, gids = kw.from_config(cfg)
    osim, oids = oracle_from_config(cfg)
    gsim.step(30)
    osim.step(30)
    of = osim.fields()
    for name in ("p", "ux", "uy", "uz", "rhox", "rhoy", "rhoz"):
        got = gsim.read_field(name)
        assert rel_l2(got, of[name]) <= 1e-4, (name, rel_l2(got, of[name]))
    assert rel_l2(gsim.read(gids[0], 1), osim.read(oids[0], 1)) <= 1e-4
    gsim.close()


def _energy(sim, p_field, c0, rho0, u_old):
    """sum p^2/(2 rho0 c0^2) + 1/2 sum rho0 u_old u_new, in float64 by z slabs"""
    e = 0.0
    u_new = [sim.read_field(n) for n in ("ux", "uy", "uz")]
    for z in range(0, p_field.shape[0], 64):
        sl = slice(z, z + 64)
        p = p_field[sl].astype(np.float64)
        c = c0[sl].astype(np.float64)
        e += float(np.sum(p * p / (2.0 * rho0 * c * c)))
        for a, b in zip(u_old, u_new):
            e += 0.5 * rho0 * float(np.sum(a[sl].astype(np.float64) * b[sl].astype(np.float64)))
    return e, u_new


def test_energy_conserved_1024(kw):
    n = 1024
    shape = (n, n, n)
    d = 1e-4
    rho0 = 1000.0
    z = np.arange(n, dtype=np.float32).reshape(n, 1, 1)
    c0 = (1500.0 + 80.0 * np.sin(2 * np.pi * z / n)).astype(np.float32) * np.ones((1, n, n), np.float32)
    c_ref = float(c0.max())
    sim = kw.Simulation(shape, (d, d, d), 0.3 * d / c_ref, c_ref)
    sim.set_medium(c0, rho0)
    cz, cy, cx = n // 2, n // 2, n // 2
    zz = np.arange(n, dtype=np.float32)
    g1 = np.exp(-((zz - cz) ** 2) / (2 * 6.0 ** 2)).astype(np.float32)
    p0 = 1e5 * g1.reshape(n, 1, 1) * g1.reshape(1, n, 1) * g1.reshape(1, 1, n)
    sim.set_initial_pressure(p0)
    del p0
    energies = []
    u_old = [sim.read_field(nm) for nm in ("ux", "uy", "uz")]
    for _ in range(3):
        p = sim.read_field("p")
        sim.step(1)
        e, u_old = _energy(sim, p, c0, rho0, u_old)
        energies.append(e)
    assert sim.status() == 0
    sim.close()
    energies = np.array(energies)
    assert np.abs(energies - energies[0]).max() <= 1e-5 * abs(energies[0]), energies
