"""Shared test helpers: build the oracle from the same config dictionary the
CUDA path gets, and the error metrics of the parity tests."""

import numpy as np

import oracle


def oracle_from_config(cfg):
    nz, ny, nx = cfg["shape"]
    dx, dy, dz = cfg["d"]
    g = oracle.Grid(nx, ny, nz, dx, dy, dz, cfg["dt"], cfg["c_ref"], cfg["pml_size"],
                    cfg["pml_alpha"], cfg["flags"], cfg["alpha_power"])
    sim = oracle.Simulation(g)
    # the CUDA path stores the medium in float32; give the oracle the same values
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    sim.set_medium(f32(cfg["c0"]), f32(cfg["rho0"]), f32(cfg["bona"]), f32(cfg["alpha0"]))
    if cfg.get("p0") is not None:
        sim.set_initial_pressure(f32(cfg["p0"]))
    for src in cfg["sources"]:                     # (idx, signal) or (idx, signal, mode)
        sim.add_source(src[0], f32(src[1]), *src[2:])
    ids = [sim.add_sensor(idx, rec) for idx, rec in cfg["sensors"]]
    return sim, ids


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def linf(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))
