"""Writes the FP64 oracle's expected outputs for the GPU parity tests at the
workloads' stated sizes (tests/test_gpu_stated_sizes.py).

Only the oracle (oracle/, through tests/helpers.oracle_from_config) and the
input generators run here; nothing comes from the CUDA path.  Each workload's
file holds a seeded sample of every sensor output (uniform random points plus
the points of largest magnitude, where the maximum error tends to sit), the
full-grid norms of each output, and the run's parameters:

  config2_256.npz  256^3 smooth random heterogeneous, nonlinear, absorbing
                   medium, planar tone burst, full-grid p_max and p_rms after
                   300 and 1500 steps (the recipe's whole horizon);
  config5_128.npz  128^3 segmented bowl (256 elements), 600 steps: the focal
                   objective J = mean |p|, p_max on the 5^3 focal box, and the
                   adjoint's dJ/ds for every element and sample;
  config3_512.npz  512^3 HIFU bowl into layered tissue, the first STEPS3 =
                   300 steps (about an hour of FP64 oracle on 16 host cores):
                   the xz-plane and focal-box sensors (p_max, p_rms,
                   intensity) and the p, u_z, rho_z fields at sampled points.

Usage: python tests/golden/make_fullsize_golden.py {2|5|3} [out_dir]
(config 5 needs about 75 GB of host memory, config 3 about 60 GB).
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from helpers import oracle_from_config          # noqa: E402
from oracle import adjoint as oadj               # noqa: E402
from paper_1408_4675_gb300 import inputs         # noqa: E402

P_MAX, P_RMS, I_AVG = 1, 2, 4
STEPS2 = (300, 1500)
STEPS3 = 300
SEED = 1408


def sample_points(values, n_uniform, n_top, seed):
    """Seeded uniform sample of the indices of `values` plus the n_top indices
    of largest magnitude, sorted and unique."""
    m = values.size
    rng = np.random.default_rng(seed)
    uni = rng.choice(m, size=min(n_uniform, m), replace=False)
    top = np.argpartition(np.abs(values), m - min(n_top, m))[m - min(n_top, m):]
    return np.unique(np.concatenate([uni, top])).astype(np.int64)


def _compact(res):
    """Sample indices as int32 and sampled values as float32 (the parity
    tolerances are 1e-3 and above); norms and short arrays stay float64."""
    out = {}
    for k, v in res.items():
        v = np.asarray(v)
        if v.dtype == np.int64 and v.size > 1:
            v = v.astype(np.int32)
        elif v.dtype == np.float64 and v.size > 1024:
            v = v.astype(np.float32)
        out[k] = v
    return out


def _norms(prefix, v):
    return {prefix + "_l2": np.linalg.norm(v), prefix + "_absmax": np.abs(v).max()}


def config2(out):
    cfg = inputs.make_config(2, n_steps=STEPS2[-1])
    sim, ids = oracle_from_config(cfg)
    res = dict(steps=np.array(STEPS2), n=256)
    done = 0
    t0 = time.time()
    for s in STEPS2:
        sim.step(s - done)
        done = s
        pmax = sim.read(ids[0], P_MAX)
        prms = sim.read(ids[0], P_RMS)
        idx = sample_points(pmax, 1 << 16, 4096, SEED + s)
        idx = np.union1d(idx, sample_points(prms, 0, 4096, 0))
        res["idx_%d" % s] = idx
        res["p_max_%d" % s] = pmax[idx]
        res["p_rms_%d" % s] = prms[idx]
        for k, v in {**_norms("p_max_%d" % s, pmax), **_norms("p_rms_%d" % s, prms)}.items():
            res[k] = np.array(v)
        print("config 2: %d steps, %.0f s" % (s, time.time() - t0), flush=True)
    np.savez_compressed(os.path.join(out, "config2_256.npz"), **_compact(res))


def config5(out):
    cfg = inputs.make_config(5)
    nt = cfg["n_steps"]
    c = dict(cfg)
    t = (np.arange(nt) + 0.5) * cfg["dt"]
    c["sources"] = [(e, a * np.sin(2 * np.pi * cfg["freq"] * t + ph))
                    for e, a, ph in zip(cfg["elements"], cfg["amps"], cfg["phases"])]
    sim, ids = oracle_from_config(c)
    value, dJdp = oadj.mean_abs_pressure(cfg["focal"], nt)
    t0 = time.time()
    rec = oadj.forward_record(sim, nt)
    J = value(rec)
    pmax = sim.read(ids[0], P_MAX)
    print("config 5: forward %d steps, %.0f s, J = %.6g" % (nt, time.time() - t0, J), flush=True)
    grads = oadj.backward(sim, rec, dJdp)
    G = np.stack([g.sum(axis=0) for g in grads])           # (elements, n_t)
    print("config 5: adjoint, %.0f s" % (time.time() - t0), flush=True)
    np.savez_compressed(os.path.join(out, "config5_128.npz"),
                        **_compact(dict(J=np.array(J), p_max=pmax, dJds=G, steps=np.array(nt), n=128)))


def config3(out):
    cfg = inputs.make_config(3, n_steps=STEPS3 + 4)
    sim, ids = oracle_from_config(cfg)
    t0 = time.time()
    for k in range(STEPS3):
        sim.step(1)
        if (k + 1) % 25 == 0 or k == 0:
            print("config 3: step %d, %.0f s" % (k + 1, time.time() - t0), flush=True)
    res = dict(steps=np.array(STEPS3), n=512)
    names = ("focal", "plane")
    for sid, (idx, rec), name in zip(ids, cfg["sensors"], names):
        for which, tag in ((P_MAX, "p_max"), (P_RMS, "p_rms")):
            v = sim.read(sid, which)
            pts = sample_points(v, 1 << 15, 4096, SEED + which)
            res["%s_%s_idx" % (name, tag)] = pts
            res["%s_%s" % (name, tag)] = v[pts]
            for k2, v2 in _norms("%s_%s" % (name, tag), v).items():
                res[k2] = np.array(v2)
        if rec & I_AVG:
            v = sim.read(sid, I_AVG)                          # (3, points)
            pts = sample_points(v[2], 1 << 15, 4096, SEED + 4)
            res["%s_I_idx" % name] = pts
            res["%s_I" % name] = v[:, pts]
            for k2, v2 in _norms("%s_I" % name, v).items():
                res[k2] = np.array(v2)
    f = sim.fields()
    for name in ("p", "uz", "rhoz"):
        v = f[name].reshape(-1)
        pts = sample_points(v, 1 << 15, 4096, SEED + len(name))
        res["field_%s_idx" % name] = pts
        res["field_%s" % name] = v[pts]
        for k2, v2 in _norms("field_%s" % name, v).items():
            res[k2] = np.array(v2)
    np.savez_compressed(os.path.join(out, "config3_512.npz"), **_compact(res))


if __name__ == "__main__":
    which = sys.argv[1]
    out = sys.argv[2] if len(sys.argv) > 2 else HERE
    {"2": config2, "5": config5, "3": config3}[which](out)
