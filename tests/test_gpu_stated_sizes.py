"""GPU parity against the FP64 oracle at the workloads' stated sizes.

The expected values (tests/golden/config*.npz) are written by
tests/golden/make_fullsize_golden.py from the oracle alone: a seeded uniform
sample of every output plus the points of largest magnitude, where the
largest errors sit, and the full-grid norms of each output.  The GPU run
computes the whole output; the errors are taken over the sampled points:

  rel L2 = ||g - o|| / ||o||,  Linf = max |g - o| / max |o|   (sampled points)

and the full-grid norm of the GPU output must match the oracle's within the
rel L2 bound (a necessary condition over every point).

* 256^3 smooth random heterogeneous, nonlinear, absorbing medium with the
  planar tone burst, 1500 steps (the recipe's whole run): full-grid p_max
  and p_rms after 300 and after 1500 steps within 1e-3 / 5e-3.
* 128^3 segmented bowl, 256 elements, 600 steps (the recipe's whole run): the
  focal objective J = mean |p| within 1e-3, focal p_max rel L2 within 1e-3,
  and the adjoint's dJ/ds of every element and sample within 2e-3 (rel L2)
  of the oracle's adjoint, checkpoints every 50 steps.
* 512^3 HIFU workload, the first 300 steps (a 512^3 step of the FP64 oracle
  takes about 12 s on 16 host cores, so the recipe's 3000 steps are out of
  reach; 300 steps take an hour): the xz-plane sensor (p_max, p_rms) and the
  p, u_z, rho_z fields within 1e-3 / 5e-3.  The focal box lies 64 mm (427
  cells) from the bowl and the wave has travelled about 90 cells: the box
  holds only the spectral precursor of the source, so its outputs (p_max,
  p_rms, intensity) are compared on the scale of the same output over the
  plane sensor, which crosses the source (intensity: on the scale
  max|p| max|u_z| of the fields): max |g - o| within 1e-4 of that scale,
  fifty times tighter than the workload's L-infinity row of 5e-3 (measured:
  5.6e-7 float32, 1.4e-5 float16 split).
"""

import os

import numpy as np
import pytest

from helpers import linf, rel_l2
from paper_1408_4675_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
P_MAX, P_RMS, I_AVG = 1, 2, 4


@pytest.fixture(scope="module")
def kw():
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    return kwgb


def _golden(name):
    return np.load(os.path.join(GOLDEN, name + ".npz"))


def _sampled(got_full, d, key, idx_key, tl2, tinf, form="f32"):
    """Errors of a full GPU output against the oracle's sampled values."""
    idx = d[idx_key].astype(np.int64)
    o = d[key].astype(np.float64)
    g = np.asarray(got_full, dtype=np.float64)
    e2, ei = rel_l2(g[..., idx], o), linf(g[..., idx], o)
    print("ERRTABLE form=%s output=%s rel_l2=%.3e linf=%.3e" % (form, key, e2, ei))
    assert e2 <= tl2 and ei <= tinf, (key, e2, ei)
    norm = float(d[key + "_l2"])
    assert abs(np.linalg.norm(g) - norm) <= tl2 * norm, (key, np.linalg.norm(g), norm)
    return e2, ei


def test_heterogeneous_256_full_horizon(kw):
    d = _golden("config2_256")
    cfg = inputs.make_config(2)
    assert cfg["shape"] == (256, 256, 256) and cfg["n_steps"] == int(d["steps"][-1])
    sim, ids = kw.from_config(cfg)
    done = 0
    for s in (int(v) for v in d["steps"]):
        sim.step(s - done)
        done = s
        for which, tag in ((P_MAX, "p_max"), (P_RMS, "p_rms")):
            _sampled(sim.read(ids[0], which), d, "%s_%d" % (tag, s), "idx_%d" % s, 1e-3, 5e-3)
    sim.close()


def test_segmented_bowl_128_forward_and_adjoint(kw):
    from paper_1408_4675_gb300.autograd import FocalProblem
    d = _golden("config5_128")
    cfg = inputs.make_config(5)
    nt = int(d["steps"])
    assert cfg["n_steps"] == nt and cfg["shape"] == (128, 128, 128)
    # forward: focal p_max through the sensor path
    sim, ids = kw.from_config(cfg)
    sim.step(nt)
    pmax = sim.read(ids[0], P_MAX)
    sim.close()
    assert rel_l2(pmax, d["p_max"]) <= 1e-3, rel_l2(pmax, d["p_max"])
    # J and dJ/ds through the adjoint
    prob = FocalProblem(cfg, n_steps=nt, checkpoint_every=50)
    J, _, _, g = prob.value_and_grad(cfg["phases"], cfg["amps"])
    Jo = float(d["J"])
    assert abs(J - Jo) <= 1e-3 * abs(Jo), (J, Jo)
    G = np.stack([x[0] for x in g])
    Go = d["dJds"].astype(np.float64)
    assert rel_l2(G, Go) <= 2e-3, rel_l2(G, Go)


@pytest.mark.parametrize("form,flag", [("f32", 0), ("f16", 8), ("bf16", 4)])
def test_hifu_512_first_300_steps(kw, form, flag):
    """The float32 form and both split-precision tensor-core forms against the
    same oracle run (errors printed with -s)."""
    d = _golden("config3_512")
    steps = int(d["steps"])
    cfg = inputs.make_config(3, n_steps=steps + 4)
    cfg["flags"] = cfg["flags"] | flag
    sim, ids = kw.from_config(cfg)
    sim.step(steps)
    focal, plane = ids
    for which, tag in ((P_MAX, "p_max"), (P_RMS, "p_rms")):
        _sampled(sim.read(plane, which), d, "plane_" + tag, "plane_%s_idx" % tag, 1e-3, 5e-3, form)
        g = sim.read(focal, which)
        idx = d["focal_%s_idx" % tag].astype(np.int64)
        scale = float(d["plane_%s_absmax" % tag])
        err = np.abs(g[idx] - d["focal_" + tag]).max() / scale
        print("ERRTABLE form=%s config=3 output=focal_%s max_err/scale=%.3e" % (form, tag, err))
        assert err <= 1e-4, (tag, err)
    # intensity p u: on the scale max|p| max|u_z| of the fields
    gi = sim.read(focal, I_AVG)
    idx = d["focal_I_idx"].astype(np.int64)
    scale = float(d["field_p_absmax"]) * float(d["field_uz_absmax"])
    err = np.abs(gi[:, idx] - d["focal_I"]).max() / scale
    print("ERRTABLE form=%s config=3 output=focal_I max_err/scale=%.3e" % (form, err))
    assert err <= 1e-4, err
    for name in ("p", "uz", "rhoz"):
        _sampled(sim.read_field(name).reshape(-1), d, "field_" + name, "field_%s_idx" % name, 1e-3, 5e-3, form)
    sim.close()
