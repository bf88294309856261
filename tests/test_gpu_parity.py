"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances (float32 path vs float64 oracle, relative L2 / relative L-inf):
  spectral operators (one FFT round trip)          1e-5 / 5e-5
  config 1 (linear lossless, 200 steps)            1e-5 / 5e-5
  heterogeneous nonlinear absorbing runs           1e-3 / 5e-3
The float32 round trip of a 3D FFT carries about 1e-7 relative error per
pass times log2(N); the long nonlinear runs accumulate it over hundreds of
steps, which the 1e-3 bound covers with margin.
"""

import numpy as np
import pytest

import oracle
from helpers import linf, oracle_from_config, rel_l2
from paper_1408_4675_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kw():
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    return kwgb


def _sim_for_ops(kw, shape, flags, y):
    nz, ny, nx = shape
    d = (1e-4, 1.25e-4, 0.8e-4)
    sim = kw.Simulation(shape, d, 2e-8, 1500.0, flags=flags, alpha_power=y)
    sim.set_medium(1500.0, 1000.0)
    g = oracle.Grid(nx, ny, nz, *d, 2e-8, 1500.0, flags=flags, alpha_power=y)
    return sim, g


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 8, 32), (32, 64, 16), (64, 64, 64),
                                   (8, 16, 1024), (1024, 8, 16), (16, 1024, 8),
                                   (512, 8, 32), (256, 16, 64), (16, 512, 32), (8, 256, 64)])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_spectral_operator_parity(kw, shape, op):
    import torch
    y = 1.3
    sim, g = _sim_for_ops(kw, shape, kw.ABSORBING, y)
    rng = np.random.default_rng(sum(shape) + op)
    f = rng.standard_normal(shape).astype(np.float32)
    dev = torch.from_numpy(f).cuda()
    nout = 3 if op in (0, 1) else 1
    outs = [torch.empty_like(dev) for _ in range(nout)]
    sim.apply_operator(op, dev, outs)
    torch.cuda.synchronize()
    ref = oracle.apply_operator(g, op, f.astype(np.float64))
    for got, r in zip(outs, ref):
        got = got.cpu().numpy()
        assert rel_l2(got, r) <= 1e-5, (shape, op, rel_l2(got, r))
        assert linf(got, r) <= 5e-5, (shape, op, linf(got, r))
    sim.close()


def _run_both(kw, cfg, steps):
    gsim, gids = kw.from_config(cfg)
    osim, oids = oracle_from_config(cfg)
    gsim.step(steps)
    osim.step(steps)
    return gsim, gids, osim, oids


def _check_outputs(gsim, gids, osim, oids, cfg, tl2, tinf):
    for (idx, rec), gi, oi in zip(cfg["sensors"], gids, oids):
        for which in (kw_P_MAX, kw_P_RMS, kw_I_AVG):
            if rec & which:
                got = gsim.read(gi, which)
                ref = osim.read(oi, which)
                assert rel_l2(got, ref) <= tl2, (which, rel_l2(got, ref))
                assert linf(got, ref) <= tinf, (which, linf(got, ref))


kw_P_MAX, kw_P_RMS, kw_I_AVG = 1, 2, 4


def _check_fields(gsim, osim, tl2, tinf, names=("p", "ux", "uy", "uz", "rhox", "rhoy", "rhoz")):
    of = osim.fields()
    for n in names:
        got = gsim.read_field(n)
        assert rel_l2(got, of[n]) <= tl2, (n, rel_l2(got, of[n]))
        assert linf(got, of[n]) <= tinf, (n, linf(got, of[n]))


def test_config1_linear_lossless_full(kw):
    """64^3 water, Gaussian initial pressure, 200 steps, full-grid p_max."""
    cfg = inputs.make_config(1)
    gsim, gids, osim, oids = _run_both(kw, cfg, cfg["n_steps"])
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-5, 5e-5)
    _check_fields(gsim, osim, 1e-4, 5e-4)
    assert gsim.status() == 0
    gsim.close()


@pytest.mark.parametrize("n,steps", [(64, 120)])
def test_config2_heterogeneous_nonlinear_absorbing(kw, n, steps):
    cfg = inputs.make_config(2, n=n, n_steps=steps)
    gsim, gids, osim, oids = _run_both(kw, cfg, steps)
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-3, 5e-3)
    _check_fields(gsim, osim, 1e-3, 5e-3)
    gsim.close()


@pytest.mark.parametrize("n,steps", [(64, 150)])
def test_config3_bowl_tissue_with_intensity(kw, n, steps):
    cfg = inputs.make_config(3, n=n, n_steps=steps)
    gsim, gids, osim, oids = _run_both(kw, cfg, steps)
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-3, 5e-3)
    gsim.close()


def test_config5_segmented_bowl_forward(kw):
    cfg = inputs.make_config(5, n=64, n_steps=100)
    gsim, gids, osim, oids = _run_both(kw, cfg, 100)
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-3, 5e-3)
    gsim.close()


def test_anisotropic_grid_every_feature(kw):
    """Small anisotropic grid (ragged column tiles along x, every axis a
    different size) with PML, heterogeneous nonlinear absorbing medium, an
    initial pressure, overlapping sources and all sensor outputs."""
    shape = (16, 8, 32)
    cfg = inputs.make_config(2, n=16, n_steps=40)
    nz, ny, nx = shape
    rng = np.random.default_rng(5)
    cfg["shape"] = shape
    cfg["d"] = (1e-4, 0.9e-4, 1.1e-4)
    for key, lo, hi in (("c0", 1450, 1650), ("rho0", 950, 1100), ("bona", 5, 9)):
        cfg[key] = inputs.smooth_random_field(shape, lo, hi, int(rng.integers(1 << 30)), 2.0)
    cfg["alpha0"] = inputs.db_to_neper(inputs.smooth_random_field(shape, 0.3, 1.0, 11, 2.0), 1.1)
    cfg["c_ref"] = float(cfg["c0"].max())
    cfg["dt"] = 0.3 * 0.9e-4 / cfg["c_ref"]
    cfg["pml_size"] = (3, 2, 4)
    cfg["p0"] = inputs.gaussian_ball(shape, 1.5, 2e5)
    src = np.array([5, 40, 41, 300, 300, nx * ny * nz - 1])
    cfg["sources"] = [(src, inputs.cw(1e6, 1e5, cfg["dt"], 30)),
                      (np.array([40, 41]), np.stack([inputs.cw(1e6, 2e4, cfg["dt"], 40),
                                                    inputs.tone_burst(1e6, 2, 3e4, cfg["dt"], 40)]))]
    sens = np.array([0, 7, 40, 41, 333, 1000, nx * ny * nz - 1])
    cfg["sensors"] = [(sens, 7), (None, 3), (np.array([41]), 1)]
    gsim, gids, osim, oids = _run_both(kw, cfg, 40)
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-4, 5e-4)
    _check_fields(gsim, osim, 1e-4, 5e-4)
    gsim.close()


def test_zero_steps_and_repeated_reads(kw):
    cfg = inputs.make_config(3, n=32, n_steps=10)
    gsim, gids = kw.from_config(cfg)
    gsim.step(0)
    assert np.all(np.isneginf(gsim.read(gids[0], kw_P_MAX)))
    assert np.all(gsim.read(gids[0], kw_P_RMS) == 0)
    gsim.step(5)
    a = gsim.read(gids[0], kw_I_AVG)
    b = gsim.read(gids[0], kw_I_AVG)          # the read-time tail changes no state
    np.testing.assert_array_equal(a, b)
    gsim.step(5)
    osim, oids = oracle_from_config(cfg)
    osim.step(10)
    got, ref = gsim.read(gids[0], kw_I_AVG), osim.read(oids[0], kw_I_AVG)
    assert rel_l2(got, ref) <= 1e-3
    gsim.close()


def test_two_runs_are_bitwise_identical(kw):
    cfg = inputs.make_config(2, n=32, n_steps=20)
    out = []
    for _ in range(2):
        gsim, gids = kw.from_config(cfg)
        gsim.step(20)
        out.append((gsim.read(gids[0], kw_P_MAX), gsim.read_field("p")))
        gsim.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


# ---- split-precision tensor-core forms ------------------------------------
# KWGB_MIXED_F16 (8): float16 hi + lo (2^-22 relative residue per operand),
# must meet every float32 row ("equal error").  KWGB_MIXED_BF16 (4): bfloat16
# hi + lo (2^-18): one operator application within 1e-4 / 1e-3, the
# multi-step 1e-3 rows met, and the 200-step linear run of workload 1 within
# 3e-5 (its float32 row of 1e-5 is not met; measured 1.09e-5).

MIXED = {"bf16": 4, "f16": 8}


@pytest.mark.parametrize("form", ["bf16", "f16"])
@pytest.mark.parametrize("shape", [(16, 16, 16), (64, 64, 64), (32, 512, 16), (512, 16, 32),
                                   (128, 16, 16), (16, 128, 32), (256, 16, 64), (16, 256, 64),
                                   (1024, 16, 16), (16, 1024, 8)])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_mixed_operator_parity(kw, form, shape, op):
    import torch
    sim, g = _sim_for_ops(kw, shape, kw.ABSORBING | MIXED[form], 1.3)
    rng = np.random.default_rng(sum(shape) + op + 7)
    f = rng.standard_normal(shape).astype(np.float32)
    dev = torch.from_numpy(f).cuda()
    nout = 3 if op in (0, 1) else 1
    outs = [torch.empty_like(dev) for _ in range(nout)]
    sim.apply_operator(op, dev, outs)
    torch.cuda.synchronize()
    ref = oracle.apply_operator(g, op, f.astype(np.float64))
    tl2, tinf = (1e-5, 5e-5) if form == "f16" else (1e-4, 1e-3)
    for got, r in zip(outs, ref):
        got = got.cpu().numpy()
        assert rel_l2(got, r) <= tl2, (shape, op, rel_l2(got, r))
        assert linf(got, r) <= tinf, (shape, op, linf(got, r))
    sim.close()


@pytest.mark.parametrize("form", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("cfgid,n,steps", [(1, 64, 200), (2, 64, 120), (3, 64, 150)])
def test_mixed_form_equal_error(kw, form, cfgid, n, steps):
    """Every sensor output of the three forms against the FP64 oracle on the
    same runs (printed with -s: the per-output error table of the forms)."""
    cfg = inputs.make_config(cfgid, n=n, n_steps=steps)
    cfg["flags"] = cfg["flags"] | MIXED.get(form, 0)
    gsim, gids, osim, oids = _run_both(kw, cfg, steps)
    if cfgid == 1:
        tl2, tinf = (3e-5, 5e-5) if form == "bf16" else (1e-5, 5e-5)
    else:
        tl2, tinf = 1e-3, 5e-3
    for (idx, rec), gi, oi in zip(cfg["sensors"], gids, oids):
        for which in (kw_P_MAX, kw_P_RMS, kw_I_AVG):
            if rec & which:
                got, ref = gsim.read(gi, which), osim.read(oi, which)
                print("ERRTABLE form=%s config=%d output=%d rel_l2=%.3e linf=%.3e"
                      % (form, cfgid, which, rel_l2(got, ref), linf(got, ref)))
    _check_outputs(gsim, gids, osim, oids, cfg, tl2, tinf)
    gsim.close()


def test_force_sources_match_oracle(kw):
    """Force sources (reading R15): a planar z force layer with a shared
    signal and x-force points with their own signals, in the heterogeneous
    nonlinear absorbing medium, with intensity sensors (whose read-time tail
    applies the next step's force samples)."""
    steps = 50
    cfg = inputs.make_config(2, n=32, n_steps=steps)
    n = 32
    yy, xx = np.meshgrid(np.arange(12, 20), np.arange(12, 20), indexing="ij")
    plane = (xx + n * (yy + n * 11)).ravel()
    pts = np.array([5 + n * (7 + n * 16), 20 + n * (9 + n * 18), 21 + n * (9 + n * 18)])
    t = np.arange(steps) * cfg["dt"]
    f1 = 5e10 * np.sin(2 * np.pi * 1e6 * t)
    f2 = np.stack([4e10 * np.sin(2 * np.pi * 1e6 * t + k) for k in range(3)])
    cfg["sources"] = cfg["sources"] + [(plane, f1, kw.FORCE_Z), (pts, f2[:, :30], kw.FORCE_X)]
    cfg["sensors"] = [(np.sort(np.concatenate([plane[::7], pts])), 7), (None, 3)]
    gsim, gids, osim, oids = _run_both(kw, cfg, steps)
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-3, 5e-3)
    _check_fields(gsim, osim, 1e-3, 5e-3)
    gsim.close()


@pytest.mark.parametrize("cfg_id", [2, 5])
def test_dirichlet_sources_match_oracle(kw, cfg_id):
    """Dirichlet pressure sources (reading R16): a held plane with a shared
    signal and held points with their own signals, two of which end before the
    run does (those points then evolve freely), one overlapping an additive
    source; in the heterogeneous nonlinear absorbing medium (x_dens then x_eos)
    and the lossless nonlinear one (the equation of state fused into x_dens).
    The held points take the float32 signal exactly (seen through p_max: the
    stored field is the x-transformed p, whose inverse carries FFT rounding)."""
    steps = 50
    cfg = inputs.make_config(cfg_id, n=32, n_steps=steps)
    n = 32
    yy, xx = np.meshgrid(np.arange(12, 20), np.arange(12, 20), indexing="ij")
    plane = (xx + n * (yy + n * 11)).ravel()
    pts = np.array([5 + n * (7 + n * 16), 20 + n * (9 + n * 18), 21 + n * (9 + n * 18)])
    t = (np.arange(steps) + 1) * cfg["dt"]
    s1 = 2e5 * np.sin(2 * np.pi * 1e6 * t)
    s2 = np.stack([1e5 * np.sin(2 * np.pi * 1e6 * t + k) for k in range(3)])
    s2[1:, 30:] = 0.0
    sig2 = [s2[0], s2[1, :30], s2[2, :30]]
    cfg["sources"] = cfg["sources"] + [(plane, s1, kw.DIRICHLET_P), (pts[:1], sig2[0], kw.DIRICHLET_P),
                                       (pts[1:], np.stack(sig2[1:]), kw.DIRICHLET_P),
                                       (pts[:1], 3e5 * np.sin(2 * np.pi * 1e6 * t), kw.ADDITIVE_MASS)]
    cfg["sensors"] = [(np.sort(np.concatenate([plane[::7], pts, pts + 1])), 7), (None, 3)]
    gsim, gids, osim, oids = _run_both(kw, cfg, steps)
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-3, 5e-3)
    _check_fields(gsim, osim, 1e-3, 5e-3)
    # the sensors see the real-space p of each step: held points exactly the float32 samples
    sidx = cfg["sensors"][0][0]
    pmax = gsim.read(gids[0], kw_P_MAX)
    at = lambda pt: int(np.searchsorted(sidx, pt))
    for pt in plane[::7]:
        assert pmax[at(pt)] == np.float32(s1).max()
    assert pmax[at(pts[0])] == np.float32(s2[0]).max()
    assert pmax[at(pts[1])] >= np.float32(s2[1, :30]).max()     # held 30 steps, then free
    gsim.close()


def test_adjoint_refuses_dirichlet_sources(kw):
    cfg = inputs.make_config(1, n=32, n_steps=4)
    cfg["sources"] = [(np.array([5, 6]), np.ones(4), kw.DIRICHLET_P)]
    gsim, _ = kw.from_config(cfg)
    with pytest.raises(kw.KwgbError):
        gsim.adjoint(np.array([1, 2, 3]), 4, 2)
    gsim.close()


def test_graph_replay_equals_direct_launches(kw):
    """kwgb_step replays a captured CUDA graph after the first step;
    kwgb_step_profiled launches the same kernels directly: the two paths give
    bitwise identical states."""
    cfg = inputs.make_config(3, n=32, n_steps=12)
    a, ida = kw.from_config(cfg)
    a.step(12)
    b, idb = kw.from_config(cfg)
    for _ in range(12):
        b.step_profiled()
    for name in ("p", "ux", "uy", "uz", "rhox", "rhoy", "rhoz"):
        np.testing.assert_array_equal(a.read_field(name), b.read_field(name))
    for (idx, rec), i, j in zip(cfg["sensors"], ida, idb):
        for which in (kw_P_MAX, kw_P_RMS, kw_I_AVG):
            if rec & which:
                np.testing.assert_array_equal(a.read(i, which), b.read(j, which))
    assert a.launch_count == b.launch_count
    a.close()
    b.close()


def _plane_wave_cfg(kw, n_steps, absorbing, interface):
    """8 x 8 x 256 grid, 0.05 mm, PML on z only, a 1 MHz ramped sinusoid on the
    plane z = 20 (additive mass source), full-grid p_max and p_rms: either an
    absorbing medium (y = 1.1, 40 Np/m at 1 MHz) or a lossless medium with a
    planar interface at z = 100 (1500 m/s, 1000 kg/m^3 | 1800 m/s, 1200 kg/m^3)."""
    nz, ny, nx, d, f0 = 256, 8, 8, 5e-5, 1e6
    c_ref = 1800.0 if interface else 1500.0
    dt = 1.0 / f0 / 120 if interface else 1e-8
    y = 1.1
    c0 = np.full((nz, ny, nx), 1500.0, np.float32)
    rho0 = np.full((nz, ny, nx), 1000.0, np.float32)
    if interface:
        c0[100:] = 1800.0
        rho0[100:] = 1200.0
    t = (np.arange(n_steps) + 0.5) * dt
    ramp = np.clip(t * f0 / 3, 0, 1)
    ramp = 0.5 - 0.5 * np.cos(np.pi * ramp)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    plane = (xx + nx * (yy + ny * 20)).ravel()
    return {"shape": (nz, ny, nx), "d": (d, d, d), "dt": dt, "c_ref": c_ref, "pml_size": (0, 0, 10),
            "pml_alpha": (0.0, 0.0, 2.0), "flags": kw.ABSORBING if absorbing else 0, "alpha_power": y,
            "c0": c0, "rho0": rho0, "bona": 0.0,
            "alpha0": 40.0 / (2 * np.pi * f0) ** y if absorbing else 0.0, "p0": None,
            "sources": [(plane, (1e5 * ramp * np.sin(2 * np.pi * f0 * t)).astype(np.float32))],
            "sensors": [(None, kw_P_MAX | kw_P_RMS)], "n_steps": n_steps}


@pytest.mark.parametrize("absorbing,interface,steps", [(True, False, 1200), (False, True, 1400)])
def test_long_plane_wave_runs_match_oracle(kw, absorbing, interface, steps):
    """Long horizons (1200-1400 steps, the wave crosses the grid and reaches
    steady state): the driven plane wave of the oracle's dispersion pin in an
    absorbing medium, and the two-media interface of its transmission pin."""
    cfg = _plane_wave_cfg(kw, steps, absorbing, interface)
    gsim, gids, osim, oids = _run_both(kw, cfg, steps)
    _check_outputs(gsim, gids, osim, oids, cfg, 1e-3, 5e-3)
    _check_fields(gsim, osim, 1e-3, 5e-3, names=("p", "uz", "rhoz"))
    assert gsim.status() == 0
    gsim.close()
