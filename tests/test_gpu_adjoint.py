"""GPU adjoint (kwgb_adjoint) against the FP64 oracle adjoint (lossless and
absorbing media; cubic grids and thin grids with 256- and 1024-point z
lines; the float16- and bfloat16-split forms), checkpoint invariance
(including every step kept), the autograd
wrapper against central finite differences, and its forward-only and
deferred-backward semantics.

Tolerances: objective J 1e-3 relative; per-sample gradients dJ/ds relative
L2 2e-3 against the oracle adjoint; phase gradients 1e-2 against FP32
central differences with h = 1e-3 rad."""

import numpy as np
import pytest

from helpers import rel_l2
from oracle import adjoint as oadj
from paper_1408_4675_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kw():
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    return kwgb


def _problem(n=64, steps=80):
    cfg = inputs.make_config(5, n=n, n_steps=steps)
    # keep the elements that received voxels on this coarse grid
    keep = [i for i, e in enumerate(cfg["elements"]) if len(e) > 0][:24]
    cfg["elements"] = [cfg["elements"][i] for i in keep]
    cfg["phases"] = cfg["phases"][keep]
    cfg["amps"] = np.full(len(keep), 2e6)
    return cfg


def _oracle_grads(cfg, steps):
    from helpers import oracle_from_config
    c = dict(cfg)
    t = (np.arange(steps) + 0.5) * cfg["dt"]
    c["sources"] = [(e, a * np.sin(2 * np.pi * cfg["freq"] * t + ph))
                    for e, a, ph in zip(cfg["elements"], cfg["amps"], cfg["phases"])]
    c["sensors"] = []
    sim, _ = oracle_from_config(c)
    value, dJdp = oadj.mean_abs_pressure(cfg["focal"], steps)
    rec = oadj.forward_record(sim, steps)
    J = value(rec)
    grads = oadj.backward(sim, rec, dJdp)
    return J, [g.sum(axis=0) for g in grads]


def test_adjoint_matches_oracle(kw):
    from paper_1408_4675_gb300.autograd import FocalProblem
    steps = 80
    cfg = _problem(steps=steps)
    prob = FocalProblem(cfg, n_steps=steps, checkpoint_every=25)
    J, dphi, damp, g = prob.value_and_grad(cfg["phases"], cfg["amps"])
    Jo, go = _oracle_grads(cfg, steps)
    assert abs(J - Jo) <= 1e-3 * abs(Jo), (J, Jo)
    G = np.stack([x[0] for x in g])
    Go = np.stack(go)
    assert rel_l2(G, Go) <= 2e-3, rel_l2(G, Go)


def test_adjoint_absorbing_matches_oracle(kw):
    """Absorbing, heterogeneous alpha0 (Eq. 8 run backwards through the
    k^{y-2} / k^{y-1} operators) against the oracle adjoint."""
    from paper_1408_4675_gb300.autograd import FocalProblem
    steps = 60
    cfg = _problem(steps=steps)
    cfg["flags"] = cfg["flags"] | 2
    cfg["alpha0"] = inputs.db_to_neper(inputs.smooth_random_field(cfg["shape"], 0.5, 1.5, 17, 3.0),
                                       cfg["alpha_power"])
    prob = FocalProblem(cfg, n_steps=steps, checkpoint_every=16)
    J, dphi, damp, g = prob.value_and_grad(cfg["phases"], cfg["amps"])
    Jo, go = _oracle_grads(cfg, steps)
    assert abs(J - Jo) <= 1e-3 * abs(Jo), (J, Jo)
    G = np.stack([x[0] for x in g])
    Go = np.stack(go)
    assert rel_l2(G, Go) <= 2e-3, rel_l2(G, Go)


def _line_problem(nz, steps, absorbing, ny=8):
    """A thin grid (nz x ny x 16) with long z lines: six elements of three
    points on the plane just inside the z PML, a 3^3 focal box ten cells
    beyond it, a smooth random c0 (and alpha0 when absorbing)."""
    shape = (nz, ny, 16)
    dx = 1e-4
    zs = 21
    c0 = inputs.smooth_random_field(shape, 1450.0, 1550.0, 71, 1.5)
    c_ref = float(c0.max())
    elems = [np.sort(inputs.linear_index(shape, [zs] * 3, [2 + e % 4] * 3, [3 + 2 * e, 4 + 2 * e, 5 + 2 * e]))
             for e in range(6)]
    rng = np.random.default_rng(72)
    cfg = dict(shape=shape, d=(dx, dx, dx), dt=0.3 * dx / c_ref, c_ref=c_ref, flags=1 | (2 if absorbing else 0),
               alpha_power=1.5, c0=c0, rho0=1000.0, bona=5.0,
               alpha0=inputs.db_to_neper(inputs.smooth_random_field(shape, 0.5, 1.5, 73, 1.5), 1.5)
               if absorbing else 0.0,
               p0=None, elements=elems, phases=rng.uniform(-0.2, 0.2, 6), amps=np.full(6, 2e5), freq=1e6,
               focal=inputs.box_mask(shape, (zs + 10, 4, 8), 1), n_steps=steps,
               pml_size=(2, 1, 20), pml_alpha=(2.0, 2.0, 2.0))
    cfg["sensors"] = [(cfg["focal"], 1)]
    return cfg


@pytest.mark.parametrize("nz,absorbing,k", [(256, False, 16), (1024, True, 40)])
def test_adjoint_long_z_lines_matches_oracle(kw, nz, absorbing, k):
    """The reverse step's z passes on 256- and 1024-point lines (the
    two-columns-per-thread Eq. 4a operator pass and the summing Eq. 4c pass;
    at 1024 points the absorption pass as well), with checkpoints every 16
    steps and with every step kept (k = 40 = the step count), against the
    oracle adjoint."""
    from paper_1408_4675_gb300.autograd import FocalProblem
    steps = 40
    cfg = _line_problem(nz, steps, absorbing)
    prob = FocalProblem(cfg, n_steps=steps, checkpoint_every=k)
    J, dphi, damp, g = prob.value_and_grad(cfg["phases"], cfg["amps"])
    Jo, go = _oracle_grads(cfg, steps)
    assert J > 0 and abs(J - Jo) <= 1e-3 * abs(Jo), (J, Jo)
    G = np.stack([x[0] for x in g])
    Go = np.stack(go)
    assert np.abs(Go).max() > 0
    assert rel_l2(G, Go) <= 2e-3, rel_l2(G, Go)


@pytest.mark.parametrize("form,flag,tol", [("f32", 0, 2e-3), ("f16", 8, 2e-3), ("bf16", 4, 2e-3)])
def test_adjoint_split_precision_forms_match_oracle(kw, form, flag, tol):
    """The reverse step in the float16- and bfloat16-split tensor-core forms
    beside float32: 64 x 64 x 16, absorbing, so that the y and z passes
    (including the adjoint's own z passes) run on the tcgen05 form; the
    focal box ten cells from the elements, 40 steps, so that the adjoint wave
    reaches them; every step kept.  Against the oracle adjoint (prints the
    errors with -s)."""
    from paper_1408_4675_gb300.autograd import FocalProblem
    steps = 40
    cfg = _line_problem(64, steps, True, ny=64)
    cfg["flags"] = cfg["flags"] | flag
    prob = FocalProblem(cfg, n_steps=steps, checkpoint_every=steps)
    J, dphi, damp, g = prob.value_and_grad(cfg["phases"], cfg["amps"])
    Jo, go = _oracle_grads(cfg, steps)
    G = np.stack([x[0] for x in g])
    Go = np.stack(go)
    print("ADJERR form=%s J_rel=%.3e grad_rel_l2=%.3e" % (form, abs(J - Jo) / abs(Jo), rel_l2(G, Go)))
    assert abs(J - Jo) <= 1e-3 * abs(Jo), (J, Jo)
    assert rel_l2(G, Go) <= tol, rel_l2(G, Go)


def test_checkpoint_interval_does_not_change_the_gradient(kw):
    """Checkpoints every 7 steps (ragged last segment) and every 20 steps
    (segments replayed from one captured graph) recompute the kept fields;
    an interval of at least the step count (40, 100) keeps every step's
    fields from the forward run itself.  All four give the same objective
    and gradient, bit for bit."""
    from paper_1408_4675_gb300.autograd import FocalProblem
    cfg = _problem(n=32, steps=40)
    res = [FocalProblem(cfg, n_steps=40, checkpoint_every=k).value_and_grad(cfg["phases"], cfg["amps"])
           for k in (40, 7, 20, 100)]
    a = res[0]
    for b in res[1:]:
        assert a[0] == b[0]
        np.testing.assert_array_equal(np.stack([x[0] for x in a[3]]), np.stack([x[0] for x in b[3]]))


def test_autograd_function_matches_finite_differences(kw):
    import torch
    from paper_1408_4675_gb300.autograd import FocalProblem, SimulateFocal
    cfg = _problem(n=32, steps=60)
    prob = FocalProblem(cfg, n_steps=60, checkpoint_every=20)
    ph = torch.tensor(cfg["phases"], dtype=torch.float64, requires_grad=True)
    am = torch.tensor(cfg["amps"], dtype=torch.float64, requires_grad=True)
    J = SimulateFocal.apply(ph, am, prob)
    J.backward()
    h = 1e-3
    for e in (0, len(cfg["phases"]) // 2):
        d = np.zeros(len(cfg["phases"]))
        d[e] = h
        fd = (prob.objective(cfg["phases"] + d, cfg["amps"]) - prob.objective(cfg["phases"] - d, cfg["amps"])) / (2 * h)
        assert abs(fd - ph.grad[e].item()) <= 1e-2 * max(abs(fd), 1e-3 * abs(J.item())), (e, fd, ph.grad[e].item())


def test_forward_only_and_deferred_backward(kw):
    """SimulateFocal without a gradient makes one forward run (J from the
    device-side objective samples, no checkpoints) and equals J taken by
    stepping and reading p; with a gradient, forward() keeps the run's
    checkpoints and backward() runs its reverse pass, which matches
    value_and_grad bitwise."""
    import torch
    from paper_1408_4675_gb300.autograd import FocalProblem, SimulateFocal
    steps = 40
    cfg = _problem(n=32, steps=steps)
    prob = FocalProblem(cfg, n_steps=steps, checkpoint_every=10)
    sim = prob.simulation(cfg["phases"], cfg["amps"])
    total = 0.0
    for _ in range(steps):
        sim.step(1)
        total += np.abs(sim.read_field("p").reshape(-1)[prob.focal].astype(np.float64)).sum()
    sim.close()
    J_hand = total / (len(prob.focal) * steps)
    ph = torch.tensor(cfg["phases"], dtype=torch.float64)
    am = torch.tensor(cfg["amps"], dtype=torch.float64)
    J0 = SimulateFocal.apply(ph, am, prob)
    assert abs(J0.item() - J_hand) <= 1e-5 * J_hand, (J0.item(), J_hand)   # p read back through a C2R
    ph.requires_grad_()
    am.requires_grad_()
    J1 = SimulateFocal.apply(ph, am, prob)
    assert J1.item() == J0.item()
    J1.backward()
    J2, dphi, damp, _ = prob.value_and_grad(cfg["phases"], cfg["amps"])
    assert J2 == J1.item()
    np.testing.assert_array_equal(ph.grad.numpy(), dphi)
    np.testing.assert_array_equal(am.grad.numpy(), damp)


def test_default_interval_keeps_every_step_when_it_fits(kw):
    """FocalProblem without an interval keeps every step's fields when they
    fit in half the free device memory (a small grid), and gives the same
    gradient as checkpoints every 10 steps."""
    from paper_1408_4675_gb300.autograd import FocalProblem
    cfg = _problem(n=32, steps=40)
    a = FocalProblem(cfg, n_steps=40)
    assert a.checkpoint_every == 40
    ra = a.value_and_grad(cfg["phases"], cfg["amps"])
    rb = FocalProblem(cfg, n_steps=40, checkpoint_every=10).value_and_grad(cfg["phases"], cfg["amps"])
    assert ra[0] == rb[0]
    np.testing.assert_array_equal(ra[1], rb[1])
