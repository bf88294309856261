"""Pins of the oracle's adjoint: the dot-product identity of the linear model
(J is linear in the source signals, so J(s) = <dJ/ds, s> exactly) and central
finite differences of the nonlinear model."""

import numpy as np
import pytest

import oracle
from oracle import adjoint
from paper_1408_4675_gb300 import inputs


def _small_sim(flags, seed=0, shape=(10, 12, 16), pml=2):
    nz, ny, nx = shape
    d = 1e-4
    c0 = inputs.smooth_random_field(shape, 1450.0, 1600.0, seed + 1, 1.5)
    g = oracle.Grid(nx, ny, nz, d, d, d, 0.3 * d / c0.max(), c0.max(), pml_size=(pml, pml, pml),
                    pml_alpha=(2.0, 2.0, 2.0), flags=flags, alpha_power=1.3)
    sim = oracle.Simulation(g)
    sim.set_medium(c0, inputs.smooth_random_field(shape, 950.0, 1100.0, seed + 2, 1.5),
                   inputs.smooth_random_field(shape, 5.0, 9.0, seed + 3, 1.5),
                   inputs.db_to_neper(inputs.smooth_random_field(shape, 0.5, 2.0, seed + 4, 1.5), 1.3))
    return sim


@pytest.mark.parametrize("flags", [0, oracle.ABSORBING])
def test_dot_product_identity_linear(flags):
    rng = np.random.default_rng(3)
    nt = 25
    sim = _small_sim(flags)
    N = sim.p.size
    src = [np.array([40, 41, 300, 777]), np.array([1000, 1234])]
    sigs = [rng.standard_normal((len(i), nt)) for i in src]
    for i, s in zip(src, sigs):
        sim.add_source(i, s)
    obs = np.array([5, 99, 500, 1500, N - 3])
    W = rng.standard_normal((nt + 1, len(obs)))

    def dJdp(n, p):
        out = np.zeros(p.size)
        out[obs] = W[n]
        return out.reshape(p.shape)
    rec = adjoint.forward_record(sim, nt)
    J = sum((W[k + 1] * rec[k]["p"].reshape(-1)[obs]).sum() for k in range(nt))
    grads = adjoint.backward(sim, rec, dJdp)
    dot = sum((gr * s).sum() for gr, s in zip(grads, sigs))
    assert abs(J - dot) <= 1e-12 * abs(J), (J, dot)


def _phased_run(phases, amps, with_grad, nonlinear_backward=True, flags=oracle.NONLINEAR):
    nt = 30
    sim = _small_sim(flags, seed=7, shape=(12, 12, 12))
    f0 = 1.5e6
    elems = [np.array([13 + 12 * (12 * 3 + 5) + k for k in range(3)]),
             np.array([20 + 12 * (12 * 3 + 7) + k for k in range(3)])]
    t = (np.arange(nt) + 0.5) * sim.g.dt
    for e, a, ph in zip(elems, amps, phases):
        sim.add_source(e, a * np.sin(2 * np.pi * f0 * t + ph))
    focal = np.array([12 * 12 * 8 + 12 * 6 + 6, 12 * 12 * 8 + 12 * 6 + 7, 12 * 12 * 9 + 12 * 6 + 6])
    value, dJdp = adjoint.mean_abs_pressure(focal, nt)
    rec = adjoint.forward_record(sim, nt)
    J = value(rec)
    if not with_grad:
        return J
    if not nonlinear_backward:
        sim.g.flags = flags & ~oracle.NONLINEAR
    grads = adjoint.backward(sim, rec, dJdp)
    dphi = np.array([(gr.sum(axis=0) * a * np.cos(2 * np.pi * f0 * t + ph)).sum()
                     for gr, a, ph in zip(grads, amps, phases)])
    damp = np.array([(gr.sum(axis=0) * np.sin(2 * np.pi * f0 * t + ph)).sum()
                     for gr, a, ph in zip(grads, amps, phases)])
    return J, dphi, damp


@pytest.mark.parametrize("flags", [oracle.NONLINEAR, oracle.NONLINEAR | oracle.ABSORBING])
def test_finite_differences_nonlinear(flags):
    phases = np.array([0.3, -0.7])
    amps = np.array([3e7, 2e7])          # strong enough that the nonlinear terms matter
    run = lambda ph, am, wg, nb=True: _phased_run(ph, am, wg, nb, flags)
    J, dphi, damp = run(phases, amps, True)
    h = 1e-6
    for e in range(2):
        dp = np.zeros(2)
        dp[e] = h
        fd = (run(phases + dp, amps, False) - run(phases - dp, amps, False)) / (2 * h)
        assert abs(fd - dphi[e]) <= 1e-6 * abs(fd), (e, fd, dphi[e])
        da = np.zeros(2)
        da[e] = h * amps[e]
        fda = (run(phases, amps + da, False) - run(phases, amps - da, False)) / (2 * h * amps[e])
        assert abs(fda - damp[e]) <= 1e-6 * abs(fda), (e, fda, damp[e])
    # the nonlinear terms of the backward pass matter at this amplitude
    _, dphi_lin, _ = run(phases, amps, True, False)
    assert np.abs(dphi_lin - dphi).max() > 1e-4 * np.abs(dphi).max()
