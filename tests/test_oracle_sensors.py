"""Brute-force pins of the oracle's sensor outputs (p_max, p_min, p_rms,
time-averaged intensity, p and u time series) on a tiny grid: every sample is taken from the stepped fields one
step at a time and combined by explicit loops, and the last velocity
u^{Nt+1/2} comes from actually taking one more step on a copy."""

import copy

import numpy as np

import oracle
from paper_1408_4675_gb300 import inputs


def _tiny_sim():
    nx, ny, nz = 8, 6, 5
    d = 1e-4
    g = oracle.Grid(nx, ny, nz, d, d, d, 0.3 * d / 1600.0, 1600.0, pml_size=(1, 1, 1),
                    pml_alpha=(2.0, 2.0, 2.0), flags=oracle.NONLINEAR | oracle.ABSORBING,
                    alpha_power=1.2)
    sim = oracle.Simulation(g)
    shape = g.shape
    sim.set_medium(inputs.smooth_random_field(shape, 1450, 1600, 7, 1.0),
                   inputs.smooth_random_field(shape, 950, 1100, 8, 1.0),
                   inputs.smooth_random_field(shape, 5, 9, 9, 1.0),
                   inputs.db_to_neper(inputs.smooth_random_field(shape, 0.3, 1.0, 10, 1.0), 1.2))
    sim.set_initial_pressure(inputs.gaussian_ball(shape, 1.2, 1e5, (2, 3, 4)))
    sim.add_source(np.array([3, 17, 40]), inputs.cw(1e6, 1e4, g.dt, 3))
    return sim


def test_sensor_outputs_brute_force():
    sim = _tiny_sim()
    nx, ny, nz = sim.g.n
    pts = [0, 5, 47, nx * ny * nz - 1, 123]            # includes wrap-around neighbours
    sid = sim.add_sensor(np.array(pts), oracle.P_MAX | oracle.P_RMS | oracle.I_AVG | oracle.P_MIN
                         | oracle.P_SERIES | oracle.U_SERIES)
    ref = copy.deepcopy(sim)
    nt = 5
    # p_hist[n-1] = p^n; u_hist[m] = u^{m-1/2}
    p_hist, u_hist = [], [[u.copy() for u in ref.u]]
    for _ in range(nt):
        ref.step(1)
        p_hist.append(ref.p.copy())
        u_hist.append([u.copy() for u in ref.u])
    extra = copy.deepcopy(ref)
    extra.step(1)
    u_hist.append([u.copy() for u in extra.u])        # u^{Nt+1/2}
    sim.step(nt)

    def coords(i):
        return i % nx, (i // nx) % ny, i // (nx * ny)

    def ubar(u, xi, i):
        x, y, z = coords(i)
        if xi == 0:
            xm, ym, zm = (x - 1) % nx, y, z
        elif xi == 1:
            xm, ym, zm = x, (y - 1) % ny, z
        else:
            xm, ym, zm = x, y, (z - 1) % nz
        return 0.5 * (u[xi][zm, ym, xm] + u[xi][z, y, x])

    pmax = sim.read(sid, oracle.P_MAX)
    pmin = sim.read(sid, oracle.P_MIN)
    prms = sim.read(sid, oracle.P_RMS)
    inten = sim.read(sid, oracle.I_AVG)
    pser = sim.read(sid, oracle.P_SERIES)
    user = sim.read(sid, oracle.U_SERIES)
    assert pser.shape == (nt, len(pts)) and user.shape == (nt, 3, len(pts))
    for j, i in enumerate(pts):
        x, y, z = coords(i)
        samples = [p_hist[n][z, y, x] for n in range(nt)]
        assert abs(pmax[j] - max(samples)) <= 1e-13 * max(abs(v) for v in samples)
        assert pmin[j] == min(samples)
        for n in range(nt):                  # p^{n+1} and u^{n+1/2} after step n
            assert pser[n, j] == p_hist[n][z, y, x]
            for xi in range(3):
                assert user[n, xi, j] == u_hist[n + 1][xi][z, y, x]
        rms = (sum(v * v for v in samples) / nt) ** 0.5
        assert abs(prms[j] - rms) <= 1e-13 * rms
        for xi in range(3):
            acc = 0.0
            for n in range(1, nt + 1):       # sample p^n uses u^{n-1/2}, u^{n+1/2}
                acc += p_hist[n - 1][z, y, x] * 0.5 * (ubar(u_hist[n], xi, i)
                                                      + ubar(u_hist[n + 1], xi, i))
            acc /= nt
            assert abs(inten[xi, j] - acc) <= 1e-12 * max(abs(acc), 1e-30), (xi, j)


def test_sensors_before_any_step():
    sim = _tiny_sim()
    sid = sim.add_sensor(None, oracle.P_MAX | oracle.P_RMS | oracle.I_AVG | oracle.P_MIN)
    assert np.all(np.isneginf(sim.read(sid, oracle.P_MAX)))
    assert np.all(np.isposinf(sim.read(sid, oracle.P_MIN)))
    assert np.all(sim.read(sid, oracle.P_RMS) == 0)
    assert np.all(sim.read(sid, oracle.I_AVG) == 0)
