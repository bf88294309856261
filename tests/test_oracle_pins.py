"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics: a direct DFT, Eq. 5 written out, closed-form derivatives of a
cosine, the exact per-mode solution of the k-space scheme, a conserved
discrete energy, the per-mode absorption recurrence derived from Eqs. 4, 6, 8,
and the power law of Eq. 3.  None of these re-runs the oracle's own formula."""

import math

import numpy as np
import pytest

import oracle
from oracle import kspace as ks
from paper_1408_4675_gb300 import inputs


def direct_dft3(a, sign=-1):
    """O(N^2) DFT along every axis written out as explicit sums."""
    out = np.asarray(a, dtype=np.complex128)
    for ax in range(3):
        n = out.shape[ax]
        j = np.arange(n)
        W = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
        out = np.moveaxis(np.tensordot(W, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


@pytest.mark.parametrize("shape", [(4, 6, 8), (8, 8, 8), (5, 7, 3)])
def test_fft_matches_direct_dft(shape):
    rng = np.random.default_rng(1)
    a = rng.standard_normal(shape)
    got = ks._ft(a)
    ref = direct_dft3(a)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12
    back = ks._ift_real(ref)
    assert np.linalg.norm(back - a) / np.linalg.norm(a) <= 1e-12


def test_wavenumbers_eq5_written_out():
    # even N = 4: [-2, -1, 0, 1] 2pi/(dN) listed in FFT order 0, 1, -2, -1
    d = 0.5
    np.testing.assert_allclose(oracle.wavenumbers(4, d),
                               np.array([0, 1, -2, -1]) * 2 * np.pi / (d * 4), rtol=0, atol=0)
    # odd N = 5: [-2 .. 2]
    np.testing.assert_allclose(oracle.wavenumbers(5, d),
                               np.array([0, 1, 2, -2, -1]) * 2 * np.pi / (d * 5), rtol=0, atol=0)


def _grid(nx, ny, nz, d=1e-4, c=1500.0, cfl=0.3, **kw):
    dt = kw.pop("dt", cfl * d / c)
    return oracle.Grid(nx, ny, nz, d, d * 1.25, d * 0.8, dt, c, **kw)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 3, "nyq"])
def test_staggered_gradient_of_cosine(axis, m):
    """d/dxi of cos(k0 xi) by Eq. 4a (4c) equals -k0 kappa(k0) sin(k0 (xi +- dxi/2)):
    pins the shift sign, the staggered position, kappa and Eq. 5."""
    g = _grid(12, 10, 16)
    n = g.n[axis]
    d = g.d[axis]
    mm = n // 2 if m == "nyq" else m
    k0 = 2 * np.pi * mm / (n * d)
    coord = np.arange(n) * d
    shape = [1, 1, 1]
    shape[2 - axis] = n
    f = np.broadcast_to(np.cos(k0 * coord).reshape(shape), g.shape)
    a = g.c_ref * k0 * g.dt / 2
    kap = math.sin(a) / a
    for op, sgn in ((oracle.OP_GRAD_FWD, +1), (oracle.OP_DIV_BWD, -1)):
        got = oracle.apply_operator(g, op, f)
        exp = -k0 * kap * np.sin(k0 * (coord + sgn * d / 2))
        exp = np.broadcast_to(exp.reshape(shape), g.shape)
        np.testing.assert_allclose(got[axis], exp, rtol=0, atol=1e-10 * k0)
        for other in range(3):
            if other != axis:
                np.testing.assert_allclose(got[other], 0.0, atol=1e-10 * k0)


def test_absorption_operators_on_a_mode():
    """k^{y-2} and k^{y-1} applied to a single mode, and zero on a constant."""
    g = _grid(8, 8, 16, flags=oracle.ABSORBING, alpha_power=1.3)
    kx, ky, kz = 2 * np.pi * 1 / (8 * g.d[0]), 2 * np.pi * 2 / (8 * g.d[1]), 2 * np.pi * 3 / (16 * g.d[2])
    z, y, x = np.meshgrid(np.arange(16) * g.d[2], np.arange(8) * g.d[1], np.arange(8) * g.d[0],
                          indexing="ij")
    f = np.cos(kx * x + ky * y + kz * z)
    k = math.sqrt(kx * kx + ky * ky + kz * kz)
    t = oracle.apply_operator(g, oracle.OP_ABS_TAU, f)[0]
    e = oracle.apply_operator(g, oracle.OP_ABS_ETA, f)[0]
    np.testing.assert_allclose(t, k ** (1.3 - 2) * f, rtol=0, atol=1e-12 * k ** (1.3 - 2))
    np.testing.assert_allclose(e, k ** (1.3 - 1) * f, rtol=0, atol=1e-12 * k ** (1.3 - 1))
    c = oracle.apply_operator(g, oracle.OP_ABS_TAU, np.ones(g.shape))[0]
    assert np.abs(c).max() == 0.0


@pytest.mark.parametrize("cfl", [0.3, 1.7])
def test_exact_propagation_at_c_ref(cfl):
    """Homogeneous, lossless, linear, c0 = c_ref, periodic: the k-space scheme
    gives p^n = IFT{ FT{p0} cos(n c k dt) } exactly, for any dt.  Derived from
    (i k kappa e^{+})(i k kappa e^{-}) = -k^2 kappa^2 and 2 cos(th) - 2 = -4 sin^2(th/2)."""
    g = _grid(16, 12, 20, cfl=cfl)
    sim = oracle.Simulation(g)
    sim.set_medium(1500.0, 1000.0)
    p0 = inputs.gaussian_ball(g.shape, 2.0, 1e6)
    sim.set_initial_pressure(p0)
    kx, ky, kz = g.k_axes()
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    P0 = np.fft.fftn(p0)
    for n in (1, 7, 200):
        sim.step(n - sim.n)
        exact = np.fft.ifftn(P0 * np.cos(n * 1500.0 * k * g.dt)).real
        err = np.linalg.norm(sim.p - exact) / np.linalg.norm(exact)
        assert err <= 1e-11, (n, err)


@pytest.mark.parametrize("hetero_rho", [False, True])
def test_discrete_energy_conserved(hetero_rho):
    """Lossless, linear, no PML, heterogeneous c0 (and rho0):
    E^n = sum p^2/(2 rho0 c0^2) + 1/2 sum rho0_sg u^{n-1/2} u^{n+1/2} is exactly
    conserved (it follows from Eq. 4c's operator being minus the adjoint of
    Eq. 4a's).  With rho0 varying it also pins the staggered density as the
    mean of the two neighbouring points (reading R8)."""
    g = _grid(12, 16, 10, c=1600.0)
    sim = oracle.Simulation(g)
    c0 = inputs.smooth_random_field(g.shape, 1400.0, 1600.0, seed=3, sigma=2.0)
    if hetero_rho:
        rho0 = inputs.smooth_random_field(g.shape, 900.0, 1200.0, seed=4, sigma=2.0)
    else:
        rho0 = np.full(g.shape, 1000.0)
    rho_sg = [0.5 * (rho0 + np.roll(rho0, -1, axis=a)) for a in (2, 1, 0)]
    sim.set_medium(c0, rho0)
    sim.set_initial_pressure(inputs.gaussian_ball(g.shape, 1.5, 1e5))
    E = []
    for _ in range(1000):
        p = sim.p.copy()
        u_old = [u.copy() for u in sim.u]
        sim.step(1)
        E.append(np.sum(p ** 2 / (2 * rho0 * c0 ** 2))
                 + 0.5 * sum(np.sum(r * a * b) for r, a, b in zip(rho_sg, u_old, sim.u)))
    E = np.array(E)
    assert np.abs(E - E[0]).max() / abs(E[0]) <= 1e-11


@pytest.mark.parametrize("y", [1.1, 1.5])
def test_absorption_mode_recurrence(y):
    """Homogeneous linear absorbing periodic medium, one Fourier mode.  With
    W = FT of sum d_xi u_xi, R = FT of rho, Eqs. 4a-4d, 6 and 8 reduce to
      W' = W + dt/rho0 kappa^2 k^2 P,   R' = R - dt rho0 W',
      P' = c0^2 (R' + tau k^{y-2} rho0 W' - eta k^{y-1} R'),
    with P^0 = 1, R^0 = 1/c0^2, W^{-1/2} = -dt/(2 rho0) kappa^2 k^2."""
    c0, rho0 = 1500.0, 1000.0
    g = _grid(8, 8, 16, flags=oracle.ABSORBING, alpha_power=y)
    a0 = 30.0 / (2 * np.pi * 1e6) ** y
    sim = oracle.Simulation(g)
    sim.set_medium(c0, rho0, 0.0, a0)
    kv = (2 * np.pi * 1 / (8 * g.d[0]), 2 * np.pi * 2 / (8 * g.d[1]), 2 * np.pi * 3 / (16 * g.d[2]))
    z, yy, x = np.meshgrid(np.arange(16) * g.d[2], np.arange(8) * g.d[1], np.arange(8) * g.d[0],
                           indexing="ij")
    mode = np.cos(kv[0] * x + kv[1] * yy + kv[2] * z)
    sim.set_initial_pressure(mode)
    k = math.sqrt(sum(v * v for v in kv))
    a = g.c_ref * k * g.dt / 2
    kap2k2 = (math.sin(a) / a) ** 2 * k * k
    tau = -2 * a0 * c0 ** (y - 1)
    eta = 2 * a0 * c0 ** y * math.tan(math.pi * y / 2)
    P, R, W = 1.0, 1.0 / c0 ** 2, -g.dt / (2 * rho0) * kap2k2
    for n in range(60):
        W = W + g.dt / rho0 * kap2k2 * P
        R = R - g.dt * rho0 * W
        P = c0 ** 2 * (R + tau * k ** (y - 2) * rho0 * W - eta * k ** (y - 1) * R)
        sim.step(1)
        np.testing.assert_allclose(sim.p, P * mode, rtol=0, atol=1e-10 * max(abs(P), 1e-3))


def _mode_envelope_decay(y, alpha_np):
    """Run one z-mode in a homogeneous absorbing medium; return the fitted
    temporal amplitude decay rate and the mode's angular frequency."""
    c0, rho0, nz, dz = 1500.0, 1000.0, 64, 1e-4
    m = 4
    k = 2 * np.pi * m / (nz * dz)
    omega = c0 * k
    a0 = alpha_np / omega ** y
    g = oracle.Grid(4, 4, nz, dz, dz, dz, 0.3 * dz / c0, c0, flags=oracle.ABSORBING, alpha_power=y)
    sim = oracle.Simulation(g)
    sim.set_medium(c0, rho0, 0.0, a0)
    z = np.arange(nz) * dz
    basis = np.broadcast_to(np.cos(k * z).reshape(nz, 1, 1), g.shape)
    sim.set_initial_pressure(basis)
    amp = []
    for _ in range(1500):
        sim.step(1)
        amp.append(np.sum(sim.p * basis) / np.sum(basis * basis))
    amp = np.array(amp)
    t = (np.arange(len(amp)) + 1) * g.dt
    # local maxima of |amp| with parabolic refinement, then a log-linear fit
    a = np.abs(amp)
    pk = [i for i in range(1, len(a) - 1) if a[i] >= a[i - 1] and a[i] > a[i + 1]]
    tp, ap = [], []
    for i in pk:
        y0, y1, y2 = a[i - 1], a[i], a[i + 1]
        den = y0 - 2 * y1 + y2
        off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        tp.append(t[i] + off * g.dt)
        ap.append(y1 - 0.25 * (y0 - y2) * off)
    slope = np.polyfit(np.array(tp), np.log(np.array(ap)), 1)[0]
    return -slope, alpha_np * c0


@pytest.mark.parametrize("y", [1.1, 1.5])
def test_power_law_decay_rate(y):
    """Eq. 3: the absorption term makes a mode of frequency omega decay in time
    at alpha0 omega^y c0 (weak absorption, alpha << k)."""
    gamma, expected = _mode_envelope_decay(y, alpha_np=20.0)
    assert abs(gamma / expected - 1) <= 0.02, (gamma, expected)


def test_db_to_neper_known_value():
    # 1 dB/(MHz cm) with y = 1 is 11.5129 Np/m at 1 MHz
    a0 = inputs.db_to_neper(1.0, 1.0)
    assert abs(a0 * (2 * np.pi * 1e6) - 100 / (20 * math.log10(math.e))) < 1e-12
    assert abs(a0 * (2 * np.pi * 1e6) - 11.512925) < 1e-5
