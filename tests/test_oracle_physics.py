"""Physics pins of the FP64 oracle: the nonlinear coefficient beta = 1 + B/2A
that Eq. 2 implies (Fubini's pre-shock harmonics of a plane wave), the
emitted amplitudes of the additive mass source, the force source and the
Dirichlet pressure source, the attenuation and phase speed of a driven plane
wave in an absorbing medium and in an absorbing layer against the dispersion
relation of the model, the transmission and reflection of a plane wave at a
planar interface, and the reflection of the PML (its profile is a reading;
the closed-form pins of its application are in test_oracle_pml.py)."""

import math

import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import jv

import oracle

C0, RHO0, DZ, DT, F0 = 1500.0, 1000.0, 5e-5, 1e-8, 1e6   # 30 points per wavelength, 100 steps per period


def _plane_wave_run(amp, bona, nonlinear, z_src, probes, nz, steps, ramp_cycles=3):
    """4 x 4 x nz grid, PML only on z, additive mass source filling the plane
    z = z_src with a ramped sinusoid; returns the last two periods of p at the
    probe planes."""
    flags = oracle.NONLINEAR if nonlinear else 0
    g = oracle.Grid(4, 4, nz, DZ, DZ, DZ, DT, C0, pml_size=(0, 0, 10), pml_alpha=(0, 0, 2.0),
                    flags=flags)
    sim = oracle.Simulation(g)
    sim.set_medium(C0, RHO0, bona, 0.0)
    t = (np.arange(steps) + 0.5) * DT
    ramp = np.clip(t * F0 / ramp_cycles, 0, 1)
    ramp = 0.5 - 0.5 * np.cos(np.pi * ramp)
    sig = amp * ramp * np.sin(2 * np.pi * F0 * t)
    yy, xx = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    idx = (xx + 4 * (yy + 4 * z_src)).ravel()
    sim.add_source(idx, sig)
    rec = []
    for n in range(steps):
        sim.step(1)
        if n >= steps - 200:
            rec.append([sim.p[z, 1, 1] for z in probes])
    return np.array(rec)           # (200, n_probes)


def _harmonics(series, nmax):
    n = len(series)
    tt = np.arange(n)
    return np.array([2 * abs(np.sum(series * np.exp(-2j * np.pi * h * tt / 100))) / n
                     for h in range(1, nmax + 1)])


def test_source_emits_its_signal_amplitude():
    """Reading R10: a planar additive mass source radiates a plane wave whose
    amplitude equals the signal amplitude (linear, 30 points per wavelength)."""
    z_src = 14
    probes = [z_src + 30, z_src + 60]
    rec = _plane_wave_run(1.0, 0.0, False, z_src, probes, 128, 700)
    for j in range(len(probes)):
        a1 = _harmonics(rec[:, j], 1)[0]
        assert abs(a1 - 1.0) <= 0.01, a1


def test_fubini_harmonics():
    """Eq. 2: the model's plane-wave nonlinearity coefficient is beta = 1 + B/2A.
    Before the shock, harmonic n of a sinusoidal plane wave is
    B_n / p_s = 2 J_n(n sigma) / (n sigma), sigma = z / x_sh,
    x_sh = rho0 c0^3 / (beta omega p_s) (Fubini's solution).

    The additive source's own near field moves the effective origin of the
    distortion (by about a third of a wavelength); one origin offset sigma0 is
    fitted to B_2 at a near probe, then all five harmonics at two far probes
    must follow Fubini.  A wrong beta changes how fast the harmonics grow
    between the probes (beta = B/2A or 1 + B/A fail by more than 10 %)."""
    bona = 10.0
    beta = 1.0 + bona / 2.0
    amp = 5e6
    z_src = 14
    x_sh_nom = RHO0 * C0 ** 3 / (beta * 2 * np.pi * F0 * amp)
    zs = [z_src + 30] + [z_src + int(round(s * x_sh_nom / DZ)) for s in (0.15, 0.35, 0.6)]
    nz = zs[-1] + 60
    steps = int((zs[-1] - z_src) / 0.3) + 600
    rec = _plane_wave_run(amp, bona, True, z_src, zs, nz, steps)
    p_s = _harmonics(rec[:, 0], 1)[0]
    x_sh = RHO0 * C0 ** 3 / (beta * 2 * np.pi * F0 * p_s)

    def fub(n, s):
        return 2 * jv(n, n * s) / (n * s)

    b2 = _harmonics(rec[:, 1], 2)[1] / p_s
    s_eff = brentq(lambda s: fub(2, s) - b2, 1e-4, 1.0)
    sigma0 = (zs[1] - z_src) * DZ / x_sh - s_eff
    assert 0 <= sigma0 < 0.05, sigma0          # a fraction of a wavelength
    for j in (2, 3):
        sigma = (zs[j] - z_src) * DZ / x_sh - sigma0
        got = _harmonics(rec[:, j], 5) / p_s
        for n in range(5):
            tol = 0.03 if n < 3 else 0.06
            assert abs(got[n] / fub(n + 1, sigma) - 1) <= tol, (sigma, n + 1, got[n])


def test_pml_reflection_below_minus_35_db():
    """Sanity check only (the paper gives no PML profile): a plane pulse that
    runs into the z PML returns less than -35 dB of its amplitude."""
    nz = 160
    g = oracle.Grid(4, 4, nz, DZ, DZ, DZ, DT, C0, pml_size=(0, 0, 10), pml_alpha=(0, 0, 2.0))
    sim = oracle.Simulation(g)
    sim.set_medium(C0, RHO0)
    z = np.arange(nz)
    p0 = np.exp(-((z - nz / 2) ** 2) / (2 * 4.0 ** 2))
    sim.set_initial_pressure(np.broadcast_to(p0.reshape(nz, 1, 1), g.shape))
    # each half-pulse (amplitude 0.5) reaches the PML after ~70 cells; give it time to return
    sim.step(int(2 * (nz / 2) / 0.3) + 40)
    interior = np.abs(sim.p[15:nz - 15, 1, 1]).max()
    assert 20 * math.log10(interior / 0.5) < -35.0, interior


def test_force_source_emits_half_its_jump():
    """Reading R15: a planar force layer F (one cell thick, density F N/m^3)
    makes a pressure jump F dz across it, so it radiates plane waves of
    pressure +F dz/2 forward and -F dz/2 backward, and velocity F dz/(2 rho0 c0)
    on both sides (linear, 30 points per wavelength)."""
    nz, z_src, steps = 160, 70, 700
    g = oracle.Grid(4, 4, nz, DZ, DZ, DZ, DT, C0, pml_size=(0, 0, 10), pml_alpha=(0, 0, 2.0))
    sim = oracle.Simulation(g)
    sim.set_medium(C0, RHO0, 0.0, 0.0)
    t = np.arange(steps) * DT
    ramp = np.clip(t * F0 / 3, 0, 1)
    ramp = 0.5 - 0.5 * np.cos(np.pi * ramp)
    F = 1e9
    yy, xx = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    sim.add_source((xx + 4 * (yy + 4 * z_src)).ravel(), F * ramp * np.sin(2 * np.pi * F0 * t), oracle.FORCE_Z)
    # the force acts at the staggered point z_src + 1/2: pressure probes 45.5 cells
    # from it on either side, velocity probes (staggered too) 45 cells
    p_probes, u_probes = [z_src - 45, z_src + 46], [z_src - 45, z_src + 45]
    rec_p, rec_u = [], []
    for n in range(steps):
        sim.step(1)
        if n >= steps - 200:
            rec_p.append([sim.p[z, 1, 1] for z in p_probes])
            rec_u.append([sim.u[2][z, 1, 1] for z in u_probes])
    rec_p, rec_u = np.array(rec_p), np.array(rec_u)
    want_p = F * DZ / 2
    for j in range(2):
        assert abs(_harmonics(rec_p[:, j], 1)[0] / want_p - 1.0) <= 0.01
        assert abs(_harmonics(rec_u[:, j], 1)[0] / (want_p / (RHO0 * C0)) - 1.0) <= 0.01
    # opposite pressure signs on the two sides, the same velocity on both
    assert np.corrcoef(rec_p[:, 0], rec_p[:, 1])[0, 1] < -0.99
    assert np.corrcoef(rec_u[:, 0], rec_u[:, 1])[0, 1] > 0.99


def test_dirichlet_source_holds_and_radiates_its_value():
    """Reading R16: a plane whose pressure is held at s(t) radiates plane waves
    of amplitude s, with the same sign, to both sides (a pressure boundary
    condition), and the held points take s exactly in every step; once the
    signal ends the plane evolves freely."""
    nz, z_src, steps, nt = 160, 70, 700, 650
    g = oracle.Grid(4, 4, nz, DZ, DZ, DZ, DT, C0, pml_size=(0, 0, 10), pml_alpha=(0, 0, 2.0))
    sim = oracle.Simulation(g)
    sim.set_medium(C0, RHO0, 0.0, 0.0)
    t = (np.arange(nt) + 1) * DT
    ramp = np.clip(t * F0 / 3, 0, 1)
    ramp = 0.5 - 0.5 * np.cos(np.pi * ramp)
    s = 1e5 * ramp * np.sin(2 * np.pi * F0 * t)
    yy, xx = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    sim.add_source((xx + 4 * (yy + 4 * z_src)).ravel(), s, oracle.DIRICHLET_P)
    probes = [z_src - 45, z_src + 45]
    rec = []
    for n in range(nt):
        sim.step(1)
        assert np.all(sim.p[z_src] == s[n])
        assert np.allclose(sim.rho[0][z_src] + sim.rho[1][z_src] + sim.rho[2][z_src], s[n] / C0 ** 2,
                           rtol=1e-12, atol=0.0)
        if n >= nt - 200:
            rec.append([sim.p[z, 1, 1] for z in probes])
    rec = np.array(rec)
    for j in range(2):
        assert abs(_harmonics(rec[:, j], 1)[0] / 1e5 - 1.0) <= 0.01
    assert np.corrcoef(rec[:, 0], rec[:, 1])[0, 1] > 0.99
    held = sim.p[z_src, 1, 1]
    sim.step(steps - nt)
    assert sim.p[z_src, 1, 1] != held and abs(sim.p[z_src, 1, 1]) < 2e5


def _dispersion_root(y, a0, omega):
    """Complex wavenumber of a plane wave of real frequency omega in the
    homogeneous linear absorbing medium of Eqs. 4a-4d, 6 and 8 (continuous
    form).  With rho, p ~ exp(i (k z - omega t)): d/dt -> -i omega, the
    operators k^(y-2), k^(y-1) act on the real part kr of k, and Eq. 6 with
    Eq. 8 gives p = c0^2 rho (1 + i omega tau kr^(y-2) - eta kr^(y-1)); the
    mass and momentum equations give omega^2 rho = k^2 p, so
    k = (omega / c0) (1 + i omega tau kr^(y-2) - eta kr^(y-1))^(-1/2),
    solved for kr by fixed-point iteration.  To first order in
    eps = 2 a0 c0 omega^(y-1): Im k = a0 omega^y (the power law of Eq. 3)."""
    tau = -2 * a0 * C0 ** (y - 1)
    eta = 2 * a0 * C0 ** y * math.tan(math.pi * y / 2)
    kr = omega / C0
    for _ in range(200):
        k = (omega / C0) / np.sqrt(1 + 1j * omega * tau * kr ** (y - 2) - eta * kr ** (y - 1))
        kr = k.real
    return k


@pytest.mark.parametrize("y", [1.1, 1.5])
def test_driven_plane_wave_attenuation_and_phase_speed(y):
    """A 1 MHz plane wave driven from a planar source into a long absorbing
    medium (4 x 4 x 512 grid, PML on z only, 40 Np/m at the source frequency):
    at steady state its amplitude decays along z at Im k and its phase advances
    at Re k of the dispersion relation above.  The phase speed pins the
    dispersion term (eta, with the sign of tan(pi y / 2)), the decay the
    absorption term (tau).  At y = 1.1 the power law a0 omega^y holds only to
    first order: Im k is 0.89 of it, Re k puts the phase speed 6 % above c0."""
    omega, alpha = 2 * np.pi * F0, 40.0
    a0 = alpha / omega ** y
    nz, z_src, steps = 512, 20, 2300
    g = oracle.Grid(4, 4, nz, DZ, DZ, DZ, DT, C0, pml_size=(0, 0, 10), pml_alpha=(0, 0, 2.0),
                    flags=oracle.ABSORBING, alpha_power=y)
    sim = oracle.Simulation(g)
    sim.set_medium(C0, RHO0, 0.0, a0)
    t = (np.arange(steps) + 0.5) * DT
    ramp = np.clip(t * F0 / 3, 0, 1)
    ramp = 0.5 - 0.5 * np.cos(np.pi * ramp)
    yy, xx = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    sim.add_source((xx + 4 * (yy + 4 * z_src)).ravel(), ramp * np.sin(omega * t))
    probes = np.arange(60, 461, 5)          # 2 mm past the source to 2 mm before the PML
    rec = []
    for n in range(steps):
        sim.step(1)
        if n >= steps - 200:                # the last two periods (100 steps each)
            rec.append(sim.p[probes, 1, 1].copy())
    rec = np.array(rec)
    amp = 2 * (rec * np.exp(-2j * np.pi * np.arange(200) / 100)[:, None]).sum(0) / 200
    z = probes * DZ
    decay = -np.polyfit(z, np.log(np.abs(amp)), 1)[0]
    kr = abs(np.polyfit(z, np.unwrap(np.angle(amp)), 1)[0])
    k = _dispersion_root(y, a0, omega)
    assert abs(decay / k.imag - 1) <= 0.015, (decay, k.imag)
    assert abs(kr / k.real - 1) <= 0.002, (kr, k.real)
    # the root reduces to the power law a0 omega^y of Eq. 3 as the absorption vanishes
    k_weak = _dispersion_root(y, a0 * 1e-3, omega)
    assert abs(k_weak.imag / (a0 * 1e-3 * omega ** y) - 1) <= 1e-2
    assert abs(k_weak.real / (omega / C0) - 1) <= 1e-3


@pytest.mark.parametrize("c1,r1,c2,r2", [(1500.0, 1000.0, 1800.0, 1200.0), (1800.0, 1200.0, 1500.0, 1000.0)])
def test_plane_interface_transmission_and_reflection(c1, r1, c2, r2):
    """Heterogeneous medium (R8's staggered density included): a 1 MHz plane
    wave of amplitude 1 (R10) from a planar source in medium 1 meets a planar
    interface to medium 2 at normal incidence.  The transmitted amplitude is
    2 Z2 / (Z1 + Z2), and on the source side the incident and reflected waves
    form a standing wave whose envelope swings between 1 + |R| and 1 - |R|,
    R = (Z2 - Z1) / (Z2 + Z1), Z = rho0 c0 (normal-incidence pressure
    coefficients of textbook acoustics).  Grid 4 x 4 x 512, 0.05 mm (30 and 36
    points per wavelength), PML on z only, linear and lossless."""
    nz, z_src, z_if, steps = 512, 20, 200, 2800
    dt = 1.0 / F0 / 120
    omega = 2 * np.pi * F0
    g = oracle.Grid(4, 4, nz, DZ, DZ, DZ, dt, max(c1, c2), pml_size=(0, 0, 10), pml_alpha=(0, 0, 2.0))
    c0 = np.full(g.shape, c1)
    c0[z_if:] = c2
    rho0 = np.full(g.shape, r1)
    rho0[z_if:] = r2
    sim = oracle.Simulation(g)
    sim.set_medium(c0, rho0, 0.0, 0.0)
    t = (np.arange(steps) + 0.5) * dt
    ramp = np.clip(t * F0 / 3, 0, 1)
    ramp = 0.5 - 0.5 * np.cos(np.pi * ramp)
    yy, xx = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    sim.add_source((xx + 4 * (yy + 4 * z_src)).ravel(), ramp * np.sin(omega * t))
    rec = []
    for n in range(steps):
        sim.step(1)
        if n >= steps - 240:                # the last two periods (120 steps each)
            rec.append(sim.p[:, 1, 1].copy())
    rec = np.array(rec)
    amp = np.abs(2 * (rec * np.exp(-2j * np.pi * np.arange(240) / 120)[:, None]).sum(0) / 240)
    z1, z2 = c1 * r1, c2 * r2
    refl, trans = (z2 - z1) / (z2 + z1), 2 * z2 / (z1 + z2)
    transmitted = amp[z_if + 40: nz - 50]
    incident_side = amp[z_src + 10: z_if - 10]
    assert np.abs(transmitted / trans - 1).max() <= 5e-3, (transmitted.min(), transmitted.max(), trans)
    assert abs(incident_side.max() / (1 + abs(refl)) - 1) <= 1e-2, (incident_side.max(), 1 + abs(refl))
    assert abs(incident_side.min() / (1 - abs(refl)) - 1) <= 1e-2, (incident_side.min(), 1 - abs(refl))


@pytest.mark.parametrize("y", [1.1, 1.5])
def test_absorbing_half_space(y):
    """Heterogeneous absorption (tau and eta of Eq. 3 as fields): the driven
    1 MHz plane wave of the dispersion pin crosses from a lossless layer into
    an absorbing one (alpha0 nonzero for z >= 150, 40 Np/m at 1 MHz).  In the
    absorbing layer it decays at Im k2 and advances at Re k2 of that medium's
    dispersion root.  On the lossless side the wave reflected at the change of
    impedance gives a standing-wave envelope of half-width |R| with
    R = (k0 - k2) / (k0 + k2), k0 = omega / c0 (plane-wave impedance
    rho0 omega / k)."""
    omega, alpha = 2 * np.pi * F0, 40.0
    a0 = alpha / omega ** y
    nz, z_src, z_if, steps = 512, 20, 150, 2300
    g = oracle.Grid(4, 4, nz, DZ, DZ, DZ, DT, C0, pml_size=(0, 0, 10), pml_alpha=(0, 0, 2.0),
                    flags=oracle.ABSORBING, alpha_power=y)
    alpha0 = np.zeros(g.shape)
    alpha0[z_if:] = a0
    sim = oracle.Simulation(g)
    sim.set_medium(C0, RHO0, 0.0, alpha0)
    t = (np.arange(steps) + 0.5) * DT
    ramp = np.clip(t * F0 / 3, 0, 1)
    ramp = 0.5 - 0.5 * np.cos(np.pi * ramp)
    yy, xx = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    sim.add_source((xx + 4 * (yy + 4 * z_src)).ravel(), ramp * np.sin(omega * t))
    rec = []
    for n in range(steps):
        sim.step(1)
        if n >= steps - 200:
            rec.append(sim.p[:, 1, 1].copy())
    rec = np.array(rec)
    amp = 2 * (rec * np.exp(-2j * np.pi * np.arange(200) / 100)[:, None]).sum(0) / 200
    k2 = _dispersion_root(y, a0, omega)
    probes = np.arange(z_if + 50, 461, 5)   # 2.5 mm into the absorbing layer to 2 mm before the PML
    z = probes * DZ
    decay = -np.polyfit(z, np.log(np.abs(amp[probes])), 1)[0]
    kr = abs(np.polyfit(z, np.unwrap(np.angle(amp[probes])), 1)[0])
    assert abs(decay / k2.imag - 1) <= 0.015, (decay, k2.imag)
    assert abs(kr / k2.real - 1) <= 0.002, (kr, k2.real)
    k0 = omega / C0
    refl = abs((k0 - k2) / (k0 + k2))
    envelope = np.abs(amp[z_src + 20: z_if - 10])
    half_width = (envelope.max() - envelope.min()) / 2
    assert abs(half_width - refl) <= 0.1 * refl + 5e-4, (half_width, refl)
