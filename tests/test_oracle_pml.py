"""Pins of the oracle's split-field PML (reading R7).

The paper names the layer only (Berenger's split field as Tabei applies it,
Sec. 2.2 after Eq. 5), so the absorption profile is a reading:

    a_xi(s) = alpha_pml (c_ref / dxi) (depth(s) / P)^4,
    depth(s) = max(0, P - s, s - (N - 1 - P)),

with s = i for the split densities (regular points) and s = i + 1/2 for the
velocities (staggered points).  What the split-field layer does with that
profile is fixed by its equations: inside the layer every split component
obeys

    d u_xi / dt   = -a_xi u_xi   - (1/rho0) d_xi p,
    d rho_xi / dt = -a_xi rho_xi - rho0 d_xi u_xi,

and the step integrates each with the integrating factor exp(-a dt): the
component's own value decays by exactly exp(-a dt) over a step, and the
forcing, taken at mid-step, is weighted by exp(-a dt / 2).  The tests below
check these closed forms one step at a time, element by element, on an
anisotropic grid with a layer of a different size and strength on every axis:

  A  zero gradient, velocity zero: rho_xi <- exp(-a_xi(i) dt) rho_xi and u
     stays zero (regular points);
  B  zero pressure: u_xi <- exp(-a_xi(i + 1/2) dt) u_xi (staggered points);
  C  zero velocity, pressure a single Fourier mode along xi: u_xi becomes
     -exp(-a_xi(i + 1/2) dt / 2) dt (d_xi p) / rho0 with the closed-form
     staggered derivative -k0 kappa(k0) sin(k0 (x + dxi/2)) of the mode;
  D  zero pressure, a constant density R, velocity chosen so that B makes
     it a single mode: rho_xi becomes
     exp(-a_xi(i) dt / 2) (exp(-a_xi(i) dt / 2) R - dt rho0 d) / (1 + 2 dt d)
     (denominator only when nonlinear) with d = -k0 kappa sin(k0 x) the
     mode's closed-form derivative at the regular points.

Mistakes each test catches (checked by planting them in a copy of the
oracle): the factor applied once instead of twice (A, B: off by the factor
itself, 0.69 to 1 in these layers); the forcing weighted by the full factor or not at all (C, D);
the regular and staggered profiles swapped (A, B, C, D: the depth differs by
half a cell, 1e-4 against 6e-6 in the first cell of a 10-cell layer and
larger deeper in); the profile power 2 instead of 4 (A-D); one axis's
spacing used for another (A-D, the axes differ here); the nonlinear
denominator dividing only the forcing term, or missing (D).
"""

import numpy as np
import pytest

import oracle

N = (24, 16, 20)                     # nx, ny, nz
D = (1.0e-4, 1.3e-4, 0.8e-4)         # dx, dy, dz
P = (5, 4, 6)                        # layer cells per axis
ALPHA = (2.0, 1.5, 2.5)              # alpha_pml per axis
C_REF = 1500.0
RHO0 = 1000.0
DT = 0.3 * min(D) / C_REF
AXES = {0: 2, 1: 1, 2: 0}            # xi -> numpy axis of the (nz, ny, nx) field


def _grid(flags=0):
    return oracle.Grid(N[0], N[1], N[2], D[0], D[1], D[2], DT, C_REF, pml_size=P,
                       pml_alpha=ALPHA, flags=flags)


def _sim(flags=0):
    sim = oracle.Simulation(_grid(flags))
    sim.set_medium(C_REF, RHO0, 5.0 if flags & oracle.NONLINEAR else 0.0, 0.0)
    return sim


def _absorption(xi, staggered):
    """Reading R7 for axis xi, written out per point: a(s) of every index."""
    n, p = N[xi], P[xi]
    out = np.zeros(n)
    for i in range(n):
        s = i + (0.5 if staggered else 0.0)
        depth = max(0.0, p - s, s - (n - 1 - p))
        out[i] = ALPHA[xi] * (C_REF / D[xi]) * (depth / p) ** 4
    return out


def _along(xi, v):
    """A 1-D profile along axis xi broadcast to the field shape."""
    shape = [1, 1, 1]
    shape[AXES[xi]] = N[xi]
    return np.broadcast_to(np.asarray(v).reshape(shape), (N[2], N[1], N[0]))


def _coords(xi, staggered):
    return (np.arange(N[xi]) + (0.5 if staggered else 0.0)) * D[xi]


def _mode(xi, m):
    k0 = 2.0 * np.pi * m / (N[xi] * D[xi])
    kap = np.sin(C_REF * k0 * DT / 2.0) / (C_REF * k0 * DT / 2.0)
    return k0, kap


def _close(got, want, scale):
    err = np.abs(np.asarray(got) - np.asarray(want)).max() / scale
    assert err <= 1e-13, err


def test_density_decays_by_the_regular_grid_factor():
    """A: constant pressure, u = 0.  No gradient acts, so each split density
    only decays, rho_xi(i) -> exp(-a_xi(i) dt) rho_xi with the profile of its
    own axis (the split components are independent), and u stays zero."""
    sim = _sim()
    r = np.array([1.0, -2.0, 0.5]) * 1e-3
    for xi in range(3):
        sim.rho[xi] = np.full(sim.p.shape, r[xi])
        sim.u[xi] = np.zeros(sim.p.shape)
    sim.p = np.full(sim.p.shape, C_REF ** 2 * r.sum())
    sim.step(1)
    for xi in range(3):
        want = r[xi] * _along(xi, np.exp(-_absorption(xi, False) * DT))
        _close(sim.rho[xi], want, abs(r[xi]))
        _close(sim.u[xi], 0.0, 1e-3)


def test_velocity_decays_by_the_staggered_grid_factor():
    """B: p = 0, rho = 0, u constant.  u_xi(i) -> exp(-a_xi(i + 1/2) dt) u_xi
    at the staggered points."""
    sim = _sim()
    u = np.array([0.3, -0.7, 1.1])
    for xi in range(3):
        sim.u[xi] = np.full(sim.p.shape, u[xi])
        sim.rho[xi] = np.zeros(sim.p.shape)
    sim.p = np.zeros(sim.p.shape)
    sim.step(1)
    for xi in range(3):
        want = u[xi] * _along(xi, np.exp(-_absorption(xi, True) * DT))
        _close(sim.u[xi], want, abs(u[xi]))


@pytest.mark.parametrize("xi", [0, 1, 2])
def test_pressure_forcing_takes_the_half_factor(xi):
    """C: u = 0, p = A cos(k0 x_xi).  The Eq. 4a operator gives the staggered
    derivative -A k0 kappa(k0) sin(k0 (x + dxi/2)) exactly (one mode, band
    limited), and the layer weights it by exp(-a(i + 1/2) dt / 2):
    u_xi = -exp(-a dt / 2) dt / rho0 * derivative; the other components stay 0."""
    sim = _sim()
    amp, m = 2.0e5, 3
    k0, kap = _mode(xi, m)
    sim.p = _along(xi, amp * np.cos(k0 * _coords(xi, False))).copy()
    for c in range(3):
        sim.u[c] = np.zeros(sim.p.shape)
        sim.rho[c] = sim.p / (3.0 * C_REF ** 2)
    sim.step(1)
    deriv = -amp * k0 * kap * np.sin(k0 * _coords(xi, True))
    half = np.exp(-_absorption(xi, True) * DT / 2.0)
    want = _along(xi, -half * DT / RHO0 * deriv)
    scale = amp * k0 * DT / RHO0
    _close(sim.u[xi], want, scale)
    for c in range(3):
        if c != xi:
            _close(sim.u[c], 0.0, scale)


@pytest.mark.parametrize("flags", [0, oracle.NONLINEAR])
@pytest.mark.parametrize("xi", [0, 1, 2])
def test_velocity_divergence_forcing_takes_the_half_factor(xi, flags):
    """D: p = 0, rho_xi = R and u_xi = V / exp(-a(i + 1/2) dt) with
    V = U cos(k0 (x + dxi/2)), so that the decay of B leaves exactly the mode
    V after the velocity update.  Its Eq. 4c derivative at the regular points
    is d = -U k0 kappa sin(k0 x), and the density update of Eq. 4d in the
    layer gives rho_xi = f (f R - dt rho0 d) / (1 + 2 dt d) with
    f = exp(-a(i) dt / 2) (denominator only in a nonlinear medium)."""
    sim = _sim(flags)
    amp, m, r = 2.0, 2, 3.0e-2
    k0, kap = _mode(xi, m)
    v = amp * np.cos(k0 * _coords(xi, True))
    sim.u[xi] = _along(xi, v / np.exp(-_absorption(xi, True) * DT)).copy()
    for c in range(3):
        if c != xi:
            sim.u[c] = np.zeros(sim.p.shape)
        sim.rho[c] = np.full(sim.p.shape, r if c == xi else 0.0)
    sim.p = np.zeros(sim.p.shape)
    sim.step(1)
    _close(sim.u[xi], _along(xi, v), amp)
    d = -amp * k0 * kap * np.sin(k0 * _coords(xi, False))
    half = np.exp(-_absorption(xi, False) * DT / 2.0)
    den = (1.0 + 2.0 * DT * d) if flags & oracle.NONLINEAR else 1.0
    want = _along(xi, half * (half * r - DT * RHO0 * d) / den)
    _close(sim.rho[xi], want, max(r, DT * RHO0 * amp * k0))
