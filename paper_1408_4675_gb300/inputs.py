"""Seeded synthetic inputs for the k-space time step.

This module only builds inputs: medium fields, source masks, drive signals
and sensor masks, in the shapes of the paper's HIFU workloads (Sec. 4.1: a
nonlinear, absorbing, fully heterogeneous medium; Sec. 5: a focused bowl
transducer driving through water into layered soft tissue).  It holds none of
the time step's arithmetic, so both the CUDA library and the FP64 oracle take
their inputs from here.

Arrays are float64 with shape (nz, ny, nx) (x fastest); masks are int64
linear indices x + nx (y + ny z), sorted.
"""

import math

import numpy as np

SEED_BASE = 14084675

# Typical soft-tissue values (c m/s, rho kg/m^3, alpha0 dB/(MHz^y cm), B/A)
TISSUE = {
    "water": (1500.0, 1000.0, 0.0025, 5.0),
    "fat": (1450.0, 950.0, 0.6, 10.0),
    "muscle": (1580.0, 1050.0, 1.1, 7.4),
    "kidney": (1560.0, 1050.0, 1.0, 7.0),
}


def db_to_neper(alpha_db, y):
    """dB/(MHz^y cm) -> Np (rad/s)^-y m^-1 (the unit of alpha0 in the power
    law alpha = alpha0 omega^y)."""
    return np.asarray(alpha_db, dtype=np.float64) * 100.0 / (20.0 * math.log10(math.e)) \
        * (2.0 * math.pi * 1e6) ** (-y)


def smooth_random_field(shape, lo, hi, seed, sigma=8.0):
    """Seeded N(0,1) noise, periodic Gaussian filter of std `sigma` cells,
    min-max scaled into [lo, hi]."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(n) * 2.0 * np.pi for n in shape]
    kz, ky, kx = np.meshgrid(*ks, indexing="ij", sparse=True)
    filt = np.exp(-0.5 * sigma * sigma * (kx * kx + ky * ky + kz * kz))
    f = np.fft.ifftn(np.fft.fftn(noise) * filt).real
    f = (f - f.min()) / (f.max() - f.min())
    return lo + (hi - lo) * f


def gaussian_ball(shape, sigma, peak, center=None):
    """Gaussian of std `sigma` cells with maximum `peak` at `center` (z, y, x)."""
    if center is None:
        center = [n // 2 for n in shape]
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij", sparse=True)
    r2 = (x - center[2]) ** 2 + (y - center[1]) ** 2 + (z - center[0]) ** 2
    return peak * np.exp(-r2 / (2.0 * sigma * sigma))


def linear_index(shape, z, y, x):
    nz, ny, nx = shape
    return (np.asarray(x, dtype=np.int64) + nx * (np.asarray(y, dtype=np.int64)
                                                  + ny * np.asarray(z, dtype=np.int64)))


def bowl_voxels(shape, dx, radius, aperture, apex_z):
    """Voxels of a spherical cap (bowl) opening towards +z: points within dx/2
    of a sphere of radius `radius` centred on the focus, lateral distance from
    the axis <= aperture/2, on the apex side of the focus.  Returns (z, y, x,
    polar angle, azimuth) arrays."""
    nz, ny, nx = shape
    cy, cx = ny // 2, nx // 2
    rc = radius / dx                       # radius in cells
    fz = apex_z + rc                       # focus z (cells)
    ra = 0.5 * aperture / dx
    zmax = int(math.ceil(apex_z + rc - math.sqrt(max(rc * rc - ra * ra, 0.0)) + 1))
    zs, ys, xs = np.meshgrid(np.arange(max(apex_z - 1, 0), min(zmax + 1, nz)),
                             np.arange(ny), np.arange(nx), indexing="ij")
    lat = np.sqrt((xs - cx) ** 2.0 + (ys - cy) ** 2.0)
    dist = np.sqrt(lat ** 2 + (zs - fz) ** 2.0)
    sel = (np.abs(dist - rc) <= 0.5) & (lat <= ra) & (zs < fz)
    z, y, x = zs[sel], ys[sel], xs[sel]
    polar = np.arctan2(np.sqrt((x - cx) ** 2.0 + (y - cy) ** 2.0), fz - z)
    azim = np.arctan2(y - cy, x - cx)
    return z, y, x, polar, azim, fz


def bowl_mask(shape, dx, radius, aperture, apex_z):
    z, y, x, _, _, fz = bowl_voxels(shape, dx, radius, aperture, apex_z)
    return np.sort(linear_index(shape, z, y, x)), fz


def segmented_bowl(shape, dx, radius, aperture, apex_z, rings=16, sectors=16):
    """Bowl split into rings x sectors elements of equal area (rings equally
    spaced in 1 - cos(polar), sectors equally spaced in azimuth).  Returns a
    list of sorted index arrays, element e = ring * sectors + sector."""
    z, y, x, polar, azim, fz = bowl_voxels(shape, dx, radius, aperture, apex_z)
    cmax = 1.0 - math.cos(math.asin(min(1.0, 0.5 * aperture / radius)))
    ring = np.minimum((1.0 - np.cos(polar)) / cmax * rings, rings - 1).astype(int)
    sector = np.minimum(((azim + math.pi) / (2 * math.pi) * sectors).astype(int), sectors - 1)
    elem = ring * sectors + sector
    idx = linear_index(shape, z, y, x)
    return [np.sort(idx[elem == e]) for e in range(rings * sectors)], fz


def box_mask(shape, center, half):
    """Cube of (2 half + 1)^3 points around center (z, y, x)."""
    zc, yc, xc = center
    r = np.arange(-half, half + 1)
    z, y, x = np.meshgrid(zc + r, yc + r, xc + r, indexing="ij")
    return np.sort(linear_index(shape, z.ravel(), y.ravel(), x.ravel()))


def tone_burst(freq, cycles, amp, dt, n_t):
    """Hann-windowed tone burst sampled at t = (n + 1/2) dt."""
    t = (np.arange(n_t) + 0.5) * dt
    dur = cycles / freq
    w = np.where(t < dur, 0.5 - 0.5 * np.cos(2.0 * math.pi * t / dur), 0.0)
    return amp * w * np.sin(2.0 * math.pi * freq * t)


def cw(freq, amp, dt, n_t, phase=0.0):
    """Continuous wave amp sin(2 pi f t + phase) sampled at t = (n + 1/2) dt."""
    t = (np.arange(n_t) + 0.5) * dt
    return amp * np.sin(2.0 * math.pi * freq * t + phase)


def layered_tissue(shape, z_start, seed):
    """Water, then seeded layers of fat / muscle / kidney normal to z from
    z_start.  Returns c0, rho0, alpha0 (dB/(MHz^y cm)) and B/A fields."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    names = ["water"] * nz
    z = z_start
    order = ["fat", "muscle", "fat", "kidney"]
    for k, name in enumerate(order):
        thick = int(rng.integers(max(2, nz // 32), max(3, nz // 12)))
        if k == len(order) - 1:
            thick = nz
        for zz in range(z, min(z + thick, nz)):
            names[zz] = name
        z += thick
        if z >= nz:
            break
    props = np.array([TISSUE[nm] for nm in names])          # (nz, 4)
    out = []
    for j in range(4):
        out.append(np.broadcast_to(props[:, j].reshape(nz, 1, 1), shape).copy())
    return out  # c0, rho0, alpha_db, bona


def make_config(i, n=None, n_steps=None):
    """One of the five workloads (1-based), optionally on a smaller cubic grid
    `n` (same physical recipe, same seeds) and with fewer steps.

    Returns a dict with the grid descriptor fields, medium, initial pressure,
    sources [(idx, signal)], sensors [(idx or None, record)] and n_steps."""
    P_MAX, P_RMS, I_AVG = 1, 2, 4
    NONLINEAR, ABSORBING = 1, 2
    pml, pml_alpha, cfl = 10, 2.0, 0.3
    if i == 1:
        n = n or 64
        shape = (n, n, n)
        dx = 1e-4
        c0 = 1500.0
        dt = cfl * dx / c0
        cfg = dict(shape=shape, d=(dx, dx, dx), dt=dt, c_ref=c0, flags=0, alpha_power=1.5,
                   c0=c0, rho0=1000.0, bona=0.0, alpha0=0.0,
                   p0=gaussian_ball(shape, 4.0, 1e6), sources=[],
                   sensors=[(None, P_MAX)], n_steps=n_steps or 200)
    elif i == 2:
        n = n or 256
        shape = (n, n, n)
        dx = 1e-4
        y = 1.1
        seed = SEED_BASE + 100 * 2
        c0 = smooth_random_field(shape, 1450.0, 1650.0, seed + 0)
        rho0 = smooth_random_field(shape, 950.0, 1100.0, seed + 1)
        bona = smooth_random_field(shape, 5.0, 9.0, seed + 2)
        adb = smooth_random_field(shape, 0.3, 1.0, seed + 3)
        c_ref = float(c0.max())
        dt = cfl * dx / c_ref
        steps = n_steps or 1500
        r = np.arange(pml, n - pml)
        yy, xx = np.meshgrid(r, r, indexing="ij")
        src = np.sort(linear_index(shape, np.full(xx.size, pml + 1), yy.ravel(), xx.ravel()))
        sig = tone_burst(1e6, 10, 0.5e6, dt, steps)
        cfg = dict(shape=shape, d=(dx, dx, dx), dt=dt, c_ref=c_ref, flags=NONLINEAR | ABSORBING,
                   alpha_power=y, c0=c0, rho0=rho0, bona=bona, alpha0=db_to_neper(adb, y),
                   p0=None, sources=[(src, sig)], sensors=[(None, P_MAX | P_RMS)], n_steps=steps)
    elif i in (3, 4):
        if i == 3:
            n = n or 512
            dx_full, amp, steps_full = 0.15e-3, 1.5e6, 3000
            n_full = 512
        else:
            n = n or 1024
            dx_full, amp, steps_full = 0.1e-3, 2.0e6, 500
            n_full = 1024
        # a smaller grid keeps the physical domain and coarsens the spacing
        dx = dx_full * n_full / n
        shape = (n, n, n)
        y = 1.1
        seed = SEED_BASE + 100 * i
        c0, rho0, adb, bona = layered_tissue(shape, int(0.45 * n), seed)
        c_ref = float(c0.max())
        dt = cfl * dx / c_ref
        steps = n_steps or steps_full
        src, fz = bowl_mask(shape, dx, 64e-3, 60e-3, pml + 1)
        sig = cw(1e6, amp, dt, steps)
        fzc = int(min(round(fz), n - pml - 1))
        half = max(1, min(32, n // 16))
        focal = box_mask(shape, (min(fzc, n - 1 - half), n // 2, n // 2), half)
        if i == 3:
            zz, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            plane = np.sort(linear_index(shape, zz.ravel(), np.full(zz.size, n // 2), xx.ravel()))
            sensors = [(focal, P_MAX | P_RMS | I_AVG), (plane, P_MAX | P_RMS)]
        else:
            sensors = [(focal, P_MAX | P_RMS)]
        cfg = dict(shape=shape, d=(dx, dx, dx), dt=dt, c_ref=c_ref, flags=NONLINEAR | ABSORBING,
                   alpha_power=y, c0=c0, rho0=rho0, bona=bona, alpha0=db_to_neper(adb, y),
                   p0=None, sources=[(src, sig)], sensors=sensors, n_steps=steps)
    elif i == 5:
        n = n or 128
        shape = (n, n, n)
        dx = 0.15e-3 * 128 / n
        seed = SEED_BASE + 100 * 5
        c0 = 1500.0 * (1.0 + 0.03 * (2.0 * smooth_random_field(shape, 0.0, 1.0, seed) - 1.0))
        c_ref = float(c0.max())
        dt = cfl * dx / c_ref
        steps = n_steps or 600
        elems, fz = segmented_bowl(shape, dx, 15e-3, 14e-3, pml + 1)
        rng = np.random.default_rng(seed + 1)
        phases = rng.uniform(-0.2, 0.2, len(elems))
        amps = np.full(len(elems), 1e5)
        fzc = int(min(round(fz), n - pml - 3))
        focal = box_mask(shape, (fzc, n // 2, n // 2), 2)
        cfg = dict(shape=shape, d=(dx, dx, dx), dt=dt, c_ref=c_ref, flags=NONLINEAR,
                   alpha_power=1.5, c0=c0, rho0=1000.0, bona=5.0, alpha0=0.0, p0=None,
                   elements=elems, phases=phases, amps=amps, freq=1e6,
                   sources=[(e, cw(1e6, a, dt, steps, ph)) for e, a, ph in zip(elems, amps, phases)],
                   sensors=[(focal, P_MAX)], focal=focal, n_steps=steps)
    else:
        raise ValueError("config must be 1..5")
    cfg["pml_size"] = (pml, pml, pml)
    cfg["pml_alpha"] = (pml_alpha, pml_alpha, pml_alpha)
    cfg["config"] = i
    return cfg
