"""FP64 oracle of the k-space pseudospectral time step (test infrastructure).

Only tests, the smoke check and the CPU-baseline leg of the benchmark use this
module.  It is a plain restatement of the paper's discrete scheme:

  Eq. 4a  d/dxi p^n          = IFT{ i k_xi kappa exp(+i k_xi dxi/2) FT{p^n} }
  Eq. 4b  u_xi^{n+1/2}       = u_xi^{n-1/2} - dt/rho0_sg * d/dxi p^n
  Eq. 4c  d/dxi u_xi^{n+1/2} = IFT{ i k_xi kappa exp(-i k_xi dxi/2) FT{u_xi} }
  Eq. 4d  rho_xi^{n+1}       = (rho_xi^n - dt rho0 d_xi u_xi) / (1 + 2 dt d_xi u_xi)
                               + dt M_xi^{n+1/2}
  Eq. 5   wavenumbers k_xi
  kappa   = sinc(c_ref k dt / 2),  k = |k|      (Sec. 2.2)
  Eq. 6   p^{n+1} = c0^2 (rho + (B/2A) rho^2 / rho0 - L_d),  rho = sum_xi rho_xi
  Eq. 8   L_d = -tau IFT{k^{y-2} FT{rho0 sum_xi d_xi u_xi}} + eta IFT{k^{y-1} FT{rho}}
  Eq. 3   tau = -2 alpha0 c0^{y-1},  eta = 2 alpha0 c0^y tan(pi y / 2)

Fields are float64 arrays of shape (nz, ny, nx): x is the fastest axis, the
linear index of (x, y, z) is x + nx (y + ny z).  The velocity component u_xi
and the gradient d/dxi p live half a cell forward along xi (Fig. 1 of the
paper): entry i of u_x sits at x_i + dx/2.

Readings where the paper is silent or ambiguous (the CUDA library implements
the same readings, written independently):

 R1  Axis order: x fastest (C order [z][y][x]); FFTs are full complex 3D FFTs.
 R2  The ()·grad(rho0) terms cancel (Sec. 2.2) and are not computed.
 R3  sinc is unnormalised, sin(x)/x, with sinc(0) = 1.
 R4  Nyquist (even N): Eq. 5 gives -N/2; the shifted operators are real there,
     so the sign is immaterial.  The Nyquist element is kept.
 R5  k^{y-2} and k^{y-1} are set to 0 at k = 0.
 R6  c_ref is an input (the generators use max(c0)).
 R7  PML (Berenger split field as in Tabei 2002; profile not given): per axis,
     absorption a(s) = alpha_pml * (c_ref / dxi) * (depth(s)/P)^4 with
     depth(s) = max(0, P - s, s - (N - 1 - P)), s = i on the regular grid and
     s = i + 1/2 on the staggered grid, P the layer size in cells.  The factor
     f = exp(-a dt / 2) is applied as u <- f (f u - dt g / rho0_sg) and
     rho_xi <- f (f rho_xi - dt rho0 d) / (1 + 2 dt d).  P = 0: no layer.
     The profile itself is the reading; its application is pinned by the
     closed forms of the split-field equations one step at a time (decay by
     exp(-a dt) of each split component on its own grid, forcing weighted by
     exp(-a dt / 2)), and the layer's plane-wave reflection is below -35 dB.
 R8  rho0 at the staggered point i+1/2 is the mean of rho0 at i and i+1
     (periodic wrap).
 R9  A single global power-law exponent y.
 R10 Sources are additive mass sources: at each mask point every split
     component gets rho_xi += dt * 2 s / (3 c0 dx); s[n] is the caller's
     signal sample for step n (taken at t = (n + 1/2) dt, M^{n+1/2} in
     Eq. 4d); s = 0 after the signal ends.  dx is the x grid spacing.
 R11 Initial pressure p0: p^0 = p0, rho_xi^0 = p0 / (3 c0^2), and
     u_xi^{-1/2} = + dt / (2 rho0_sg) * d/dxi p0 (Eq. 4a operator, no PML),
     which makes u(t=0) = 0 by time symmetry.
 R12 Sensors sample p^1 .. p^Nt (after each step).  p_max = max_n p^n,
     p_rms = sqrt(mean_n (p^n)^2),
     I_xi = mean_n p^n * (ubar^{n-1/2} + ubar^{n+1/2}) / 2 with
     ubar_xi[i] = (u_xi[i-1] + u_xi[i]) / 2 along xi (periodic wrap).  The
     last term needs u^{Nt+1/2}: it is computed at read time by one extra
     velocity update that is not stored.
 R13 With no step taken: p_max = -inf, p_rms = 0, I = 0.
 R14 Time-series outputs (the paper's code stores aggregates such as the
     peak positive and negative pressure, and time-varying p and u at the
     sensor points, Sec. 3.4): p_min = min_n p^n (+inf with no step);
     the p series holds p^1 .. p^Nt at the sensor points, the u series
     u_xi^{1/2} .. u_xi^{Nt-1/2} (the value at the staggered point i + 1/2
     as stored, no averaging), both ordered [n][point] and [n][xi][point].
 R15 Force sources (the paper's velocity-updating source kind, Sec. 3.4;
     scaling not given): an additive force density F_xi [N/m^3] at the
     mask points, u_xi^{n+1/2} += dt F_xi^n / rho0_sg after the update of
     Eq. 4b (PML included), F^n = the caller's sample n (t = n dt, the time
     level of the right-hand side of Eq. 4b); 0 after the signal ends.  A
     planar force layer radiates pressure +-F dz/2 on its two sides.
 R16 Dirichlet pressure sources (Sec. 3.4: a source sets the value of the
     pressure at its grid points): in step n, after the update of Eq. 4d
     and the additive sources, rho_xi^{n+1} = s / (3 c0^2) for every xi at
     the mask points, and after Eq. 6, p^{n+1} = s there; s is the caller's
     sample n, summed over the Dirichlet sources that share a point.  A
     point is held only in the steps for which one of its signals has a
     sample; afterwards it evolves freely.  These points enter the
     absorption term of Eq. 8 with the reset densities.
"""

import os

import numpy as np
import scipy.fft as _fft

NONLINEAR = 1
ABSORBING = 2

P_MAX = 1
P_RMS = 2
I_AVG = 4
P_MIN = 8
P_SERIES = 16
U_SERIES = 32

ADDITIVE_MASS = 0
FORCE_X, FORCE_Y, FORCE_Z = 1, 2, 3
DIRICHLET_P = 4

OP_GRAD_FWD = 0   # Eq. 4a operator: i k_xi kappa exp(+i k_xi dxi / 2)
OP_DIV_BWD = 1    # Eq. 4c operator: i k_xi kappa exp(-i k_xi dxi / 2)
OP_ABS_TAU = 2    # Eq. 8 first term operator: k^{y-2}
OP_ABS_ETA = 3    # Eq. 8 second term operator: k^{y-1}

_WORKERS = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def workers():
    """Number of host threads the oracle's FFTs use."""
    return _WORKERS


def _ft(a):
    return _fft.fftn(a, workers=_WORKERS)


def _ift_real(a):
    return _fft.ifftn(a, workers=_WORKERS).real


def wavenumbers(n, d):
    """Eq. 5: k = [-N/2 .. N/2-1] 2pi/(d N) (even N) or
    [-(N-1)/2 .. (N-1)/2] 2pi/(d N) (odd N), returned in FFT storage order
    (index j holds the wavenumber of the j-th DFT bin)."""
    j = np.arange(n)
    if n % 2 == 0:
        m = np.where(j < n // 2, j, j - n)      # j = N/2 -> -N/2 (Eq. 5)
    else:
        m = np.where(j <= (n - 1) // 2, j, j - n)
    return m.astype(np.float64) * (2.0 * np.pi / (d * n))


def sinc(x):
    """Unnormalised sinc, sin(x)/x with sinc(0) = 1 (reading R3)."""
    return np.sinc(np.asarray(x) / np.pi)


class Grid:
    """Grid and run parameters (mirrors the C-ABI grid descriptor)."""

    def __init__(self, nx, ny, nz, dx, dy, dz, dt, c_ref, pml_size=(0, 0, 0),
                 pml_alpha=(0.0, 0.0, 0.0), flags=0, alpha_power=1.5):
        self.n = (int(nx), int(ny), int(nz))
        self.d = (float(dx), float(dy), float(dz))
        self.dt = float(dt)
        self.c_ref = float(c_ref)
        self.pml_size = tuple(int(v) for v in pml_size)
        self.pml_alpha = tuple(float(v) for v in pml_alpha)
        self.flags = int(flags)
        self.alpha_power = float(alpha_power)

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    @property
    def nonlinear(self):
        return bool(self.flags & NONLINEAR)

    @property
    def absorbing(self):
        return bool(self.flags & ABSORBING)

    def k_axes(self):
        """k_x, k_y, k_z (Eq. 5) broadcast to the (nz, ny, nx) field shape."""
        nx, ny, nz = self.n
        dx, dy, dz = self.d
        kx = wavenumbers(nx, dx).reshape(1, 1, nx)
        ky = wavenumbers(ny, dy).reshape(1, ny, 1)
        kz = wavenumbers(nz, dz).reshape(nz, 1, 1)
        return kx, ky, kz

    def k_mag(self):
        kx, ky, kz = self.k_axes()
        return np.sqrt(kx * kx + ky * ky + kz * kz)


def kappa(grid):
    """k-space correction kappa = sinc(c_ref k dt / 2) (Sec. 2.2, after Eq. 5)."""
    return sinc(grid.c_ref * grid.k_mag() * grid.dt / 2.0)


def shift_gradient_ops(grid, sign):
    """Spectral operators i k_xi kappa exp(sign i k_xi dxi / 2) for xi = x, y, z
    (Eq. 4a with sign = +1, Eq. 4c with sign = -1)."""
    kap = kappa(grid)
    ops = []
    for k, d in zip(grid.k_axes(), grid.d):
        ops.append(1j * k * kap * np.exp(sign * 1j * k * d / 2.0))
    return ops


def absorption_ops(grid):
    """k^{y-2} and k^{y-1} of Eq. 8, zero at k = 0 (reading R5)."""
    k = grid.k_mag()
    y = grid.alpha_power
    with np.errstate(divide="ignore", invalid="ignore"):
        tau_op = np.where(k > 0, k ** (y - 2.0), 0.0)
        eta_op = np.where(k > 0, k ** (y - 1.0), 0.0)
    return tau_op, eta_op


def apply_operator(grid, op, f):
    """IFT{O FT{f}} for one of the step's spectral operators.

    OP_GRAD_FWD / OP_DIV_BWD return [x, y, z] components (Eq. 4a / 4c);
    OP_ABS_TAU / OP_ABS_ETA return a one-element list (the two IFT terms of
    Eq. 8 without the tau / eta prefactors)."""
    F = _ft(np.asarray(f, dtype=np.float64))
    if op == OP_GRAD_FWD:
        return [_ift_real(o * F) for o in shift_gradient_ops(grid, +1)]
    if op == OP_DIV_BWD:
        return [_ift_real(o * F) for o in shift_gradient_ops(grid, -1)]
    tau_op, eta_op = absorption_ops(grid)
    if op == OP_ABS_TAU:
        return [_ift_real(tau_op * F)]
    if op == OP_ABS_ETA:
        return [_ift_real(eta_op * F)]
    raise ValueError("unknown operator")


def pml_profile(n, size, alpha_pml, c_ref, d, dt, staggered):
    """Per-axis PML factor f = exp(-a dt / 2) on the regular (s = i) or
    staggered (s = i + 1/2) grid (reading R7)."""
    s = np.arange(n, dtype=np.float64) + (0.5 if staggered else 0.0)
    if size <= 0:
        return np.ones(n)
    depth = np.maximum(0.0, np.maximum(size - s, s - (n - 1 - size)))
    a = alpha_pml * (c_ref / d) * (depth / size) ** 4
    return np.exp(-a * dt / 2.0)


class Simulation:
    """Stateful FP64 simulation mirroring the C-ABI call sequence:
    create -> set_medium -> [set_initial_pressure] -> add_source* ->
    add_sensor* -> step(n)* -> read."""

    def __init__(self, grid):
        self.g = grid
        shape = grid.shape
        self.p = np.zeros(shape)
        self.u = [np.zeros(shape) for _ in range(3)]
        self.rho = [np.zeros(shape) for _ in range(3)]
        self.n = 0
        self.sources = []
        self.forces = []
        self.dirichlet = []
        self.sensors = []
        self.medium_set = False
        self._build_operators()

    # -- set-up ---------------------------------------------------------
    def _build_operators(self):
        g = self.g
        self.Df = shift_gradient_ops(g, +1)
        self.Db = shift_gradient_ops(g, -1)
        if g.absorbing:
            self.tau_op, self.eta_op = absorption_ops(g)
        nx, ny, nz = g.n
        shapes = [(1, 1, nx), (1, ny, 1), (nz, 1, 1)]
        self.f = []
        self.f_sg = []
        for ax in range(3):
            n = g.n[ax]
            self.f.append(pml_profile(n, g.pml_size[ax], g.pml_alpha[ax], g.c_ref,
                                      g.d[ax], g.dt, False).reshape(shapes[ax]))
            self.f_sg.append(pml_profile(n, g.pml_size[ax], g.pml_alpha[ax], g.c_ref,
                                         g.d[ax], g.dt, True).reshape(shapes[ax]))

    def set_medium(self, c0, rho0, bona=0.0, alpha0=0.0):
        """Medium: sound speed c0, ambient density rho0, B/A, and the power-law
        prefactor alpha0 in Np (rad/s)^-y m^-1 (Eq. 3).  Scalars or fields."""
        shape = self.g.shape
        self.c0 = np.broadcast_to(np.asarray(c0, dtype=np.float64), shape).copy()
        self.rho0 = np.broadcast_to(np.asarray(rho0, dtype=np.float64), shape).copy()
        self.bona = np.broadcast_to(np.asarray(bona, dtype=np.float64), shape).copy()
        self.alpha0 = np.broadcast_to(np.asarray(alpha0, dtype=np.float64), shape).copy()
        # rho0 on the staggered grid, reading R8 (axis 2 = x, 1 = y, 0 = z)
        self.rho0_sg = [0.5 * (self.rho0 + np.roll(self.rho0, -1, axis=a)) for a in (2, 1, 0)]
        y = self.g.alpha_power
        self.tau = -2.0 * self.alpha0 * self.c0 ** (y - 1.0)                       # Eq. 3
        self.eta = 2.0 * self.alpha0 * self.c0 ** y * np.tan(np.pi * y / 2.0)      # Eq. 3
        self.medium_set = True

    def set_initial_pressure(self, p0):
        """Reading R11."""
        p0 = np.asarray(p0, dtype=np.float64).reshape(self.g.shape)
        self.p = p0.copy()
        self.rho = [p0 / (3.0 * self.c0 ** 2) for _ in range(3)]
        P = _ft(p0)
        self.u = [self.g.dt / (2.0 * self.rho0_sg[i]) * _ift_real(self.Df[i] * P)
                  for i in range(3)]

    def add_source(self, idx, signal, mode=ADDITIVE_MASS):
        """Additive mass source (reading R10), force source along x, y or z
        (FORCE_X/Y/Z, reading R15) or Dirichlet pressure source (DIRICHLET_P,
        reading R16) at linear indices idx; signal has shape (n_t,) (shared)
        or (len(idx), n_t) (per point)."""
        if mode not in (ADDITIVE_MASS, FORCE_X, FORCE_Y, FORCE_Z, DIRICHLET_P):
            raise ValueError("unknown source mode")
        idx = np.asarray(idx, dtype=np.int64)
        sig = np.asarray(signal, dtype=np.float64)
        if sig.ndim == 1:
            sig = np.broadcast_to(sig, (len(idx), sig.shape[0]))
        if mode == ADDITIVE_MASS:
            self.sources.append((idx, sig))
        elif mode == DIRICHLET_P:
            self.dirichlet.append((idx, sig))
        else:
            self.forces.append((idx, sig, mode - 1))
        return len(self.sources) + len(self.forces) + len(self.dirichlet) - 1

    def _dirichlet_values(self, n):
        """(points, summed sample) of the Dirichlet sources held in step n (R16)."""
        val = np.zeros(self.p.size)
        held = np.zeros(self.p.size, dtype=bool)
        for idx, sig in self.dirichlet:
            if n < sig.shape[1]:
                np.add.at(val, idx, sig[:, n])
                held[idx] = True
        pts = np.nonzero(held)[0]
        return pts, val[pts]

    def add_sensor(self, idx=None, record=P_MAX):
        """Sensor at linear indices idx (None = every grid point)."""
        if idx is None:
            idx = np.arange(self.p.size, dtype=np.int64)
        idx = np.asarray(idx, dtype=np.int64)
        m = len(idx)
        s = dict(idx=idx, record=record, p_max=np.full(m, -np.inf), p_min=np.full(m, np.inf), p2=np.zeros(m),
                 I=np.zeros((3, m)), count=0, p_series=[], u_series=[])
        self.sensors.append(s)
        return len(self.sensors) - 1

    # -- the time step ----------------------------------------------------
    def _source_term(self, n):
        """M_xi^{n+1/2} dt for each split component (reading R10)."""
        add = np.zeros(self.p.size)
        dx = self.g.d[0]
        c0 = self.c0.reshape(-1)
        for idx, sig in self.sources:
            if n < sig.shape[1]:
                s = sig[:, n]
                np.add.at(add, idx, self.g.dt * 2.0 * s / (3.0 * c0[idx] * dx))
        return add.reshape(self.g.shape)

    def _velocity_update(self, p, n):
        """Eq. 4a then Eq. 4b with the PML of reading R7 and the force sources
        of step n (reading R15); returns new u."""
        P = _ft(p)
        out = []
        for i in range(3):
            g = _ift_real(self.Df[i] * P)                                            # Eq. 4a
            out.append(self.f_sg[i] * (self.f_sg[i] * self.u[i]
                                       - self.g.dt * g / self.rho0_sg[i]))           # Eq. 4b
        for idx, sig, ax in self.forces:
            if n < sig.shape[1]:
                flat = out[ax].reshape(-1)
                np.add.at(flat, idx, self.g.dt * sig[:, n] / self.rho0_sg[ax].reshape(-1)[idx])
        return out

    def _accumulate_intensity(self, p, u_old, u_new):
        for s in self.sensors:
            if not (s["record"] & I_AVG):
                continue
            idx = s["idx"]
            pf = p.reshape(-1)[idx]
            for i, ax in enumerate((2, 1, 0)):
                ubar_old = 0.5 * (np.roll(u_old[i], 1, axis=ax) + u_old[i])
                ubar_new = 0.5 * (np.roll(u_new[i], 1, axis=ax) + u_new[i])
                s["I"][i] += pf * 0.5 * (ubar_old.reshape(-1)[idx] + ubar_new.reshape(-1)[idx])

    def step(self, nsteps=1):
        g = self.g
        dt = g.dt
        for _ in range(int(nsteps)):
            u_new = self._velocity_update(self.p, self.n)
            if self.n >= 1:
                self._accumulate_intensity(self.p, self.u, u_new)
            self.u = u_new
            d = [_ift_real(self.Db[i] * _ft(self.u[i])) for i in range(3)]           # Eq. 4c
            src = self._source_term(self.n) if self.sources else None
            for i in range(3):
                num = self.f[i] * (self.f[i] * self.rho[i] - dt * self.rho0 * d[i])
                den = (1.0 + 2.0 * dt * d[i]) if g.nonlinear else 1.0
                self.rho[i] = num / den                                              # Eq. 4d
                if src is not None:
                    self.rho[i] = self.rho[i] + src
            if self.dirichlet:                                                       # R16
                pts, sv = self._dirichlet_values(self.n)
                c0f = self.c0.reshape(-1)
                for i in range(3):
                    self.rho[i].reshape(-1)[pts] = sv / (3.0 * c0f[pts] ** 2)
            rho = self.rho[0] + self.rho[1] + self.rho[2]
            if g.absorbing:
                dsum = self.rho0 * (d[0] + d[1] + d[2])
                Ld = (-self.tau * _ift_real(self.tau_op * _ft(dsum))
                      + self.eta * _ift_real(self.eta_op * _ft(rho)))                 # Eq. 8
            else:
                Ld = 0.0
            nl = (self.bona / 2.0) * rho * rho / self.rho0 if g.nonlinear else 0.0
            self.p = self.c0 ** 2 * (rho + nl - Ld)                                  # Eq. 6
            if self.dirichlet:
                self.p.reshape(-1)[pts] = sv                                         # R16
            self.n += 1
            self._record(self.p)

    def _record(self, p):
        pf = p.reshape(-1)
        for s in self.sensors:
            v = pf[s["idx"]]
            s["p_max"] = np.maximum(s["p_max"], v)
            s["p_min"] = np.minimum(s["p_min"], v)
            s["p2"] += v * v
            s["count"] += 1
            if s["record"] & P_SERIES:
                s["p_series"].append(v.copy())
            if s["record"] & U_SERIES:                         # u^{n+1/2} of this step (R14)
                s["u_series"].append(np.stack([u.reshape(-1)[s["idx"]] for u in self.u]))

    # -- outputs ----------------------------------------------------------
    def read(self, sensor_id, which):
        s = self.sensors[sensor_id]
        nt = s["count"]
        if which == P_MAX:
            return s["p_max"].copy()
        if which == P_MIN:
            return s["p_min"].copy()
        if which == P_SERIES:
            return np.array(s["p_series"]).reshape(len(s["p_series"]), len(s["idx"]))
        if which == U_SERIES:
            return np.array(s["u_series"]).reshape(len(s["u_series"]), 3, len(s["idx"]))
        if which == P_RMS:
            return np.sqrt(s["p2"] / nt) if nt else np.zeros_like(s["p2"])
        if which == I_AVG:
            if nt == 0:
                return np.zeros_like(s["I"])
            tail = np.zeros_like(s["I"])
            u_tail = self._velocity_update(self.p, self.n)   # u^{Nt+1/2}, not stored (R12)
            pf = self.p.reshape(-1)[s["idx"]]
            for i, ax in enumerate((2, 1, 0)):
                ubar_old = 0.5 * (np.roll(self.u[i], 1, axis=ax) + self.u[i])
                ubar_new = 0.5 * (np.roll(u_tail[i], 1, axis=ax) + u_tail[i])
                tail[i] = pf * 0.5 * (ubar_old.reshape(-1)[s["idx"]] + ubar_new.reshape(-1)[s["idx"]])
            return (s["I"] + tail) / nt
        raise ValueError("unknown output")

    def fields(self):
        """Current state: p^n, u^{n-1/2} (x, y, z), rho_xi^n (x, y, z)."""
        return dict(p=self.p.copy(), ux=self.u[0].copy(), uy=self.u[1].copy(),
                    uz=self.u[2].copy(), rhox=self.rho[0].copy(),
                    rhoy=self.rho[1].copy(), rhoz=self.rho[2].copy())
