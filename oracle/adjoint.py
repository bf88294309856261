"""FP64 adjoint (reverse mode) of the oracle's time step (test infrastructure).

The forward step of kspace.Simulation (Eqs. 4a-4d, 6, 8 with the PML and
source readings) is differentiated backwards, step by step, from the stored
forward states.  Facts used:

* the adjoint of IFT{O FT{.}} on real fields is IFT{conj(O) FT{.}}, so the
  adjoint of the Eq. 4a operator is IFT{conj(i k kappa e^{+ik d/2}) FT{.}}
  and that of Eq. 4c is IFT{conj(i k kappa e^{-ik d/2}) FT{.}};
  k^{y-2}, k^{y-1} and kappa are real and even, hence self-adjoint;
* Eq. 4d: d rho_xi'/d rho_xi = f^2 / (1 + 2 dt d),
          d rho_xi'/d d      = -f dt (rho0 + 2 f rho_xi) / (1 + 2 dt d)^2
  (linear model: f^2 and -f dt rho0);
* Eq. 6:  d p / d rho = c0^2 (1 + (B/A) rho / rho0) (linear: c0^2), and the
  absorption term contributes -c0^2 eta k^{y-1} on rho and
  +c0^2 tau k^{y-2} rho0 on each d_xi (Eq. 8);
* the additive source adds dt 2 s / (3 c0 dx) to every rho_xi, so
  dJ/ds^n = sum_xi lambda_rho_xi' dt 2 / (3 c0 dx) at the source points.

Pinned by tests/test_oracle_adjoint.py (dot-product identity of the linear
model, central finite differences of the nonlinear model).
"""

import numpy as np

from . import kspace as ks


def forward_record(sim, nsteps):
    """Run nsteps steps of `sim`, recording what the backward pass needs:
    rho_xi before each step, u after it, p after it, and the step index."""
    rec = []
    for _ in range(int(nsteps)):
        rho_before = [r.copy() for r in sim.rho]
        n = sim.n
        sim.step(1)
        rec.append(dict(n=n, rho=rho_before, u=[u.copy() for u in sim.u], p=sim.p.copy()))
    return rec


def backward(sim, rec, dJdp):
    """Reverse pass over the recorded steps.

    dJdp(n, p) returns the explicit sensitivity dJ/dp^n (an array shaped like
    the grid) of the objective to the sample p^n, n = 1..Nt.  Returns, for
    every source of `sim` (in add order), dJ/dsignal per source point: an
    (n_points, n_t) array (sum over the points for a shared signal)."""
    if sim.forces or sim.dirichlet:
        raise NotImplementedError("the adjoint covers additive mass sources only")
    g = sim.g
    dt = g.dt
    dx = g.d[0]
    shape = g.shape
    c2 = sim.c0 ** 2
    lam_p = np.zeros(shape)
    lam_u = [np.zeros(shape) for _ in range(3)]
    lam_rho = [np.zeros(shape) for _ in range(3)]
    grads = [np.zeros_like(sig) for _, sig in sim.sources]
    c0f = sim.c0.reshape(-1)
    for k in reversed(range(len(rec))):
        r = rec[k]
        n = r["n"]
        rho_after = rec[k + 1]["rho"] if k + 1 < len(rec) else sim.rho
        rho_tot = rho_after[0] + rho_after[1] + rho_after[2]
        d = [ks._ift_real(sim.Db[i] * ks._ft(r["u"][i])) for i in range(3)]          # Eq. 4c, recomputed
        lam_p = lam_p + dJdp(n + 1, r["p"])
        # Eq. 6 (and Eq. 8): p = c0^2 (rho + B/2A rho^2/rho0 - L_d)
        if g.nonlinear:
            lam_rt = c2 * (1.0 + sim.bona * rho_tot / sim.rho0) * lam_p
        else:
            lam_rt = c2 * lam_p
        lam_dsum = None
        if g.absorbing:
            lam_rt = lam_rt + ks._ift_real(sim.eta_op * ks._ft(-sim.eta * c2 * lam_p))
            lam_dsum = sim.rho0 * ks._ift_real(sim.tau_op * ks._ft(sim.tau * c2 * lam_p))
        lam_p_new = np.zeros(shape)
        lam_src = np.zeros(shape)                      # sum_xi lambda_rho_xi' (source gradient)
        for i in range(3):
            lam_rp = lam_rho[i] + lam_rt               # rho = sum_xi rho_xi
            lam_src += lam_rp
            f = sim.f[i]
            if g.nonlinear:
                den = 1.0 + 2.0 * dt * d[i]
                lam_rho[i] = lam_rp * f * f / den
                lam_d = -lam_rp * f * dt * (sim.rho0 + 2.0 * f * r["rho"][i]) / (den * den)
            else:
                lam_rho[i] = lam_rp * f * f
                lam_d = -lam_rp * f * dt * sim.rho0
            if lam_dsum is not None:
                lam_d = lam_d + lam_dsum
            # d_xi = IFT{Db FT{u_xi'}}  ->  lambda_u' += IFT{conj(Db) FT{lambda_d}}
            lam_up = lam_u[i] + ks._ift_real(np.conj(sim.Db[i]) * ks._ft(lam_d))
            fs = sim.f_sg[i]
            lam_u[i] = fs * fs * lam_up                # Eq. 4b w.r.t. u^{n-1/2}
            lam_g = -fs * dt / sim.rho0_sg[i] * lam_up
            # g_xi = IFT{Df FT{p^n}}  ->  lambda_p^n += IFT{conj(Df) FT{lambda_g}}
            lam_p_new += ks._ift_real(np.conj(sim.Df[i]) * ks._ft(lam_g))
        flat = lam_src.reshape(-1)
        for s, (idx, sig) in enumerate(sim.sources):
            if n < sig.shape[1]:
                grads[s][:, n] += flat[idx] * dt * 2.0 / (3.0 * c0f[idx] * dx)
        lam_p = lam_p_new
    return grads


def mean_abs_pressure(idx, nt):
    """J = 1/(|F| Nt) sum_n sum_{i in F} |p^n(i)| and its explicit
    sensitivity dJ/dp^n = sign(p^n) / (|F| Nt) on F (d|p|/dp = sign(p))."""
    idx = np.asarray(idx, dtype=np.int64)
    w = 1.0 / (len(idx) * nt)

    def value(rec):
        return w * sum(np.abs(r["p"].reshape(-1)[idx]).sum() for r in rec)

    def dJdp(n, p):
        out = np.zeros(p.size)
        out[idx] = w * np.sign(p.reshape(-1)[idx])
        return out.reshape(p.shape)
    return value, dJdp
