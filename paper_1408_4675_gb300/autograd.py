"""Differentiable focal-pressure objective of a segmented transducer.

SimulateFocal(phases, amps) runs the GPU time step with one additive mass
source per transducer element driven by s_e(t) = A_e sin(omega t + phi_e)
(sampled at t = (n + 1/2) dt) and returns J = mean |p| over a focal region
and all steps.  forward() makes one forward run (kwgb_adjoint_forward: J is
accumulated from the focal points on the device; when an input needs a
gradient the run also keeps a checkpoint every K steps, and the simulation
that holds them is kept for backward(); when every step's density fields
fit in half the free device memory they are kept instead, and the reverse
pass recomputes nothing).  backward() runs the library's hand-written
reverse pass (kwgb_adjoint_backward: segment recomputation if
checkpointed, reverse steps) and the chain rule
    dJ/dA_e   = sum_n dJ/ds_e^n sin(omega t_n + phi_e),
    dJ/dphi_e = sum_n dJ/ds_e^n A_e cos(omega t_n + phi_e).
"""

import numpy as np
import torch

from . import kwgb


class FocalProblem:
    """Grid, medium, element masks, focal region and drive frequency of a
    segmented-transducer problem (everything except phases and amplitudes)."""

    def __init__(self, cfg, n_steps=None, checkpoint_every=None):
        """checkpoint_every: the adjoint's checkpoint interval K (K >= the
        step count keeps every step's fields); None takes every step when
        its fields (28 bytes per grid point per step) fit in half the free
        device memory, else K = 50."""
        self.cfg = cfg
        self.elements = cfg["elements"]
        self.focal = np.asarray(cfg["focal"], dtype=np.int64)
        self.freq = cfg["freq"]
        self.n_steps = int(n_steps or cfg["n_steps"])
        if checkpoint_every is None:
            keep = 28 * int(np.prod(cfg["shape"])) * self.n_steps
            free = torch.cuda.mem_get_info()[0] if torch.cuda.is_available() else 0
            checkpoint_every = self.n_steps if keep <= free // 2 else 50
        self.checkpoint_every = int(checkpoint_every)
        self.t = (np.arange(self.n_steps) + 0.5) * cfg["dt"]
        self.last_device_bytes = 0

    def signals(self, phases, amps):
        w = 2.0 * np.pi * self.freq
        return [a * np.sin(w * self.t + ph) for a, ph in zip(amps, phases)]

    def simulation(self, phases, amps):
        c = self.cfg
        sim = kwgb.Simulation(c["shape"], c["d"], c["dt"], c["c_ref"], c["pml_size"], c["pml_alpha"],
                              c["flags"], c["alpha_power"])
        sim.set_medium(c["c0"], c["rho0"], c["bona"], c["alpha0"])
        for e, sig in zip(self.elements, self.signals(phases, amps)):
            sim.add_source(e, sig)
        return sim

    def objective(self, phases, amps):
        """J only: one forward run, no checkpoints."""
        sim = self.simulation(phases, amps)
        try:
            return sim.adjoint_forward(self.focal, self.n_steps, checkpoint_every=0)
        finally:
            sim.close()

    def forward(self, phases, amps):
        """Forward run that keeps its checkpoints: returns (J, simulation);
        pass the simulation to backward()."""
        sim = self.simulation(phases, amps)
        J = sim.adjoint_forward(self.focal, self.n_steps, self.checkpoint_every)
        return J, sim

    def backward(self, sim, phases, amps):
        """Reverse pass of forward()'s run (closes the simulation): returns
        dJ/dphases, dJ/damps and dJ/dsignal per element."""
        try:
            g = sim.adjoint_backward()
            self.last_device_bytes = sim.device_bytes
        finally:
            sim.close()
        w = 2.0 * np.pi * self.freq
        dphi = np.array([(gr[0] * a * np.cos(w * self.t + ph)).sum() for gr, a, ph in zip(g, amps, phases)])
        damp = np.array([(gr[0] * np.sin(w * self.t + ph)).sum() for gr, a, ph in zip(g, amps, phases)])
        return dphi, damp, g

    def value_and_grad(self, phases, amps):
        J, sim = self.forward(phases, amps)
        dphi, damp, g = self.backward(sim, phases, amps)
        return J, dphi, damp, g


class SimulateFocal(torch.autograd.Function):
    """J = SimulateFocal.apply(phases, amps, problem)."""

    @staticmethod
    def forward(ctx, phases, amps, problem):
        ph = phases.detach().double().cpu().numpy()
        am = amps.detach().double().cpu().numpy()
        ctx.sim = None
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            J, ctx.sim = problem.forward(ph, am)
            ctx.problem, ctx.ph, ctx.am = problem, ph, am
        else:
            J = problem.objective(ph, am)
        return torch.tensor(J, dtype=phases.dtype, device=phases.device)

    @staticmethod
    def backward(ctx, gJ):
        dphi, damp, _ = ctx.problem.backward(ctx.sim, ctx.ph, ctx.am)
        ctx.sim = None
        dphi = torch.from_numpy(dphi).to(gJ.device, gJ.dtype)
        damp = torch.from_numpy(damp).to(gJ.device, gJ.dtype)
        return gJ * dphi, gJ * damp, None
