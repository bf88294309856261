"""Differentiable focal-pressure objective of a segmented transducer.

SimulateFocal(phases, amps) runs the GPU time step with one additive mass
source per transducer element driven by s_e(t) = A_e sin(omega t + phi_e)
(sampled at t = (n + 1/2) dt) and returns J = mean |p| over a focal region
and all steps.  Its backward pass uses the library's hand-written adjoint
(kwgb_adjoint: checkpoints every K steps, segment recomputation, reverse
steps) and the chain rule
    dJ/dA_e   = sum_n dJ/ds_e^n sin(omega t_n + phi_e),
    dJ/dphi_e = sum_n dJ/ds_e^n A_e cos(omega t_n + phi_e).
When no input needs a gradient only the forward run is made.
"""

import numpy as np
import torch

from . import kwgb


class FocalProblem:
    """Grid, medium, element masks, focal region and drive frequency of a
    segmented-transducer problem (everything except phases and amplitudes)."""

    def __init__(self, cfg, n_steps=None, checkpoint_every=50):
        self.cfg = cfg
        self.elements = cfg["elements"]
        self.focal = np.asarray(cfg["focal"], dtype=np.int64)
        self.freq = cfg["freq"]
        self.n_steps = int(n_steps or cfg["n_steps"])
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
        """J only (plain forward run through the sensor outputs)."""
        sim = self.simulation(phases, amps)
        sid = sim.add_sensor(self.focal, kwgb.P_MAX)
        total = np.zeros(len(self.focal))
        # J = mean |p|: step one at a time and accumulate |p| at the focus
        for _ in range(self.n_steps):
            sim.step(1)
            total += np.abs(sim.read_field("p").reshape(-1)[self.focal])
        sim.close()
        del sid
        return total.sum() / (len(self.focal) * self.n_steps)

    def value_and_grad(self, phases, amps):
        sim = self.simulation(phases, amps)
        J, g = sim.adjoint(self.focal, self.n_steps, self.checkpoint_every)
        self.last_device_bytes = sim.device_bytes
        sim.close()
        w = 2.0 * np.pi * self.freq
        dphi = np.array([(gr[0] * a * np.cos(w * self.t + ph)).sum() for gr, a, ph in zip(g, amps, phases)])
        damp = np.array([(gr[0] * np.sin(w * self.t + ph)).sum() for gr, a, ph in zip(g, amps, phases)])
        return J, dphi, damp, g


class SimulateFocal(torch.autograd.Function):
    """J = SimulateFocal.apply(phases, amps, problem)."""

    @staticmethod
    def forward(ctx, phases, amps, problem):
        ph = phases.detach().double().cpu().numpy()
        am = amps.detach().double().cpu().numpy()
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            J, dphi, damp, _ = problem.value_and_grad(ph, am)
            ctx.save_for_backward(torch.from_numpy(dphi).to(phases.device, phases.dtype),
                                  torch.from_numpy(damp).to(amps.device, amps.dtype))
        else:
            J = problem.objective(ph, am)
        return torch.tensor(J, dtype=phases.dtype, device=phases.device)

    @staticmethod
    def backward(ctx, gJ):
        dphi, damp = ctx.saved_tensors
        return gJ * dphi, gJ * damp, None
