#!/usr/bin/env python3
"""Benchmark of the GB300 k-space pseudospectral time step.

Workload (default): the 512^3 HIFU case -- spherical bowl (R = 64 mm,
aperture 60 mm) driving 1 MHz CW at 1.5 MPa through water into seeded layered
soft tissue; nonlinear, power-law absorbing, every medium property a full
field; sensors on a 65^3 focal box (p_max, p_rms, intensity) and the central
xz-plane (p_max, p_rms).  ``--config 4`` runs the 1024^3 case instead.

One step = one full time step (Eqs. 4a-4d, 6, 8: 14 FFT-equivalents, the
fused updates, sources and sensors).  The metric is ms per step (lower is
better), measured with CUDA events on the stream the library launches on,
after warm-up; every field is larger than the 129 MB L2, so no flush is
needed between steps.  The roofline object reports the dominant kernel's
algorithmic bytes per launch over its event-timed duration against the
measured HBM copy bandwidth.

``--impl reference`` times the FP64 CPU oracle (test infrastructure) on the
host cores instead: W warm-up and K timed steps of the same workload.
``--oracle-table`` times the oracle on every workload at its stated size
beside the GPU step of the same workload (a CPU-baseline table, not the
bench line).
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1408_4675_gb300 import inputs  # noqa: E402

METRIC = "ms_per_step"
UNIT = "ms/step"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=3, choices=[3, 4])
    ap.add_argument("--grid", "--n", dest="n", type=int, default=None,
                    help="cubic grid size override (same recipe; for profiling small cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 1024^3 step and the adjoint measurements")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-case", type=int, nargs=3, metavar=("NZ", "NY", "NX"), default=None,
                    help="small case for ncu captures: a heterogeneous nonlinear absorbing medium on an "
                         "NZ x NY x NX grid stepped --steps times, no timing")
    ap.add_argument("--oracle-table", action="store_true",
                    help="CPU-baseline table instead of the bench line: the FP64 oracle on every workload "
                         "at its stated size on the host cores, beside the GPU step of the same workload")
    ap.add_argument("--profile-adjoint", type=int, nargs=2, metavar=("N", "STEPS"), default=None,
                    help="small case for ncu captures of the adjoint: the segmented bowl on an N^3 grid, "
                         "STEPS forward steps keeping every step's fields, then the reverse pass; no timing")
    ap.add_argument("--profile-flags", type=int, default=0,
                    help="extra grid flags of the profiling case (4: bfloat16-split, 8: float16-split form)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class Replicas:
    """Host side of an N-GPU run.  The time step has no exchange between
    devices, so each rank steps its own copy of the workload; the ranks meet
    at a barrier on both sides of the timed region and the job's time per step
    is the slowest rank's.  `backend` is "nccl" on GPUs ("gloo" exercises the
    same logic on host cores)."""

    def __init__(self, world, backend="nccl"):
        self.world = world
        self.device = "cuda" if backend == "nccl" else "cpu"
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, value):
        """Largest `value` over the ranks (every rank receives it)."""
        if self.world == 1:
            return float(value)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(value)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def workload_name(cfg):
    n = cfg["shape"][0]
    kind = {1: "water_gaussian_initial_pressure", 2: "smooth_random_heterogeneous_tone_burst",
            5: "segmented_bowl_256_elements"}.get(cfg.get("config"), "hifu_bowl_layered_tissue")
    return "%s_%d^3" % (kind, n)


# ---------------------------------------------------------------- byte model
def kernel_bytes(cfg):
    """Algorithmic HBM bytes per launch of each kernel kind: every array the
    kernel must read or write, counted once (spectra as the nx/2+1 complex
    columns actually used; scalar medium properties take no bytes)."""
    nz, ny, nx = cfg["shape"]
    N = nx * ny * nz
    S = (nx // 2 + 1) * 8 * ny * nz
    F = 4 * N
    fld = lambda k: 0 if np.isscalar(cfg[k]) or np.ndim(cfg[k]) == 0 else F
    nonlinear = bool(cfg["flags"] & 1)
    absorbing = bool(cfg["flags"] & 2)
    nfull = sum(1 for idx, _ in cfg["sensors"] if idx is None)
    full = nfull * 24 * N
    b = {
        "y_fwd_p": 2 * S, "z_grad": 4 * S, "y_inv_grad": 6 * S,
        "x_vel": 6 * S + 6 * F + fld("rho0"),
        "y_fwd_u": 6 * S, "z_div": 6 * S, "y_inv_div": 6 * S,
    }
    if absorbing:
        b["x_dens"] = 5 * S + 7 * F + fld("rho0")
        b.update({"y_fwd_abs": 4 * S, "z_abs": 4 * S, "y_inv_abs": 4 * S})
        b["x_eos"] = 3 * S + F + fld("c0") + fld("alpha0") + (fld("rho0") + fld("bona") if nonlinear else 0) + full
    else:
        b["x_dens"] = 4 * S + 6 * F + fld("rho0") + fld("c0") + (fld("bona") if nonlinear else 0) + full
    return b


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 50 ms) of the SM clock, power and throttle
    reasons; the statistics use the samples taken inside [t0, t1] (host clock,
    set by region()), or all samples if none falls inside."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def region(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        import datetime
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    try:
                        ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    except ValueError:
                        ts = None
                    rows.append([ts] + parts[1:])
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = [r for r in rows if self.t0 is not None and r[0] is not None and self.t0 <= r[0] <= self.t1]
        n_all = len(rows)
        if inside:
            rows = inside

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        # row: timestamp, index, clocks.sm, clocks.max.sm, power.draw, active mask, four reasons
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        pw = [num(r[4]) for r in rows if num(r[4]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": n_all, "samples_in_timed_region": len(inside), "reasons": reasons}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel, shape):
    """dram bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current sources."""
    try:
        from paper_1408_4675_gb300 import build
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t.get("%s@%d" % (kernel, shape[0]))
        if e and e.get("source_digest") == build._digest():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


# ---------------------------------------------------------------- oracle (CPU)
def oracle_timed(cfg_id, n, warmup, steps):
    """Time the FP64 oracle on the workload itself (same grid, medium, sources
    and sensors): build it (not timed), run `warmup` steps, then time `steps`
    steps one by one.  Returns (seconds per step, per-step list, threads)."""
    from oracle import kspace
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import oracle_from_config
    cfg = inputs.make_config(cfg_id, n=n, n_steps=warmup + steps + 1)
    sim, _ = oracle_from_config(cfg)
    sim.step(warmup)
    per = []
    for _ in range(steps):
        t0 = time.perf_counter()
        sim.step(1)
        per.append(time.perf_counter() - t0)
    return statistics.mean(per), per, kspace.workers()


# ---------------------------------------------------------------- arms
def bench_config(cfg, world):
    """The `config` object of the JSON line (the same for both arms)."""
    n_points = int(np.prod(cfg["shape"]))
    return {"workload": workload_name(cfg), "grid": list(cfg["shape"]),
            "nonlinear": bool(cfg["flags"] & 1), "absorbing": bool(cfg["flags"] & 2),
            "heterogeneous": not np.isscalar(cfg["c0"]),
            "l2": ("every field (%d MB) exceeds the 129 MB L2; no flush needed" % (4 * n_points // 10 ** 6)
                   if 4 * n_points > 129 * 10 ** 6 else
                   "fields (%d MB) fit in the 129 MB L2: not flushed, small-grid timings include L2 reuse"
                   % (4 * n_points // 10 ** 6)),
            "parallelism": "replicas" if world > 1 else "single_gpu"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    cfg = inputs.make_config(args.config, n=args.n, n_steps=1)
    sec, per, cores = oracle_timed(args.config, args.n, args.warmup, args.steps)
    ms = 1e3 * sec
    sample = ("FP64 oracle on the workload itself (%d^3 grid, medium, bowl source, sensors), %d warm-up "
              "steps, then %d steps timed one by one (host set-up not timed); per-step %.1f-%.1f s"
              % (cfg["shape"][0], args.warmup, args.steps, min(per), max(per)))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(ms, 3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(cfg, world),
        "cpu_baseline": {"value": round(ms, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(ms, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    reps = Replicas(world, "nccl")
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()

    cfg = inputs.make_config(args.config, n=args.n, n_steps=args.warmup + args.steps + 16)
    stream = torch.cuda.current_stream()
    sim, ids = kwgb.from_config(cfg)

    sim.step(args.warmup, stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    time.sleep(0.4)
    reps.barrier()
    torch.cuda.synchronize()
    l0 = sim.launch_count
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t_region = time.time()
    ev0.record(stream)
    sim.step(args.steps, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.region(t_region, time.time())
    reps.barrier()
    launches = sim.launch_count - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    # per-kernel durations from event-instrumented steps
    prof = {}
    for _ in range(min(5, max(args.steps, 1))):
        for name, t in sim.step_profiled(stream):
            prof.setdefault(name, []).append(t)
    clk = clocks.stop()
    ms = reps.max(ms)
    status = sim.status()
    sim.close()

    kb = kernel_bytes(cfg)
    steps_prof = min(5, max(args.steps, 1))
    per_kernel = {k: sum(v) / steps_prof for k, v in prof.items()}
    step_prof_ms = sum(per_kernel.values())
    dom = max(per_kernel, key=per_kernel.get)
    dom_ms = statistics.mean(prof[dom])
    peak, peak_src = measured_peaks()
    achieved = kb.get(dom, 0) / (dom_ms * 1e-3) / 1e9
    step_bytes = sum(kb.get(k, 0) for k in per_kernel)
    N = cfg["shape"][0] * cfg["shape"][1] * cfg["shape"][2]

    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(cfg, world),
        "grid_point_steps_per_s": round(world * N / (ms * 1e-3), 1),
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": ncu_traffic(dom, cfg["shape"]),
                     "algorithmic_bytes_per_launch": kb.get(dom), "launch_ms": round(dom_ms, 4),
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "byte_model": "every array the kernel must read or write, counted once; spectra as the "
                                   "nx/2+1 columns used; rho0 read once and averaged to the staggered points "
                                   "in the kernel",
                     "frac_three_staggered_fields": (round((kb.get(dom, 0) + 2 * 4 * N) / (dom_ms * 1e-3) / 1e9 / peak, 4)
                                                     if dom == "x_vel" and not np.isscalar(cfg["rho0"]) else None)},
        "step_roofline": {"bytes_per_step": step_bytes, "achieved_gbs": round(step_bytes / (ms * 1e-3) / 1e9, 1),
                          "frac": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 4),
                          "frac_78_fields": round(78 * 4 * N / (ms * 1e-3) / 1e9 / peak, 4)},
        "kernels_ms": {k: round(v, 4) for k, v in sorted(per_kernel.items(), key=lambda kv: -kv[1])},
        "clocks": clk,
        "device_status": status,
    }

    if not args.no_e2e:
        out["e2e"] = e2e(args, cfg, kwgb, torch, reps)
    if not args.no_extra and args.config == 3 and args.n is None:
        out["mixed_f16"] = step_variant(args, kwgb, torch, 3, 8)
        out["mixed_bf16"] = step_variant(args, kwgb, torch, 3, 4)
        out["also_1024"] = step_variant(args, kwgb, torch, 4, 0)
        out["mixed_f16_1024"] = step_variant(args, kwgb, torch, 4, 8)
        out["mixed_bf16_1024"] = step_variant(args, kwgb, torch, 4, 4)
        out["linear_lossless_512"] = step_variant(args, kwgb, torch, 3, 0, _linear_lossless,
                                                  "float32, linear lossless (10 FFTs, EOS fused into x_dens)")
        out["homogeneous_512"] = step_variant(args, kwgb, torch, 3, 0, _homogeneous,
                                              "float32, homogeneous nonlinear absorbing (scalar medium)")
        out["adjoint"] = adjoint_measure(kwgb, torch)
    if not args.no_extra and world == 1:
        out["cufft_unfused"] = cufft_unfused(args, torch)
    if rank == 0 and world == 1 and not args.no_cpu:
        sec, per, cores = oracle_timed(args.config, args.n, 1, 2)
        out["cpu_baseline"] = {"value": round(1e3 * sec, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "FP64 oracle on the workload itself (%d^3 grid, medium, bowl source, "
                                         "sensors): 1 warm-up step, then 2 steps timed one by one (%.1f, %.1f s); "
                                         "host set-up not timed" % (cfg["shape"][0], per[0], per[1])}
    if rank == 0:
        print(json.dumps(out))
    reps.close()


def step_variant(args, kwgb, torch, cfg_id, extra_flags, modify=None, form=None):
    """Another workload or form, timed like the main line: the 1024^3 workload
    (same bowl and tissue recipe at 0.1 mm), the float16- / bfloat16-split
    tensor-core forms (extra_flags = 8 / 4) of the 512^3 workload, or a
    specialised medium (`modify` edits the configuration)."""
    cfg = inputs.make_config(cfg_id, n_steps=args.warmup + args.steps + 8)
    cfg["flags"] = cfg["flags"] | extra_flags
    if modify is not None:
        modify(cfg)
    sim, _ = kwgb.from_config(cfg)
    stream = torch.cuda.current_stream()
    sim.step(args.warmup, stream)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = {}
    for name, t in sim.step_profiled(stream):
        prof[name] = prof.get(name, 0.0) + t
    bytes_ = sum(kernel_bytes(cfg).get(k, 0) for k in prof)
    peak, _ = measured_peaks()
    form = form or {4: "bf16-split tensor-core y/z stages", 8: "f16-split tensor-core y/z stages"}.get(extra_flags, "float32")
    res = {"workload": workload_name(cfg), "form": form,
           "ms_per_step": round(ms, 3),
           "bytes_per_step": bytes_, "frac": round(bytes_ / (ms * 1e-3) / 1e9 / peak, 4),
           "device_gb": round(sim.device_bytes / 1e9, 2), "status": sim.status(),
           "kernels_ms": {k: round(v, 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1])}}
    sim.close()
    return res


def _linear_lossless(cfg):
    """Specialised step: linear, lossless (heterogeneous c0 and rho0 kept)."""
    cfg["flags"] = 0
    cfg["alpha0"] = 0.0
    cfg["bona"] = 0.0


def _homogeneous(cfg):
    """Specialised step: every medium property one scalar (soft tissue)."""
    cfg["c0"], cfg["rho0"], cfg["bona"] = 1540.0, 1040.0, 7.0
    cfg["alpha0"] = float(inputs.db_to_neper(0.75, cfg["alpha_power"]))
    cfg["c_ref"] = 1540.0


def adjoint_measure(kwgb, torch):
    """Forward + hand-written adjoint of the 256-element segmented bowl at 128^3
    (600 steps), two ways: checkpoints every 50 steps (the reverse pass
    recomputes each segment) and every step's density fields kept by the
    forward run (7 fields a step, 35 GB; nothing recomputed).  Time per step of
    each leg and device memory, beside the plain forward step of the same
    problem and the objective-only run (one forward run, no checkpoints)."""
    from paper_1408_4675_gb300.autograd import FocalProblem
    cfg = inputs.make_config(5)
    nt = int(cfg["n_steps"])

    def per_step(t0):
        return (time.perf_counter() - t0) * 1e3 / nt
    prob = FocalProblem(cfg, checkpoint_every=50)
    warm = prob.simulation(cfg["phases"], cfg["amps"])     # one-time set-up (kernel attributes, graph capture)
    warm.step(8)
    warm.close()
    sim = prob.simulation(cfg["phases"], cfg["amps"])
    sim.step(2)                                            # the step's graph is captured after the first step
    sim.status()
    t0 = time.perf_counter()
    sim.step(nt)
    sim.status()
    fwd = per_step(t0)
    sim.close()
    t0 = time.perf_counter()
    prob.objective(cfg["phases"], cfg["amps"])
    obj = per_step(t0)
    out = {"workload": "segmented_bowl_256_elements_128^3", "steps": nt,
           "forward_ms_per_step": round(fwd, 4), "objective_only_ms_per_step": round(obj, 4)}
    for name, K in (("checkpoint_every_50", 50), ("every_step_kept", nt)):
        prob = FocalProblem(cfg, checkpoint_every=K)
        t0 = time.perf_counter()
        J, sim = prob.forward(cfg["phases"], cfg["amps"])
        fwd_ck = per_step(t0)
        t1 = time.perf_counter()
        dphi, damp, _ = prob.backward(sim, cfg["phases"], cfg["amps"])
        bwd = per_step(t1)
        tot = per_step(t0)
        out[name] = {"checkpoint_every": K, "forward_ms_per_step": round(fwd_ck, 4),
                     "reverse_ms_per_step": round(bwd, 4), "forward_plus_adjoint_ms_per_step": round(tot, 4),
                     "ratio_to_forward": round(tot / fwd, 3), "device_gb": round(prob.last_device_bytes / 1e9, 3),
                     "J": J, "grad_norm_phases": float(np.linalg.norm(dphi))}
    return out


class CufftStep:
    """Comparator timed beside the library, not part of it: the same workload
    stepped by plain PyTorch ops -- 14 cuFFT 3-D real transforms per step
    (torch.fft.rfftn / irfftn), stored 3-D operator arrays (i k kappa
    exp(+-i k d/2) per axis, k^{y-2}, k^{y-1}) and one unfused kernel per
    element-wise operation: the direct GPU transcription of Eqs. 4a-4d, 6 and
    8 (readings as in the library: PML, staggered rho0, additive mass source,
    initial pressure).  Sensors: p_max and sum p^2 at each mask."""

    def __init__(self, cfg, device="cuda"):
        import torch
        self.t = torch
        self.dev = device
        nz, ny, nx = self.shape = tuple(cfg["shape"])
        self.dt = dt = float(cfg["dt"])
        y = float(cfg["alpha_power"])
        self.nonlinear = bool(cfg["flags"] & 1)
        self.absorbing = bool(cfg["flags"] & 2)
        f64 = dict(dtype=torch.float64, device=device)

        def field(v):
            a = torch.as_tensor(np.asarray(v, dtype=np.float32), device=device)
            return a.expand(nz, ny, nx).contiguous() if a.ndim == 0 else a.reshape(nz, ny, nx)

        self.c0, self.rho0, self.bona, self.alpha0 = (field(cfg[k]) for k in ("c0", "rho0", "bona", "alpha0"))

        def kvec(n, d, half=False):
            m = torch.arange(n // 2 + 1 if half else n, **f64)
            if not half:
                m = torch.where(m < n // 2, m, m - n)            # Eq. 5, Nyquist at -N/2
            return m * (2.0 * math.pi / (d * n))

        dx, dy, dz = cfg["d"]
        kx = kvec(nx, dx, True).reshape(1, 1, -1)
        ky = kvec(ny, dy).reshape(1, -1, 1)
        kz = kvec(nz, dz).reshape(-1, 1, 1)
        kmag = torch.sqrt(kx * kx + ky * ky + kz * kz)
        arg = float(cfg["c_ref"]) * kmag * dt / 2.0
        kappa = torch.where(arg > 0, torch.sin(arg) / torch.where(arg > 0, arg, 1.0), 1.0)
        self.Dp, self.Dm = [], []
        for k, d in ((kx, dx), (ky, dy), (kz, dz)):
            for sign, lst in ((1.0, self.Dp), (-1.0, self.Dm)):
                op = (1j * k) * torch.exp(sign * 1j * k * d / 2.0) * kappa
                lst.append(op.to(torch.complex64))
        if self.absorbing:
            safe = torch.where(kmag > 0, kmag, 1.0)
            self.tau_op = torch.where(kmag > 0, safe ** (y - 2.0), 0.0).float()
            self.eta_op = torch.where(kmag > 0, safe ** (y - 1.0), 0.0).float()
            c64, a64 = self.c0.double(), self.alpha0.double()
            self.tau = (-2.0 * a64 * c64 ** (y - 1.0)).float()
            self.eta = (2.0 * a64 * c64 ** y * math.tan(math.pi * y / 2.0)).float()
        del kmag, arg, kappa
        self.rho0_sg = [0.5 * (self.rho0 + torch.roll(self.rho0, -1, dims=a)) for a in (2, 1, 0)]

        def pml(n, size, alpha, d, stag):
            s = torch.arange(n, **f64) + (0.5 if stag else 0.0)
            if size <= 0:
                return torch.ones(n, **f64)
            depth = torch.clamp(torch.maximum(size - s, s - (n - 1 - size)), min=0.0)
            return torch.exp(-alpha * (float(cfg["c_ref"]) / d) * (depth / size) ** 4 * dt / 2.0)

        shp = [(1, 1, nx), (1, ny, 1), (nz, 1, 1)]
        ns, ds = (nx, ny, nz), (dx, dy, dz)
        self.f = [pml(ns[a], cfg["pml_size"][a], cfg["pml_alpha"][a], ds[a], False).float().reshape(shp[a])
                  for a in range(3)]
        self.fs = [pml(ns[a], cfg["pml_size"][a], cfg["pml_alpha"][a], ds[a], True).float().reshape(shp[a])
                   for a in range(3)]
        zeros = lambda: torch.zeros(self.shape, dtype=torch.float32, device=device)
        self.u = [zeros() for _ in range(3)]
        self.rho = [zeros() for _ in range(3)]
        self.p = zeros()
        if cfg.get("p0") is not None:
            p0 = field(cfg["p0"])
            self.p = p0.clone()
            self.rho = [p0 / (3.0 * self.c0 ** 2) for _ in range(3)]
            P = self.rfft(p0)
            self.u = [dt / (2.0 * self.rho0_sg[i]) * self.irfft(P * self.Dp[i]) for i in range(3)]
        c0f = self.c0.reshape(-1)
        self.src = []
        for idx, sig in cfg["sources"]:
            ii = torch.as_tensor(np.asarray(idx, dtype=np.int64), device=device)
            sg = torch.as_tensor(np.atleast_2d(np.asarray(sig, dtype=np.float32)), device=device)
            scale = dt * 2.0 / (3.0 * c0f[ii] * dx)
            self.src.append((ii, sg, scale))
        self.sens = []
        for idx, _ in cfg["sensors"]:
            n = nz * ny * nx if idx is None else len(idx)
            ii = None if idx is None else torch.as_tensor(np.asarray(idx, dtype=np.int64), device=device)
            self.sens.append((ii, torch.full((n,), -math.inf, device=device),
                              torch.zeros(n, dtype=torch.float64, device=device)))
        self.n = 0

    def rfft(self, a):
        return self.t.fft.rfftn(a, dim=(0, 1, 2))

    def irfft(self, a):
        return self.t.fft.irfftn(a, s=self.shape, dim=(0, 1, 2))

    def step(self, nsteps=1):
        t, dt = self.t, self.dt
        for _ in range(nsteps):
            P = self.rfft(self.p)                                                    # 1 FFT
            for i in range(3):
                g = self.irfft(P * self.Dp[i])                                       # Eq. 4a
                self.u[i] = self.fs[i] * (self.fs[i] * self.u[i] - dt * g / self.rho0_sg[i])   # Eq. 4b
            d = [self.irfft(self.rfft(self.u[i]) * self.Dm[i]) for i in range(3)]    # Eq. 4c
            for i in range(3):
                num = self.f[i] * (self.f[i] * self.rho[i] - dt * self.rho0 * d[i])
                self.rho[i] = num / (1.0 + 2.0 * dt * d[i]) if self.nonlinear else num      # Eq. 4d
            for ii, sg, scale in self.src:
                if self.n < sg.shape[-1]:
                    s = sg[:, self.n] if sg.shape[0] > 1 else sg[0, self.n]
                    add = scale * s
                    for i in range(3):
                        self.rho[i].view(-1).index_add_(0, ii, add)
            rho = self.rho[0] + self.rho[1] + self.rho[2]
            q = rho + (self.bona / 2.0) * rho * rho / self.rho0 if self.nonlinear else rho
            if self.absorbing:
                dsum = self.rho0 * (d[0] + d[1] + d[2])
                Ld = (-self.tau * self.irfft(self.tau_op * self.rfft(dsum))
                      + self.eta * self.irfft(self.eta_op * self.rfft(rho)))       # Eq. 8
                q = q - Ld
            self.p = self.c0 * self.c0 * q                                           # Eq. 6
            self.n += 1
            pf = self.p.reshape(-1)
            for ii, pm, p2 in self.sens:
                v = pf if ii is None else pf[ii]
                t.maximum(pm, v, out=pm)
                p2.add_(v.double() * v.double())


def cufft_unfused(args, torch):
    """Time CufftStep on the bench workload: ms per step with CUDA events."""
    cfg = inputs.make_config(args.config, n=args.n, n_steps=args.warmup + args.steps + 8)
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    try:
        st = CufftStep(cfg)
    except torch.cuda.OutOfMemoryError as e:
        return {"unavailable": "out of memory: %s" % str(e).splitlines()[0]}
    stream = torch.cuda.current_stream()
    st.step(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    peak_gb = torch.cuda.max_memory_allocated() / 1e9
    del st
    torch.cuda.empty_cache()
    return {"ms_per_step": round(ms, 3), "ffts_per_step": 14,
            "what": "same workload stepped by plain PyTorch CUDA ops: cuFFT 3-D R2C/C2R transforms, stored "
                    "3-D operator arrays, unfused element-wise kernels (comparator, not the library)",
            "peak_device_gb": round(peak_gb, 2)}


def e2e(args, cfg, kwgb, torch, reps):
    """The same metric through the public API with host buffers: set-up from
    pinned host arrays, K steps, and every sensor output read back, all inside
    the timed region (wall clock, synchronised; the slowest rank's time)."""
    def pinned(a):
        a = np.asarray(a, dtype=np.float32)
        t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()
    host = {k: (cfg[k] if np.ndim(cfg[k]) == 0 else pinned(cfg[k])) for k in ("c0", "rho0", "bona", "alpha0")}
    h2d = sum(v.nbytes for v in host.values() if not np.isscalar(v) and np.ndim(v) > 0)
    h2d += sum(idx.nbytes + 4 * np.size(sig) for idx, sig in cfg["sources"])
    h2d += sum(idx.nbytes for idx, _ in cfg["sensors"] if idx is not None)
    torch.cuda.synchronize()
    reps.barrier()
    t0 = time.perf_counter()
    sim = kwgb.Simulation(cfg["shape"], cfg["d"], cfg["dt"], cfg["c_ref"], cfg["pml_size"],
                          cfg["pml_alpha"], cfg["flags"], cfg["alpha_power"])
    sim.set_medium(host["c0"], host["rho0"], host["bona"], host["alpha0"])
    for idx, sig in cfg["sources"]:
        sim.add_source(idx, sig)
    ids = [sim.add_sensor(idx, rec) for idx, rec in cfg["sensors"]]
    sim.step(args.steps)
    d2h = 0
    for (idx, rec), i in zip(cfg["sensors"], ids):
        for which in (1, 2, 4):
            if rec & which:
                d2h += sim.read(i, which).nbytes
    t1 = time.perf_counter()
    sim.close()
    ms = reps.max(1e3 * (t1 - t0) / args.steps)
    return {"value": round(ms, 4), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d // args.steps), "d2h_bytes_per_step": int(d2h // args.steps),
            "what": "create + medium upload from pinned host memory + sources/sensors + %d steps + "
                    "read of every sensor output, per step" % args.steps}


def run_profile_case(args):
    """A small grid with the kernels of the benchmark (same row and line
    lengths along the transformed axes), for `ncu --set full` captures that
    must stay a few GB: smooth random c0, rho0, B/A, alpha0 (y = 1.1), a
    Gaussian initial pressure, a PML of 10 cells and a 9^3 sensor box."""
    import torch
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    shape = tuple(args.profile_case)
    d = 1e-4
    c0 = inputs.smooth_random_field(shape, 1450.0, 1650.0, 11, 3.0)
    rho0 = inputs.smooth_random_field(shape, 950.0, 1100.0, 12, 3.0)
    bona = inputs.smooth_random_field(shape, 5.0, 9.0, 13, 3.0)
    alpha0 = inputs.db_to_neper(inputs.smooth_random_field(shape, 0.3, 1.0, 14, 3.0), 1.1)
    c_ref = float(c0.max())
    sim = kwgb.Simulation(shape, (d, d, d), 0.3 * d / c_ref, c_ref, (10, 10, 10), (2.0, 2.0, 2.0),
                          flags=3 | args.profile_flags, alpha_power=1.1)
    sim.set_medium(c0, rho0, bona, alpha0)
    sim.set_initial_pressure(inputs.gaussian_ball(shape, 3.0, 1e5))
    sim.add_sensor(inputs.box_mask(shape, tuple(n // 2 for n in shape), 4), 3)
    sim.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": list(shape), "steps": args.steps, "status": sim.status()}))
    sim.close()


def run_oracle_table(args):
    """The CPU-baseline leg over every workload at its stated size: the FP64
    oracle on the host cores (one warm-up step, then configs 1 and 5 over
    their whole runs of 200 and 600 steps, config 2 over 20 steps and config 3
    over 5, each step timed), beside the GPU's event-timed step of the same
    workload (5 warm-up + 50 steps).  Config 4 is not run: its FP64 oracle
    state (about 480 GB at 1024^3) exceeds the host memory."""
    import torch
    from paper_1408_4675_gb300 import build, kwgb
    build.build()
    kwgb.load()
    rows = []
    for cid, steps in ((1, 200), (5, 600), (2, 20), (3, 5)):
        sec, per, cores = oracle_timed(cid, None, 1, steps)
        gpu = step_variant(SimpleNamespace(warmup=5, steps=50), kwgb, torch, cid, 0)
        rows.append({"config": cid, "workload": gpu["workload"], "oracle_steps": steps,
                     "oracle_ms_per_step": round(1e3 * sec, 2), "oracle_cores": cores,
                     "gpu_ms_per_step": gpu["ms_per_step"],
                     "oracle_over_gpu": round(1e3 * sec / gpu["ms_per_step"], 1)})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"oracle_table": rows,
                      "not_run": {"config": 4, "why": "FP64 oracle state at 1024^3 (about 480 GB) exceeds the "
                                                     "host memory"}}))


def run_profile_adjoint(args):
    """The adjoint of the segmented bowl (256 elements) on an N^3 grid for
    `ncu` launch lists: one forward run of STEPS steps keeping every step's
    fields, then the reverse pass."""
    from paper_1408_4675_gb300 import build, kwgb
    from paper_1408_4675_gb300.autograd import FocalProblem
    build.build()
    kwgb.load()
    n, steps = args.profile_adjoint
    cfg = inputs.make_config(5, n=n, n_steps=steps)
    prob = FocalProblem(cfg, n_steps=steps, checkpoint_every=steps)
    J, dphi, damp, _ = prob.value_and_grad(cfg["phases"], cfg["amps"])
    print(json.dumps({"profile_adjoint": [n, steps], "J": J, "grad_norm_phases": float(np.linalg.norm(dphi))}))


def main():
    args = parse()
    if args.profile_adjoint is not None:
        run_profile_adjoint(args)
        return
    if args.oracle_table:
        run_oracle_table(args)
        return
    if args.profile_case is not None:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
