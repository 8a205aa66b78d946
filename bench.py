#!/usr/bin/env python
"""Throughput of the SPH terrain step on B300: active SPH particle-steps per second.

Workload: the single grousered wheel on a soil bin -- 120,000 SPH particles on a
2.0 x 0.4 x 0.15 m bin at d0 = 0.01 m (h = 1.2 d0), 3-layer BCE walls, a rigid
wheel (r = 0.2 m, width 0.15 m, 12 grousers 0.01 m tall) with prescribed spin and
slip 0.3 and a free vertical DOF under a 100 N load, friction 33 deg, cohesion
500 Pa, dt = 5e-5 s, exact 2h neighbour sets at every step (ps_freq = 1).
Synthetic, seeded inputs (scenes.wheel_bin).

One step = the whole per-step path: the search decision, BCE extrapolation and
pair sums for both RK2 stages, return map, FP64 wrench and body update.  With the
default Verlet skin (0.1) the cell sort and 27-cell search (keys, scan, scatter,
reorder, radius 2h (1 + skin)) run only in the steps where the device-side skin
test calls for them -- a few per hundred steps here, amortised over the timed
steps and counted in `cell_searches` -- while every step's first stage filters
the skin lists to that step's exact 2h sets.  `--skin 0` times the literal every-
step rebuild of Alg. 2 instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl crm|reference]

The line also carries the adjoint measurement on the differentiable wheel test
(30,000 SPH particles, 400 steps): recorded forward, reverse sweep, their ratio to
the plain forward step, the gradients, and as its CPU baseline the oracle's own
FP64 adjoint timed over a few steps on the host cores.

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the workload ("replicas only": the method has no exchange step on
one terrain here), so value = all ranks' particle-steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "active SPH particle-steps/sec on 1 B300"
UNIT = "particle-steps/s"
WORKLOAD = ("wheel_bin: 120,000 SPH particles, 2.0x0.4x0.15 m bin at d0=0.01 m, h=1.2 d0, "
            "3-layer BCE walls + grousered wheel (r=0.2 m, 12 grousers), slip 0.3, 100 N, "
            "phi=33 deg, c=500 Pa, dt=5e-5 s, ps_freq=1")
# Arithmetic of one fluid-fluid or fluid-marker pair in the pair kernel, counted
# from its source (FMA = 2): offsets 6, r^2 5, rsqrt/scale 3, dW/dr 5, V_j 1,
# f V_j 1, V_j grad W 3, u_ji 3, sum of V_j grad W 3, sigma_j . V_j grad W 18,
# velocity gradient 18 (continuity is its trace), artificial viscosity 18 => 84;
# per particle: sigma_i . sum V_j grad W and the trace 20, stress rate, update
# and return map ~100 => 120.
FLOP_PER_PAIR = 84
FLOP_PER_PARTICLE = 120
SM_FP32_LANES = 128
BODY_BYTES = 352   # one body's device record, copied out by the exchange


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        self.f.close()
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(world: int, times, units: float, device=None):
    """Cross-rank reduction of one run: each timing is the maximum over ranks (the
    job lasts as long as its slowest replica) and the units (particle-steps) are
    summed over ranks.  Returns (times, total units)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in times], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return [float(v) for v in t], float(u[0])


def cpu_baseline(budget_s: float = 15.0) -> dict:
    """The FP64 oracle as it stands, on this host's cores, on a bounded sample of
    the same workload: as many whole steps as fit in ~budget_s (at least 2)."""
    import oracle
    import scenes
    sc = scenes.wheel_bin()
    st = oracle.State(sc)
    t0 = time.perf_counter()
    n = 0
    while n < 2 or time.perf_counter() - t0 < budget_s:
        st.step()
        n += 1
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # the same oracle on one thread, a shorter sample continuing the same run
    prev = oracle.set_threads(1)
    try:
        t1 = time.perf_counter()
        n1 = 0
        while n1 < 1 or time.perf_counter() - t1 < budget_s / 3:
            st.step()
            n1 += 1
        el1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(prev)
    return {"value": sc.n_fluid * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"wheel_bin workload, first {n} whole steps ({el:.1f} s, FP64, OpenMP), "
                      f"cpu={_cpu_model()}",
            "single_thread": {"value": sc.n_fluid * n1 / el1, "unit": UNIT, "cores": 1,
                              "sample": f"the next {n1} whole steps ({el1:.1f} s)"}}


def cpu_baseline_strip(budget_s: float = 15.0) -> dict:
    """The FP64 oracle on the active-domain strip's 20 m window around the rover
    (the oracle integrates the Active particles of Alg. 3 only, as the library
    does): whole steps within ~budget_s, as active particle-steps per second."""
    import oracle
    import scenes
    sc = scenes.strip(x_window=(4990.75, 5010.75))
    st = oracle.State(sc)
    t0 = time.perf_counter()
    n, units = 0, 0
    while n < 2 or time.perf_counter() - t0 < budget_s:
        st.step()
        units += int((st.flags == 2).sum())
        n += 1
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": units / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"strip, 20 m window at x = 5000 m ({sc.n_fluid:,} SPH stored), first {n} "
                      f"whole steps ({el:.1f} s, FP64, OpenMP), cpu={_cpu_model()}"}


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    """Reference arm: the FP64 oracle, one whole step of the workload per step."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    import scenes
    sc = scenes.wheel_bin()
    st = oracle.State(sc)
    for _ in range(args.warmup):
        st.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.step()
    el = time.perf_counter() - t0
    value = sc.n_fluid * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_sph": sc.n_fluid, "n_bce": sc.n_markers,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"wheel_bin workload, {args.steps} whole steps after "
                                       f"{args.warmup} warm-up, cpu={_cpu_model()}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


KERNEL_SOURCE = {"pair_stage1": "crm_step.cu", "pair_stage2": "crm_step.cu", "bce": "crm_bce.cu",
                 "compact": "crm_bce.cu", "skin": "crm_bin.cu", "keys": "crm_bin.cu",
                 "scan": "crm_bin.cu", "scatter": "crm_bin.cu", "reorder": "crm_bin.cu",
                 "neighbors": "crm_bin.cu", "export": "crm_step.cu"}


def _traffic(kernel: str, captured: bool = True):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.txt: kernel, bytes per launch, sha256[:16] of the source
    file the kernel lives in followed by the shared device header, when it was
    captured), if it was taken on the
    current source (else None).  captured: the line's workload is the one the
    summary was captured on (the wheel bin); on any other the figure does not
    apply and None is returned."""
    if not captured:
        return None
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    csrc = os.path.join(ROOT, "paper_2507_05643_b300", "csrc")
    h = hashlib.sha256()
    for f in (KERNEL_SOURCE.get(kernel, "crm_step.cu"), "crm_internal.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    h = h.hexdigest()[:16]
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = ln.split()
        if len(f) >= 3 and not ln.startswith("#") and f[0] == kernel and f[2] == h:
            return float(f[1])
    return None


def dominant_kernel(per_launch_ms: dict, workload: str) -> str:
    """The kernel id the roofline is quoted for: the single kernel with the largest
    share of the event-timed step, taken as the largest time per launch -- an id
    that counts several kernels (bce: the two marker-state passes, the wrench pass
    and the body update) is not one kernel, and its per-step total is a sum of four.
    With active domains and the skin (the strip), only the kernels that work at
    every step compete: the gated gather and search kernels are launched every step
    in the direct-launch pass but mostly return at once."""
    every = ("pair_stage1", "pair_stage2", "bce") if workload == "strip" else tuple(per_launch_ms)
    return max((k for k in per_launch_ms if k in every), key=lambda k: per_launch_ms[k])


def _workload(args):
    """The benchmark workload; --bin-scale S > 1 widens the bin S-fold in x and y
    (a profiling case larger than L2, not a bench line); --workload strip runs the
    active-domain strip (a window of --strip-length m around the rover at
    x = 5000 m; 10000 = the whole 10 km strip)."""
    import scenes
    if args.workload == "strip":
        half = args.strip_length / 2
        win = None if args.strip_length >= 1.0e4 else (5000.75 - half, 5000.75 + half)
        return scenes.strip(x_window=win)
    if args.bin_scale == 1:
        return scenes.wheel_bin()
    s = args.bin_scale
    return scenes.wheel_bin(nx=200 * s, ny=40 * s, wheel_x=0.4 * s)


def adj_workload(n_steps: int = 400, every: int = 20) -> str:
    half = n_steps // 2
    return ("differentiable wheel test: 30,000 SPH particles, 1.0x0.3x0.1 m bin at d0=0.01 m, "
            f"the wheel_bin wheel and material, skin 0, ps_freq=1, {n_steps} steps of 5e-5 s, "
            f"checkpoint every {every}; J = mean over steps {half + 1}-{n_steps} of drawbar "
            "pull F_x and of sinkage z0 - z")


def _adjoint_scene():
    import scenes
    sc = scenes.wheel_bin(seed=3, nx=100, ny=30, nz=10)
    sc.params["skin"] = 0.0
    return sc


def _adjoint_objectives(n_steps: int, nb: int = 1):
    """dJ/d wrench and dJ/d centre of the two objectives (mean drawbar pull F_x and
    mean sinkage z0 - z over the second half of the run)."""
    import numpy as np
    half = n_steps // 2
    lw_dp = np.zeros((n_steps, nb, 6))
    lw_dp[half:, 0, 0] = 1.0 / (n_steps - half)
    lc_sink = np.zeros((n_steps, nb, 3))
    lc_sink[half:, 0, 2] = -1.0 / (n_steps - half)
    return {"drawbar_pull": (lw_dp, None), "sinkage": (None, lc_sink)}


def _phi_grads(g, mu_s: float, body=None) -> dict:
    """(phi [rad], c, E, rho0) from the library's parameter gradients, mu_s = tan phi;
    with the wheel's body gradients also its prescribed forward speed and spin."""
    out = {"phi": g["mu_s"] * (1.0 + mu_s * mu_s), "cohesion": g["cohesion"], "E": g["E"],
           "rho0": g["rho0"]}
    if body is not None:
        out["speed_x"] = float(body[3])      # d J / d v_x (prescribed forward speed)
        out["omega_y"] = float(body[13])     # d J / d w_y (prescribed spin)
    return out


def _oracle_adjoint_sample(sc, n: int) -> dict:
    """The oracle's own FP64 adjoint (autograd over its PyTorch CPU restatement of
    the step) timed on the host cores over the first n steps of the same test:
    forward with the tape, then the reverse sweep of the drawbar-pull objective."""
    import numpy as np
    import torch

    from oracle import adjoint as oadj
    r = oadj.Run(sc, "cells")
    t0 = time.perf_counter()
    r.forward(sc.dt, n)
    t1 = time.perf_counter()
    lw = np.zeros((n, 1, 6))
    lw[:, 0, 0] = 1.0 / n
    r.backward(lw)
    t2 = time.perf_counter()
    return {"value": 1e3 * (t2 - t1) / n, "unit": "ms per step of the reverse sweep",
            "forward_ms_per_step": 1e3 * (t1 - t0) / n, "cores": torch.get_num_threads(),
            "kind": "oracle", "what": "the oracle's own FP64 adjoint (autograd, CPU)",
            "sample": f"the first {n} steps of the differentiable wheel test"}


def adjoint_line(stream, dev, n_steps: int = 400, every: int = 20, fd: bool = False,
                 oracle_steps: int = 0) -> dict:
    """Adjoint cost against the forward step on the differentiable wheel test, and
    the gradients of both objectives (optionally against FP64 central differences
    of the oracle, relative step 1e-4, lists rebuilt as the oracle does)."""
    import numpy as np
    import torch

    import paper_2507_05643_b300 as crm
    sc = _adjoint_scene()
    dt = sc.dt
    with torch.cuda.stream(stream):
        # plain forward: graph-replayed steps, CUDA events on the library's stream
        t = crm.from_scene(sc, stream=stream)
        t.step(dt, 4)            # commit, graph capture, warm-up
        t.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        t.step(dt, n_steps)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        fwd_ms = ev[0].elapsed_time(ev[1]) / n_steps
        t.close()
        t = crm.from_scene(sc, stream=stream)
        # the initial state, to record the same run again with the tape allocated
        nbytes = t.state_bytes()
        init = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        used = t.save_state(init.data_ptr(), nbytes)
        w0 = time.perf_counter()
        t.adjoint_forward(dt, n_steps, every)       # allocates the tape and checkpoints
        first_s = time.perf_counter() - w0
        t.load_state(init.data_ptr(), used)
        w0 = time.perf_counter()
        wr, pose = t.adjoint_forward(dt, n_steps, every)
        rec_s = time.perf_counter() - w0
        grads, bwd_s = {}, []
        for name, (lw, lc) in _adjoint_objectives(n_steps).items():
            w0 = time.perf_counter()
            g = t.adjoint_backward(lw, lc)
            bwd_s.append(time.perf_counter() - w0)
            grads[name] = _phi_grads(g["param_grads"], sc.params["mu_s"], g["body"][0])
        prof = t.profile()
        # the same run with the whole tape resident in HBM (no checkpoints, no re-run)
        t.load_state(init.data_ptr(), used)
        w0 = time.perf_counter()
        t.adjoint_forward(dt, n_steps, 0)           # allocates the resident tape
        first_res = time.perf_counter() - w0
        t.load_state(init.data_ptr(), used)
        w0 = time.perf_counter()
        t.adjoint_forward(dt, n_steps, 0)
        rec_res = time.perf_counter() - w0
        lw, lc = _adjoint_objectives(n_steps)["drawbar_pull"]
        w0 = time.perf_counter()
        g_res = t.adjoint_backward(lw, lc)
        bwd_res = time.perf_counter() - w0
        t.close()
    half = n_steps // 2
    out = {
        "workload": adj_workload(n_steps, every), "n_sph": sc.n_fluid, "n_bce": sc.n_markers,
        "forward_ms_per_step": fwd_ms,
        "recorded_forward_ms_per_step": 1e3 * rec_s / n_steps,
        "first_recording_s": first_s,
        "backward_ms_per_step": 1e3 * statistics.mean(bwd_s) / n_steps,
        "adjoint_over_forward": 1e3 * statistics.mean(bwd_s) / n_steps / fwd_ms,
        "objectives": {"drawbar_pull_N": float(wr[half:, 0, 0].mean()),
                       "sinkage_m": float((sc.bodies[0].pose[2] - pose[half:, 0, 2]).mean())},
        "gradients": grads,
        "gradient_units": "per rad (phi), per Pa (cohesion, E), per kg/m^3 (rho0), per m/s "
                          "(speed_x), per rad/s (omega_y)",
        "adjoint_launches": prof["launches"].get("adjoint", 0),
        "resident_tape": {
            "recorded_forward_ms_per_step": 1e3 * rec_res / n_steps,
            "first_recording_s": first_res,
            "backward_ms_per_step": 1e3 * bwd_res / n_steps,
            "adjoint_over_forward": 1e3 * bwd_res / n_steps / fwd_ms,
            "drawbar_pull_grad_phi": g_res["param_grads"]["mu_s"] * (1.0 + sc.params["mu_s"] ** 2),
            "form": "crm_adjoint_forward(every = 0): every step's tape kept in HBM"},
        "timing": "forward: CUDA events over the graph-replayed steps; recording and backward: "
                  "host wall time of crm_adjoint_forward (its second call, tape allocated) and "
                  "crm_adjoint_backward (re-run of every segment + reverse sweep)",
    }
    if oracle_steps > 0:
        out["cpu_baseline"] = _oracle_adjoint_sample(sc, oracle_steps)
    if fd:
        out["fd_check"] = _adjoint_fd(sc, n_steps, grads)
    return out


def _adjoint_fd(sc, n_steps: int, grads: dict, rels=(1e-4, 1e-6)) -> dict:
    """FP64 central differences of both objectives with the oracle at relative
    steps `rels` (mu_2 follows mu_s).  The objectives are piecewise smooth (each
    particle's return-map case can switch), so a difference converges to the
    derivative only once the step is below the nearest switch."""
    import math

    import numpy as np

    import oracle
    half = n_steps // 2
    dt = sc.dt
    z0 = sc.bodies[0].pose[2]

    def run(params, twist=None):
        s2 = sc.copy()
        s2.params = params
        if twist is not None:
            s2.bodies[0].twist = twist
        st = oracle.State(s2)
        fx, z = [], []
        for _ in range(n_steps):
            st.step(dt)
            fx.append(st.bodies.wrench[0, 0])
            z.append(st.bodies.pose[0, 2])
        return {"drawbar_pull": float(np.mean(fx[half:])), "sinkage": float(np.mean(z0 - np.array(z[half:])))}

    res = {}
    phi = math.atan(sc.params["mu_s"])
    for rel in rels:
        for name in ("phi", "cohesion", "E", "rho0", "speed_x", "omega_y"):
            pp, pm = dict(sc.params), dict(sc.params)
            tp = tm = None
            if name == "phi":
                e = rel * phi
                pp["mu_s"] = pp["mu_2"] = math.tan(phi + e)
                pm["mu_s"] = pm["mu_2"] = math.tan(phi - e)
            elif name in ("speed_x", "omega_y"):
                k = 0 if name == "speed_x" else 4
                e = rel * abs(sc.bodies[0].twist[k])
                tp, tm = sc.bodies[0].twist.copy(), sc.bodies[0].twist.copy()
                tp[k] += e
                tm[k] -= e
            else:
                e = rel * abs(sc.params[name])
                pp[name] += e
                pm[name] -= e
            jp, jm = run(pp, tp), run(pm, tm)
            for obj in ("drawbar_pull", "sinkage"):
                fdv = (jp[obj] - jm[obj]) / (2 * e)
                res.setdefault(f"step {rel:g}", {}).setdefault(obj, {})[name] = {
                    "adjoint": grads[obj][name], "fd": fdv,
                    "rel_err": abs(grads[obj][name] - fdv) / max(abs(fdv), 1e-300)}
    return res


def run_adjoint(args):
    """--workload adjoint: the adjoint measurement alone (a profiling and
    diagnostics line; the default line carries the same object)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    adj = adjoint_line(stream, dev, n_steps=args.adjoint_steps, fd=args.adjoint_fd,
                       oracle_steps=args.oracle_adjoint_steps)
    line = {"metric": "adjoint step cost / forward step cost", "value": adj["adjoint_over_forward"],
            "unit": "ratio", "n_gpus": 1, "steps": args.adjoint_steps, "warmup": 4,
            "ms_per_step": adj["backward_ms_per_step"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": adj["workload"]},
            "adjoint": adj}
    print(json.dumps(line), flush=True)


def _oracle_sample(scs, budget_s: float) -> dict:
    """The FP64 oracle on a bounded sample of a workload: whole steps of each scene
    in `scs` (at least 2 each) within ~budget_s, as particle-steps per second."""
    import oracle
    done, el = 0, 0.0
    per = budget_s / max(len(scs), 1)
    parts = []
    for sc in scs:
        st = oracle.State(sc)
        t0 = time.perf_counter()
        n = 0
        while n < 2 or time.perf_counter() - t0 < per:
            st.step()
            n += 1
        e = time.perf_counter() - t0
        done += sc.n_fluid * n
        el += e
        parts.append(f"{sc.n_fluid:,} SPH x {n} steps")
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{'; '.join(parts)} ({el:.1f} s, FP64, OpenMP), cpu={_cpu_model()}"}


def run_batch(args):
    """The batched ensemble (64 single-wheel bins of uneven size) after a
    per-member autotune (lanes x cell tile), stepped by crm_batch_step in its
    stream form (each member's step graph on its own stream; the library's
    default and the faster form here) -- the headline -- and in its persistent
    form (one graph per batch step, one launch per stage over all bins), against
    the same members stepped one at a time (the per-instance form)."""
    import numpy as np
    import torch

    import paper_2507_05643_b300 as crm
    import scenes

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    bins = scenes.ensemble_bins(n=args.batch_n)
    streams = [torch.cuda.Stream(device=dev) for _ in bins]
    mem = [crm.from_scene(sc, stream=st) for sc, st in zip(bins, streams)]
    dts = [sc.dt for sc in bins]
    main = torch.cuda.Stream(device=dev)
    batch = crm.Batch(mem, stream=main)
    picks = batch.autotune(dts, trial_steps=3)

    def timed(persistent: bool):
        batch.set_persistent(persistent)
        batch.step(dts, args.warmup)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(main):
            e0.record(main)
            batch.step(dts, args.steps)
            e1.record(main)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    ms_pers = timed(True)
    sampler = ClockSampler(0)
    ms_b = timed(False)
    clocks = sampler.stop()
    n_act = sum(m.counts()[0] for m in mem)
    # per-instance form: each member alone, one after the other
    ms_s = 0.0
    for m, st, dt in zip(mem, streams, dts):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(st)
        m.step(dt, args.steps)
        b.record(st)
        torch.cuda.synchronize(dev)
        ms_s += a.elapsed_time(b)
    units = n_act * args.steps
    lanes = picks & 0xF
    tile = [f"{(p >> 4) & 0xF}x{(p >> 8) & 0xF}x{(p >> 12) & 0xF}" for p in picks.tolist()]
    line = {"metric": METRIC, "value": units / (ms_b * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"ensemble: {len(bins)} single-wheel bins, 0.3 m wide, "
                                   f"{min(b.n_fluid for b in bins):,}-{max(b.n_fluid for b in bins):,} "
                                   f"SPH each ({sum(b.n_fluid for b in bins):,} in total), slip "
                                   "U(0.1,0.7), friction U(25,40) deg, cohesion U(0,2000) Pa, "
                                   "dt=5e-5 s, one batched step per step",
                       "form": "streams: each member's step graph on its own stream",
                       "l2": "not flushed: the ensemble's working set (~10 GB) exceeds L2",
                       "pair_lanes": {str(k): int((lanes == k).sum()) for k in (1, 2, 4)},
                       "cell_tiles": {k: tile.count(k) for k in sorted(set(tile))}},
            "persistent": {"value": units / (ms_pers * 1e-3), "ms_per_step": ms_pers / args.steps,
                           "form": "one graph per batch step: every member's gated search, "
                                   "then one persistent launch per stage over all bins"},
            "sequential": {"value": units / (ms_s * 1e-3), "ms_per_step": ms_s / args.steps,
                           "form": "the same members stepped one at a time"},
            "batched_over_sequential": ms_s / ms_b,
            "persistent_over_streams": ms_b / ms_pers,
            "gpu_launches": sum(m.profile()["launches"][k] for m in mem
                                for k in m.profile()["launches"]),
            "clocks": clocks}
    if not args.no_cpu_baseline:
        sizes = [b.n_fluid for b in bins]
        order = np.argsort(sizes)
        pick3 = [bins[int(order[0])], bins[int(order[len(order) // 2])], bins[int(order[-1])]]
        line["cpu_baseline"] = _oracle_sample(pick3, args.cpu_seconds)
        line["cpu_baseline"]["sample"] = ("smallest, median and largest bins: "
                                          + line["cpu_baseline"]["sample"])
    print(json.dumps(line), flush=True)
    batch.close()


def run_crm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2507_05643_b300 as crm
    import scenes

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sc = _workload(args)
    over = {}
    if args.skin is not None:
        over["skin"] = args.skin
    if args.ps_freq != 1:
        over["ps_freq"] = args.ps_freq
    t = crm.from_scene(sc, stream=stream, **over)
    dt = sc.dt
    warmup = args.warmup
    if args.workload == "strip":
        # past the first shrink test of the active arrays (Sec. 3.2: every S_I = 50
        # steps), a one-time resize of the first capacity estimate
        warmup = max(warmup, int(sc.params.get("shrink_interval", 50)) + 1)
    with torch.cuda.stream(stream):
        t.step(dt, warmup)
        t.sync()
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        t.profile_reset(timing=False)
        sampler = ClockSampler(local)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            t.step(dt, 1)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        clocks = sampler.stop()
        t.sync()
        launches = t.profile()
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        # kernel-level breakdown: the same steps with every launch bracketed by
        # CUDA events on the library's stream (direct launches, not the graph)
        prof_steps = min(args.steps, 50)
        t.profile_reset(timing=True)
        for k in range(prof_steps):
            flush.fill_(k & 0xFF)
            t.step(dt, 1)
        prof = t.profile()
        t.profile_reset(timing=False)
    n_active, n_ext, n_bce = t.counts()
    # neighbour pairs of the current exact lists (fluid rows, then all rows)
    off, _ = t.neighbors()
    fluid_pairs = int(off[sc.n_fluid] - off[0])
    all_pairs = int(off[-1])

    # end to end through the public API: per step the co-simulation exchange of
    # Sec. 2.4 -- the bodies' pose/twist host->device, step, wrench + body state
    # device->host, one synchronous call (crm_cosim_step, pinned staging)
    pose, twist = t.body_state(0)
    nb = t.n_bodies
    hpose = np.tile(pose, (nb, 1))
    htwist = np.tile(twist, (nb, 1))
    for b in range(nb):
        hpose[b], htwist[b] = t.body_state(b)
    e2e_steps = max(args.steps, 1)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    w0 = time.perf_counter()
    out = (np.zeros((nb, 6)), np.zeros((nb, 7)), np.zeros((nb, 6)))
    for _ in range(e2e_steps):
        W, P, V = t.cosim_step(dt, 1, hpose, htwist, out=out)
        hpose[:], htwist[:] = P, V     # the multibody side's next motion (here: the same)
    e2e_s = time.perf_counter() - w0
    t.sync()

    # max over ranks of the timings, sum of the active particle-steps
    (ms_max, e2e_max), units = aggregate(world, [ms, e2e_s], n_active * args.steps, dev)
    if rank == 0:
        peaks, kind = _peaks()
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        n_all = sc.n_fluid + sc.n_markers
        per = {k: prof["ms"][k] / max(prof["launches"][k], 1) for k in prof["ms"]
               if prof["launches"][k]}
        kern = dominant_kernel(per, args.workload)
        avg_ms = per[kern]
        # the ncu DRAM bytes in profiles/ were captured on the wheel bin as quoted
        same_case = args.workload == "wheel_bin" and args.bin_scale == 1 and args.ps_freq == 1
        fp32_peak = nsm * SM_FP32_LANES * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        n_f, n_m = sc.n_fluid, sc.n_markers
        if args.workload == "strip":   # the working set, not the stored terrain
            n_f, n_m = n_active + n_ext, n_bce
            n_all = n_f + n_m
        alg_bytes = {   # algorithmic DRAM bytes per launch (state read / written once)
            "keys": 40 * n_all, "scan": 8 * (2 * 60000 + 1), "scatter": 12 * n_all,
            "reorder": 2 * 60 * n_all, "neighbors": 20 * n_all + 4 * all_pairs * 1.33,
            "skin": 60 * n_all, "compact": 12 * n_m,
            "bce": 56 * 2 * n_m + 4 * (all_pairs - fluid_pairs),
            "pair_stage1": 56 * 2 * n_f + 56 * n_m + 4 * fluid_pairs,
            "pair_stage2": 56 * 3 * n_f + 56 * n_m + 4 * fluid_pairs,
            "export": 88 * n_f}
        if kern.startswith("pair"):
            flop = fluid_pairs * FLOP_PER_PAIR + n_active * FLOP_PER_PARTICLE
            achieved = flop / (avg_ms * 1e-3) / 1e12
            roof = {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                    "peak_source": f"{nsm} SMs x {SM_FP32_LANES} FP32 lanes x 2 x "
                                   f"{peaks['sm_max_mhz']:.0f} MHz ({kind} max clock)",
                    "traffic": _traffic(kern, same_case), "flop_per_launch": flop, "ms_per_launch": avg_ms}
        else:
            b = alg_bytes.get(kern, 0.0)
            achieved = b / (avg_ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": kern, "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "peak_source": f"hbm_gbs ({kind})",
                    "traffic": _traffic(kern, same_case), "bytes_per_launch": b, "ms_per_launch": avg_ms}
        pair_ms = per.get("pair_stage2", 0.0)
        pair_fp32 = ((fluid_pairs * FLOP_PER_PAIR + n_f * FLOP_PER_PARTICLE)
                     / (pair_ms * 1e-3) / 1e12 / fp32_peak) if pair_ms else None
        line = {
            "metric": METRIC,
            "value": units / (ms_max * 1e-3),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_sph": sc.n_fluid, "n_active": n_active,
                       "n_bce": n_bce, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write outside the events)"},
            "e2e": {"value": units * e2e_steps / args.steps / e2e_max, "unit": UNIT,
                    "h2d_bytes_per_step": 13 * 8 * nb, "d2h_bytes_per_step": BODY_BYTES * nb + 4,
                    "loop": "crm_cosim_step: bodies' pose/twist in, one step, every body's "
                            "state and wrench out, one synchronisation per step"},
            "gpu_launches": sum(launches["launches"].values()),
            "kernels_us_per_step": {k: 1e3 * prof["ms"][k] / max(prof["steps"], 1)
                                    for k in per},
            "kernel_launches_per_step": {k: prof["launches"][k] / max(prof["steps"], 1)
                                         for k in per},
            "cell_searches": launches["launches"]["neighbors"],
            "pair_stage2_fp32_frac": pair_fp32,
            # the pair kernels against the other roof: DRAM bytes per launch (ncu,
            # profiles/traffic.txt) over the event-timed launch
            "pair_hbm": {k: {"traffic": _traffic(k), "ms_per_launch": per[k],
                             "achieved_gbs": _traffic(k) / (per[k] * 1e-3) / 1e9,
                             "frac": _traffic(k) / (per[k] * 1e-3) / 1e9 / peaks["hbm_gbs"]}
                         for k in ("pair_stage1", "pair_stage2")
                         if per.get(k) and _traffic(k, same_case)},
            "roofline": roof,
            "clocks": clocks,
        }
        if args.bin_scale != 1:
            line["config"]["workload"] = f"profiling case: wheel_bin widened {args.bin_scale}x in x and y"
        if args.ps_freq != 1:
            line["config"]["workload"] = WORKLOAD.replace("ps_freq=1", f"ps_freq={args.ps_freq}")
        if args.workload == "strip":
            line["config"]["workload"] = (
                f"strip: {args.strip_length:g} m of the 10 km x 2 m x 0.1 m strip at d0=0.025 m "
                f"({sc.n_fluid:,} SPH stored), four-wheel rover at x=5000 m, 1 m/s, 1 m active "
                f"boxes, dt=1e-4 s")
        line["config"]["skin"] = args.skin if args.skin is not None else 0.1
        if not args.no_adjoint and args.workload == "wheel_bin" and args.bin_scale == 1:
            line["adjoint"] = adjoint_line(
                stream, dev, n_steps=args.adjoint_steps, fd=args.adjoint_fd,
                oracle_steps=0 if args.no_cpu_baseline or world > 1 else args.oracle_adjoint_steps)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = (cpu_baseline_strip(args.cpu_seconds) if args.workload == "strip"
                                    else cpu_baseline(args.cpu_seconds))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["crm", "reference"], default="crm")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skin", type=float, default=None,
                    help="Verlet skin as a fraction of 2h (default: the library's 0.1)")
    ap.add_argument("--ps-freq", type=int, default=1,
                    help="neighbour-list rebuild period (Alg. 2); the workload is quoted at 1")
    ap.add_argument("--workload", choices=["wheel_bin", "strip", "batch", "adjoint"],
                    default="wheel_bin",
                    help="strip: the 10 km active-domain strip; batch: the 64-bin ensemble; "
                         "adjoint: the adjoint measurement alone (not the headline line)")
    ap.add_argument("--batch-n", type=int, default=64, help="bins in the batched ensemble")
    ap.add_argument("--strip-length", type=float, default=20.0,
                    help="length in m of the strip window around the rover")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint-cost measurement on the differentiable wheel test")
    ap.add_argument("--adjoint-steps", type=int, default=400,
                    help="steps of the differentiable wheel test (the test is quoted at 400)")
    ap.add_argument("--oracle-adjoint-steps", type=int, default=2,
                    help="steps of the differentiable wheel test over which the oracle's own "
                         "FP64 adjoint is timed on the host cores (0: skip; ~6 s per step)")
    ap.add_argument("--adjoint-fd", action="store_true",
                    help="also check its gradients against FP64 central differences of the "
                         "oracle (about 8 oracle runs of 400 steps)")
    ap.add_argument("--bin-scale", type=int, default=1,
                    help="profiling only: widen the bin S-fold in x and y")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_crm(args)


if __name__ == "__main__":
    main()
