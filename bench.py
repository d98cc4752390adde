"""Benchmark of the coupled power-law / Cahn-Hilliard D2Q9 step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--nx NX]

One step = one time step of the whole lattice (Sec. 2.2-2.3 of arXiv
2207.09431: moments, chemical potentials, gradients, velocity and pressure,
power-law relaxation time, collision of g and h, streaming with bounce-back).
Workload: the rising-bubble set-up at 2048 x 4096 (R = 256, density ratio
1000, n = 0.7, Eo = 10), synthetic and seeded.  The state (about 1.3 GB) is
larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank advances its own
replica of the lattice (the method has no exchange between independent
lattices), timing is the max over ranks and `value` the total over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2207_09431_gb300 import inputs, replicas  # noqa: E402

METRIC = "coupled-step MLUPS (D2Q9, 2 components, FP32)"
UNIT = "MLUPS"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-cases", type=int, default=128)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the collapsed and FP16 state-form lines")
    ap.add_argument("--no-three", action="store_true", help="skip the three-component line")
    ap.add_argument("--state-form", default="populations", choices=["populations", "collapsed", "fp16"],
                    help="state form of the main line (for profiling the other forms; the headline is the "
                         "population form)")
    ap.add_argument("--kernel-config", type=int, default=-1,
                    help="launch configuration of the step kernel (default: autotuned)")
    ap.add_argument("--stability", action="store_true",
                    help="also compare the central and mixed difference schemes on the 36-case paper grid")
    ap.add_argument("--reference-seconds", type=float, default=150.0,
                    help="host time the reference arm spends in its warm-up and timed steps together")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons.  Started and
    awaited before the warm-up, so that its start-up does not overlap the
    timed region; only the samples taken inside the timed window count."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.window = None

    def start(self, wait_s=15.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t_end = time.perf_counter() + wait_s
        while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def begin(self):
        self.window = [time.perf_counter(), None]

    def end(self):
        if self.window is not None:
            self.window[1] = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(self.INTERVAL_MS * 1.5e-3)   # the sample that closes the window
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lines = self.lines
        if self.window is not None and self.window[1] is not None:
            t0, t1 = self.window[0], self.window[1] + self.INTERVAL_MS * 1e-3
            inside = [x for x in lines if t0 <= x[0] <= t1]
            lines = inside or lines[-1:]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for_smi(local, torch):
    """nvidia-smi id of this process's GPU: its UUID when torch exposes it."""
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[local] if vis else str(local)


KERNEL_SOURCES = ("paper_2207_09431_gb300/csrc/lbm_fused.cu", "paper_2207_09431_gb300/csrc/lbm_sweep.cu",
                  "paper_2207_09431_gb300/csrc/lbm_node.cuh", "paper_2207_09431_gb300/csrc/lbm_device.cuh",
                  "paper_2207_09431_gb300/csrc/lbm_devparams.h", "paper_2207_09431_gb300/csrc/lbm_kernels.h")


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, nodes: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.json: bytes per node measured on a smaller case), or None
    when the kernel sources changed since that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    per_node = d.get("bytes_per_node", {}).get(kernel)
    return None if per_node is None else round(per_node * nodes)


def profiled_inst_per_node(kernel: str):
    """Thread instructions per node of `kernel` from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("inst_per_node", {}).get(kernel)


def issue_roofline(inst_per_node, mlups, sm_mhz):
    """The step kernel's instruction issue against the issue peak of the GPU:
    one warp instruction per cycle per scheduler, 4 schedulers per SM,
    152 SMs, 32 lanes, at the SM clock sampled during the timed region."""
    if inst_per_node is None or not sm_mhz:
        return None
    peak = 152 * 4 * 32 * sm_mhz * 1e6
    achieved = inst_per_node * mlups * 1e6
    return {"bound": "issue", "inst_per_node": inst_per_node, "achieved": round(achieved / 1e12, 2),
            "peak": round(peak / 1e12, 2), "unit": "T thread instructions/s", "frac": round(achieved / peak, 4)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Algorithmic bytes per node of each kernel of the step (2 components, FP32):
# every input plane read once and every output plane written once.
def kernel_bytes_per_node(nh: int) -> dict:
    f = 4
    return {
        "k_moments": f * (9 * nh + nh),
        "k_fields": f * (nh + 9 + 1 + 3 + 3 + 1 + 1),
        "k_sources": f * (nh + nh + nh),
        "k_collide": f * (9 + nh + 3 + 1 + 2 + 1 + nh + 9 + 9 * nh),
    }


def step_bytes_per_node(nh: int, form: str = "populations") -> int:
    """Algorithmic bytes of one time step, every state array read and written
    once: populations g (9), h (9 nh) and tau; or g, C (nh) and tau; or FP16 g
    deviations (9 halves) with their FP32 reference, C and tau."""
    if form == "collapsed":
        return 4 * 2 * (9 + nh + 1)
    if form == "fp16":
        return 2 * (9 * 2 + 4 + 4 * nh + 4)
    return 4 * 2 * (9 + 9 * nh + 1)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2207_09431_gb300 import lbm

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p, bubbles = inputs.sweep_case(args.nx)
    form = args.state_form
    if form != "populations":
        p = dict(p, collapse_h=1, storage=1 if form == "fp16" else 0)
    nx, ny = p["nx"], p["ny"]
    nodes = nx * ny
    nh = p["ncomp"] - 1
    sbpn = step_bytes_per_node(nh, form)
    C = inputs.bubble_fields(nx, ny, 2, p["xi"], bubbles, seed=rank, noise=1e-8)
    stream = torch.cuda.Stream(device=dev)
    lat = lbm.Lattice(p, device=dev, stream=stream)
    lat.set_fields(C)
    if args.kernel_config >= 0:
        lbm.lbm_set_kernel_config(lat.h, args.kernel_config)
        kernel_config = lbm.lbm_kernel_name(lat.h, 0)
    else:
        kernel_config = lat.autotune(reps=5)
    clocks = ClockSampler(gpu_id_for_smi(local, torch))
    clocks.start()
    lat.step(args.warmup)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks.begin()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.end()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = replicas.job_time_ms(ms, dist if world > 1 else None)
    value = world * nodes * args.steps / (ms_max * 1e-3) / 1e6

    # dominant kernel: per-kernel device time measured by the library on this stream
    kt = lat.kernel_times(reps=max(3, min(args.steps, 20)))
    hbm, peak_kind = measured_peaks()
    bpn = kernel_bytes_per_node(nh)
    if kt:
        dom = max(kt, key=kt.get)
        achieved = bpn.get(dom, sbpn) * nodes / (kt[dom] * 1e-3) / 1e9
    else:
        dom = "step"
        achieved = sbpn * nodes / (ms_max / args.steps * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": profiled_traffic(dom if form == "populations" else f"{form}:{dom}", nodes),
                "traffic_unit": "bytes per launch", "step_bytes_per_node": sbpn,
                "step_frac": round(sbpn * nodes / (ms_max / args.steps * 1e-3) / 1e9 / hbm, 4)}

    # end to end through the C ABI with host buffers: upload the initial fields,
    # advance K steps, read back the observables
    e2e_lat = lat
    # the step's input, the initial fields as the caller holds them: FP64 in
    # pinned host memory (the library uploads them as they are and converts
    # them on the device)
    C_host = torch.empty(C.shape, dtype=torch.float64, pin_memory=True).numpy()
    C_host[...] = C
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_lat.set_fields(C_host)
    ta = time.perf_counter()
    e2e_lat.step(args.steps)
    tb = time.perf_counter()
    obs = e2e_lat.observables()
    t1 = time.perf_counter()
    h2d = 8 * nodes * nh
    d2h = 16 * 8 + 8 * 4 + 4 * args.steps * 0
    e2e = {"value": round(nodes * args.steps / (t1 - t0) / 1e6, 1), "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "what": "lbm_set_fields from pinned host doubles + lbm_step(K) + lbm_observables, wall clock",
           "set_fields_ms": round((ta - t0) * 1e3, 2), "steps_ms": round((tb - ta) * 1e3, 2),
           "observables_ms": round((t1 - tb) * 1e3, 2),
           "note": "the set-up (upload of the FP64 fields, conversion and initial equilibria on the device) is "
                   "paid once per run; with K steps it is amortised over K"}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded rising bubble)",
        "config": dict(workload_config(nx, world), **({} if form == "populations" else {"state_form": form})),
        "issue": issue_roofline(profiled_inst_per_node(dom if form == "populations" else f"{form}:{dom}"),
                                value / world, clk.get("sm_max_mhz")),
        "roofline": roofline, "e2e": e2e, "clocks": clk,
        "gpu_launches": lat.launches_per_step() * args.steps,
        "kernel_ms": {k: round(v, 5) for k, v in kt.items()},
        "kernel_config": kernel_config,
        "observables_after": {"rise_velocity": obs["rise_velocity"], "mass1": obs["mass"][0]},
    }
    if not args.no_forms:
        for key, storage, form in (("collapsed", 0, "collapsed"), ("fp16_storage", 1, "fp16")):
            leg = run_state_form(args, torch, dev, stream, C, hbm, storage=storage)
            leg["issue"] = issue_roofline(profiled_inst_per_node(f"{form}:{leg['kernel']}"), leg["mlups"],
                                          clk.get("sm_max_mhz"))
            line[key] = leg
    if not args.no_three:
        line["three_comp"] = run_three_comp(args, torch, dev, stream, hbm)
    if not args.no_batched:
        line["batched"] = run_batched(args, torch, dev, stream, rank, world, dist if world > 1 else None)
    if not args.no_surrogate and rank == 0:
        line["surrogate"] = run_surrogate(stream)
    if args.stability and rank == 0:
        from paper_2207_09431_gb300 import stability

        rows, summary = stability.compare(steps=20000, stream=stream)
        line["stability"] = {"steps": 20000, "summary": summary, "cases": rows}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(target_s=15.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_surrogate(stream):
    """C_D error of the surrogate: 1024 seeded 100 x 200 cases solved to their
    terminal state by the batched solver train the ensemble; 128 held-out cases
    solved in full judge it (not part of the timed step)."""
    from paper_2207_09431_gb300 import surrogate

    t0 = time.perf_counter()
    s = surrogate.evaluate(n_train=1024, n_test=128, stream=stream)
    s["wall_s"] = round(time.perf_counter() - t0, 1)
    return s


def run_state_form(args, torch, dev, stream, C, hbm, storage):
    """The same workload with the state held as C instead of h (collapse_h):
    88 algorithmic bytes per node-step instead of 152; with storage = 1 g is
    also kept as FP16 deviations from an FP32 per-node reference: 60 bytes."""
    from paper_2207_09431_gb300 import lbm

    p, _ = inputs.sweep_case(args.nx)
    p = dict(p, collapse_h=1, storage=storage)
    nodes = p["nx"] * p["ny"]
    lat = lbm.Lattice(p, device=dev, stream=stream)
    lat.set_fields(C)
    name = lat.autotune(reps=5)
    lat.step(max(3, args.warmup))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    lat.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / args.steps
    bpn = 2 * (9 * 2 + 4 + 4 + 4) if storage else 4 * 2 * (9 + 1 + 1)
    gbs = bpn * nodes / (ms * 1e-3) / 1e9
    state = "FP16 g deviations + FP32 reference, C, tau" if storage else "g, C, tau (collapse_h = 1)"
    return {"state": state, "mlups": round(nodes / (ms * 1e3), 1), "ms_per_step": round(ms, 4),
            "bytes_per_node": bpn, "achieved_gbs": round(gbs, 1), "frac": round(gbs / hbm, 4), "kernel": name}


def run_three_comp(args, torch, dev, stream, hbm):
    """Three components (the set-up of the three-component configuration:
    power-law matrix, two droplets of component 2, a bubble of component 3,
    fully periodic, no gravity) on an nx x nx lattice, population and collapsed
    state forms, each autotuned and timed with CUDA events like the main line."""
    from paper_2207_09431_gb300 import lbm

    nx = args.nx
    p, discs = inputs.three_comp_case(nx)
    C = inputs.bubble_fields(nx, nx, 3, p["xi"], discs, seed=0, noise=1e-8, periodic_y=True)
    out = {"workload": f"three components {nx}x{nx}, fully periodic, droplets R = {discs[0][2]:g}, "
                       f"{discs[1][2]:g} and bubble R = {discs[2][2]:g}"}
    for form, collapse in (("populations", 0), ("collapsed", 1)):
        q = dict(p, collapse_h=collapse)
        lat = lbm.Lattice(q, device=dev, stream=stream)
        lat.set_fields(C)
        name = lat.autotune(reps=5)
        lat.step(max(3, args.warmup))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1) / args.steps
        bpn = 4 * 2 * (9 + (2 if collapse else 18) + 1)
        gbs = bpn * nx * nx / (ms * 1e-3) / 1e9
        out[form] = {"mlups": round(nx * nx / (ms * 1e3), 1), "ms_per_step": round(ms, 4), "bytes_per_node": bpn,
                     "achieved_gbs": round(gbs, 1), "frac": round(gbs / hbm, 4), "kernel": name}
        del lat
    return out




def _per_case_to_terminal(lbm, case, seed, window, rtol, max_steps, dev, stream):
    """One case alone on its own lattice (lbm_step, the single-lattice kernel)
    to the terminal state of lbm_batch_run's criterion; returns (U_t or None,
    steps, outcome)."""
    p, b, _ = case
    lat = lbm.Lattice(p, device=dev, stream=stream)
    lat.set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=seed, noise=1e-8))
    ob = lat.observables()
    ys, top = [ob["centroid"][1]], p["ny"] - 1 - 1.5 * ob["d_eq"]
    steps = 0
    while True:
        try:
            lat.step(window)
        except lbm.LbmError as err:
            if err.status != -4:
                raise
            return None, steps + window, "diverged"
        steps += window
        ob = lat.observables()
        ys.append(ob["centroid"][1])
        u = np.diff(ys) / window
        if len(u) >= 3 and all(abs(u[-j] - u[-j - 1]) < rtol * abs(u[-j]) for j in (1, 2)):
            return float(u[-1]), steps, "terminal"
        if ys[-1] > top:
            return float(u[-1]), steps, "top"
        if steps >= max_steps:
            return float(u[-1]), steps, "max_steps"


def run_batched(args, torch, dev, stream, rank=0, world=1, dist=None):
    """The ensemble workload: 128 seeded rising-bubble cases on grids from
    {100x200, 150x300, 200x400, 300x600}, density ratio 1000, each run to its
    terminal state (lbm_batch_run: window-averaged rise velocity over 2000-step
    windows changing by less than 5 % twice, or the bubble 1.5 diameters below
    the top, or 40000 steps), (a) all together in persistent launches and (b)
    one case after another on its own lattice (lbm_step), the latter on every
    eighth case.  Cases/hour = cases run to a stop per wall-clock hour.  Both
    forms compute the same node values, so their terminal velocities agree
    (checked on the shared cases).  The C state form and FP16 g storage run
    the same ensemble too (state_forms).  With several ranks every rank takes
    its share of the cases and the times are the slowest rank's."""
    from paper_2207_09431_gb300 import lbm

    window, rtol, max_steps = 2000, 0.05, 40000
    all_cases = inputs.ensemble_cases(args.batch_cases, seed=0, density_ratio=1000.0)
    cases = replicas.shard(all_cases, rank, world)
    nodes = sum(p["nx"] * p["ny"] for p, _, _ in all_cases)
    batch = lbm.Batch([c[0] for c in cases], device=dev, stream=stream)
    batch.set_persistent(True)
    for i, (p, b, _) in enumerate(cases):
        batch.case(i).set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=i, noise=1e-8))
    chosen = batch.autotune(reps=3)
    # kernel view: device time of K persistent steps over every case (cases
    # that turn non-finite keep being computed until the call returns, when
    # they are deactivated)
    K = max(16, (args.steps // 16) * 16)
    batch.step(2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    try:
        batch.step(K)
    except lbm.LbmError as err:
        if err.status != -4:
            raise
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_batch = replicas.job_time_ms(ev0.elapsed_time(ev1) / K, dist)
    # the run to terminal, from fresh initial states
    for i, (p, b, _) in enumerate(cases):
        batch.set_active(i, True)
        batch.case(i).set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=i, noise=1e-8))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = batch.run(window=window, rtol=rtol, max_steps=max_steps, top_margin=1.5)
    torch.cuda.synchronize(dev)
    wall_batch = replicas.job_time_ms((time.perf_counter() - t0) * 1e3, dist) / 1e3
    outcomes = {}
    for r in res:
        outcomes[r["outcome"]] = outcomes.get(r["outcome"], 0) + 1
    stopped = len(cases) - outcomes.get("diverged", 0)
    # one case after another, every eighth case
    sub = list(range(0, len(cases), 8))
    t0 = time.perf_counter()
    single = [_per_case_to_terminal(lbm, cases[i], i, window, rtol, max_steps, dev, stream) for i in sub]
    torch.cuda.synchronize(dev)
    wall_single = time.perf_counter() - t0
    stopped_single = sum(1 for u, _, o in single if o != "diverged")
    same = [abs(u / res[i]["rise_velocity"] - 1.0) for (u, _, o), i in zip(single, sub)
            if o != "diverged" and res[i]["outcome"] != "diverged" and res[i]["rise_velocity"] != 0.0]
    step_bytes = step_bytes_per_node(1)
    forms = {key: _batched_form(lbm, torch, dev, stream, cases, res, extra, K, window, rtol, max_steps, nodes, dist)
             for key, extra in (("collapsed", {"collapse_h": 1}), ("fp16_storage", {"collapse_h": 1, "storage": 1}))}
    return {"cases": len(all_cases), "nodes": nodes, "ranks": world, "density_ratio": 1000.0,
            "mode": "persistent cooperative launches of up to 4096 steps, whole launches replayed from a CUDA graph",
            "ms_per_step": round(ms_batch, 4), "mlups": round(nodes / (ms_batch * 1e3), 1),
            "achieved_gbs": round(step_bytes * nodes / (ms_batch * 1e-3) / 1e9, 1),
            "frac": round(step_bytes * nodes / (ms_batch * 1e-3) / 1e9 / measured_peaks()[0], 4),
            "terminal_rule": f"{window}-step windows, {rtol:g} relative change twice, top margin 1.5 d, "
                             f"at most {max_steps} steps",
            "outcomes": outcomes, "wall_s_to_terminal": round(wall_batch, 2),
            "cases_per_hour": round(stopped / wall_batch * 3600.0, 1),
            "per_case": {"cases": len(sub), "stopped": stopped_single, "wall_s": round(wall_single, 2),
                         "cases_per_hour": round(stopped_single / wall_single * 3600.0, 1),
                         "max_rel_diff_U_t_vs_batched": max(same) if same else None},
            "speedup_cases_per_hour": round((stopped / wall_batch) / max(stopped_single / wall_single, 1e-12), 2),
            "kernel_config": chosen, "state_forms": forms}


def _batched_form(lbm, torch, dev, stream, cases, res32, extra, K, window, rtol, max_steps, nodes, dist):
    """The same ensemble in a C state form (collapse_h = 1, 88 B per node-step)
    or with FP16 g storage on it (60 B): kernel view over K persistent steps,
    then every case run to its terminal state from fresh initial states; U_t
    against the FP32 population batch on the cases that stop in both."""
    batch = lbm.Batch([dict(c[0], **extra) for c in cases], device=dev, stream=stream)
    batch.set_persistent(True)

    def init():
        for i, (p, b, _) in enumerate(cases):
            batch.set_active(i, True)
            batch.case(i).set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=i, noise=1e-8))

    init()
    chosen = batch.autotune(reps=3)
    batch.step(2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    try:
        batch.step(K)
    except lbm.LbmError as err:
        if err.status != -4:
            raise
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = replicas.job_time_ms(ev0.elapsed_time(ev1) / K, dist)
    init()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = batch.run(window=window, rtol=rtol, max_steps=max_steps, top_margin=1.5)
    torch.cuda.synchronize(dev)
    wall = replicas.job_time_ms((time.perf_counter() - t0) * 1e3, dist) / 1e3
    outcomes = {}
    for r in res:
        outcomes[r["outcome"]] = outcomes.get(r["outcome"], 0) + 1
    stops = ("terminal", "top")
    d = [abs(r["rise_velocity"] / r32["rise_velocity"] - 1.0) for r, r32 in zip(res, res32)
         if r["outcome"] in stops and r32["outcome"] in stops and r32["rise_velocity"] != 0.0]
    bpn = 2 * (9 * 2 + 4 + 4 + 4) if extra.get("storage") else 4 * 2 * (9 + 1 + 1)
    del batch
    return {"bytes_per_node": bpn, "ms_per_step": round(ms, 4), "mlups": round(nodes / (ms * 1e3), 1),
            "outcomes": outcomes, "wall_s_to_terminal": round(wall, 2),
            "cases_per_hour": round((len(cases) - outcomes.get("diverged", 0)) / wall * 3600.0, 1),
            "U_t_rel_diff_vs_fp32_populations": {
                "cases": len(d), "median": float(np.median(d)) if d else None,
                "p90": float(np.percentile(d, 90)) if d else None, "max": max(d) if d else None},
            "kernel_config": chosen}


def workload_config(nx, world):
    ny = 2 * nx
    return {"workload": f"rising bubble {nx}x{ny}, R={nx // 8}, density ratio 1000, n=0.7, Eo=10, "
                        "2 components, walls top/bottom",
            "nx": nx, "ny": ny, "nodes": nx * ny, "l2": "state 1.3 GB > L2 (no flush needed)",
            "parallelism": f"replicas x{world}"}


def oracle_window(nx, w=256, h=512):
    """A w x h window of the nx x 2nx workload's initial fields, centred on the
    lower interface of the bubble (a bounded sample of the workload for the
    FP64 oracle; the window has its own walls at its top and bottom)."""
    p, b = inputs.sweep_case(nx)
    cx, cy, R, _ = b[0]
    x0 = max(0, min(p["nx"] - w, int(cx) - w // 2))
    y0 = max(0, min(p["ny"] - h, int(cy - R) - h // 2))
    C = inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=0, noise=1e-8)[:, y0:y0 + h, x0:x0 + w]
    desc = f"{w}x{h} window (x {x0}-{x0 + w - 1}, y {y0}-{y0 + h - 1}) of the {p['nx']}x{p['ny']} workload"
    return dict(p, nx=w, ny=h), C, desc


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_mlups(p, C, precision, target_s):
    """MLUPS of one oracle build on one set-up, for about target_s seconds."""
    import oracle

    o = oracle.Oracle(p, precision)
    o.set_fields(C)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    steps = max(1, int(target_s / max(t1 - t0, 1e-6)))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return p["nx"] * p["ny"] * steps / dt / 1e6, steps


def cpu_baseline(target_s=15.0, nx=2048):
    """The FP64 oracle as it stands on the host's cores: the OpenMP build on all
    cores (the headline value) and the serial build on one core, on a bounded
    sample of the workload (a window around the bubble's lower interface), and
    both builds on the rising bubble at 64 x 128, 200 x 400 and 512 x 1024
    (R = nx / 8, the same physics)."""
    cores = host_cores()
    p, C, desc = oracle_window(nx)
    per = target_s / 8.0
    v_omp, s_omp = _oracle_mlups(p, C, "f64-omp", 2 * per)
    v_one, s_one = _oracle_mlups(p, C, "f64", 2 * per)
    grids = {}
    for gx in (64, 200, 512):
        q, b = inputs.sweep_case(gx)
        Cg = inputs.bubble_fields(q["nx"], q["ny"], 2, q["xi"], b, seed=0, noise=1e-8)
        one, _ = _oracle_mlups(q, Cg, "f64", per / 2)
        omp, _ = _oracle_mlups(q, Cg, "f64-omp", per / 2)
        grids[f"{q['nx']}x{q['ny']}"] = {"mlups_1_thread": round(one, 4), f"mlups_{cores}_threads": round(omp, 4)}
    return {"value": round(v_omp, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{desc}, {s_omp} steps, FP64 C oracle (gcc -O3, OpenMP over the nodes of each pass), "
                      f"{cores} threads",
            "one_thread": {"value": round(v_one, 4), "steps": s_one}, "grids": grids}


def run_reference(args):
    """The oracle timed as the reference arm (its OpenMP build on every host
    core), bounded per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    p, C, desc = oracle_window(args.nx)
    cores = host_cores()
    o = oracle.Oracle(p, "f64-omp")
    o.set_fields(C)
    # lattice steps per bench step: a bounded sample, sized so that the whole
    # run (warm-up and timed steps) takes about --reference-seconds of host time
    t0 = time.perf_counter()
    o.step(1)
    t_one = time.perf_counter() - t0
    sub = max(1, int(args.reference_seconds / (max(args.steps + args.warmup, 1) * max(t_one, 1e-6))))
    o.step(args.warmup * sub)
    t0 = time.perf_counter()
    o.step(args.steps * sub)
    dt = time.perf_counter() - t0
    nodes = p["nx"] * p["ny"]
    value = nodes * args.steps * sub / dt / 1e6
    sample = f"{desc}, {sub} lattice steps per bench step, FP64 C oracle (OpenMP), {cores} threads"
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded rising bubble)",
            "impl": "reference", "config": workload_config(args.nx, world),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
