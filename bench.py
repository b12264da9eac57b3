#!/usr/bin/env python
"""Benchmark of the SDM coalescence step on one B300 (per rank).

Workload (default): the 256 x 256 lognormal grid -- 65 536 cells of dV = 1e3
m^3 holding Poisson(256) super-droplets each (1.68e7 SDs), radii lognormal
(median 15 um, sigma_g 1.4), n0 = 1e8 m^-3, gravitational kernel, dt = 1 s,
FP64-exact decisions: the largest of the workloads that fits one GPU.  A
"step" is one coalescence timestep over all super-droplets (Fig. "fig:algo":
removal, shuffle, pairing, eq. (p), gamma, update).  Metric: super-droplet-steps
per second (live SDs x steps / time).

Each step is timed alone with CUDA events on the library's stream, after a
256 MB write that evicts L2 (the 268 MB state is larger than L2 as well);
ms_per_step is their mean.  With --graph G, G steps are captured into one CUDA
graph (a device step counter advances the random-number stream) and the
replays are timed instead (the batched-ensemble form: --workload ensemble
--precision fp32 --graph 100).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload W] [--precision P] [--shuffle S] [--graph G]

Under torchrun each rank runs its own copy of the workload (independent
problems: weak scaling, no collective on the data path); rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2101_06318_b300 import inputs  # noqa: E402

SURROGATE_TRAIN_STEPS = 8000
METRIC = "coalescence super-droplet-steps/s on 1 B300, % HBM roofline; batched/surrogate vs FP64"
UNIT = "SD-steps/s"
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _source_hash():
    """sha256 over the per-file sha256 lines of the device-code headers (the kernels' source)."""
    import hashlib
    files = [os.path.join(ROOT, "paper_2101_06318_b300", "csrc", f) for f in ("sdm_kernels.cuh", "sdm_math.cuh")]
    lines = []
    for f in files:
        with open(f, "rb") as fh:
            digest = hashlib.sha256(fh.read()).hexdigest()
        lines.append(f"{digest}  {os.path.relpath(f, ROOT)}\n")
    return hashlib.sha256("".join(lines).encode()).hexdigest()


def _profiled_traffic(kernel, workload_name, n_sd):
    """DRAM bytes per launch from the committed ncu summary of this kernel and workload, when the
    summary was taken on the current sources (else None: the counters are stale)."""
    short = kernel.split("::")[-1]
    path = os.path.join(ROOT, "profiles", f"{short}_{workload_name}_{n_sd >> 20}M.md")
    try:
        with open(path) as f:
            txt = f.read()
    except OSError:
        return None
    fields = dict(ln.split(":", 1) for ln in txt.splitlines() if ln.startswith(("csrc_sha256:", "dram_bytes")))
    if fields.get("csrc_sha256", "").strip() != _source_hash():
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def workload(name, rank=0, grid_ny=None):
    if name == "gravitational_box":
        return inputs.gravitational_box(seed=42 + rank)
    if name.startswith("grid_"):
        return inputs.WORKLOADS[name](ny=grid_ny or 256, seed=42 + rank)   # grid_ny: a smaller grid
    if name == "ensemble":
        return inputs.ensemble(seed=42 + rank)
    return inputs.WORKLOADS[name]()


def sample_of(name, s, frac):
    """A bounded sample of workload s holding about frac of its SDs, of the same kind: fewer
    grid rows, fewer ensemble members, or a smaller box (the CPU legs' samples)."""
    if frac >= 1.0:
        return s
    if name.startswith("grid_"):
        ny = max(1, int(s["meta"]["ny"] * frac))
        return inputs.WORKLOADS[name](ny=ny)
    if name == "ensemble":
        return inputs.ensemble(n_members=max(2, int(1024 * frac)))
    if name == "gravitational_box":
        return inputs.gravitational_box(n_sd=1 << max(10, int(np.floor(np.log2(len(s["xi"]) * frac)))))
    return s


def cpu_baseline(s, budget_s=12.0, shuffle="prp", name=None):
    """The oracle as it stands, single-threaded on a host core, on a bounded sample of steps (a
    smaller sample of the same workload when one full step would take more than the budget)."""
    import oracle

    def system(t):
        return oracle.System(t["xi"], t["v"], t["cell_start"], t["dv"], t["kernel_id"], t["golovin_b"],
                             shuffle=shuffle)
    o = system(s)
    t0 = time.perf_counter()
    o.step(s["dt"], 42, 0)
    t1 = time.perf_counter() - t0
    first = 1
    if name and t1 > budget_s / 4:
        s = sample_of(name, s, budget_s / 8 / t1)
        o = system(s)
        first = 0
    n_live = int(np.count_nonzero(o.xi))
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(s["dt"], 42, first + steps)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n_live * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of the {s['name']} workload ({n_live} SDs, {len(s['dv'])} cells), "
                      f"single-threaded C, FP64"}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    s = workload(args.workload, grid_ny=getattr(args, "grid_ny", None))
    n = len(s["xi"])
    # bound the run to a few minutes: a full step of the oracle on this workload
    shuf = getattr(args, "shuffle", "prp")
    probe = oracle.System(s["xi"], s["v"], s["cell_start"], s["dv"], s["kernel_id"], s["golovin_b"], shuffle=shuf)
    t0 = time.perf_counter()
    probe.step(s["dt"], 42, 0)
    t_step = time.perf_counter() - t0
    sample = s
    if (args.steps + args.warmup) * t_step > 150.0:
        sample = sample_of(args.workload, s, 150.0 / ((args.steps + args.warmup) * t_step))
    o = oracle.System(sample["xi"], sample["v"], sample["cell_start"], sample["dv"], sample["kernel_id"],
                      sample["golovin_b"], shuffle=shuf)
    for w in range(args.warmup):
        o.step(sample["dt"], 42, w)
    n_live = int(np.count_nonzero(o.xi))
    t0 = time.perf_counter()
    for k in range(args.steps):
        o.step(sample["dt"], 42, args.warmup + k)
    el = time.perf_counter() - t0
    value = n_live * args.steps / el
    desc = (f"{args.steps} timed steps of {sample['name']} with {len(sample['xi'])} SDs "
            f"(oracle, single-threaded C, FP64)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "n_sd": len(sample["xi"]),
                                            "n_cell": len(sample["dv"]), "kernel": _kernels(sample),
                                            "precision": "fp64", "shuffle": shuf},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _kernels(s):
    k = set(int(x) for x in np.unique(s["kernel_id"]))
    return {0: "golovin", 1: "gravitational"}[k.pop()] if len(k) == 1 else "golovin+gravitational"


def combine_ranks(tot_ms, sd_steps, e2e_s, dist, world, device):
    """Whole-job figures from every rank's own: the slowest rank's timed span (max), the SD-steps
    of all ranks (sum) and the slowest end-to-end step (max).  One all_gather; no collective
    touches the data path."""
    if not dist or world == 1:
        return tot_ms, sd_steps, e2e_s
    import torch
    t = torch.tensor([tot_ms, sd_steps, e2e_s], dtype=torch.float64, device=device)
    ts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(ts, t)
    return (max(float(x[0]) for x in ts), sum(float(x[1]) for x in ts), max(float(x[2]) for x in ts))


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2101_06318_b300 import sdm
    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    s = workload(args.workload, rank, getattr(args, "grid_ny", None))
    n = len(s["xi"])
    prec = args.precision
    shuf = getattr(args, "shuffle", "prp")
    surr_info = None
    with torch.cuda.stream(stream):
        st = sdm.from_inputs(s)
        if args.schedule:
            st.set_schedule(**json.loads(args.schedule))
        if prec == "surrogate":
            # the network is trained once, outside the timed region, by the library's own kernels
            t0 = time.perf_counter()
            surr = sdm.Surrogate(n_train=10_000_000, seed=7, r_min=1e-6, r_max=3e-3, stream=stream)
            loss = surr.train(SURROGATE_TRAIN_STEPS, batch=8192, lr=5e-3)
            frac, _ = surr.build_mask(0.01)
            torch.cuda.synchronize()
            surr_info = {"train_steps": SURROGATE_TRAIN_STEPS, "train_batch": 8192,
                         "train_s": round(time.perf_counter() - t0, 3), "final_loss": float(loss[-50:].mean()),
                         "mask_tiles_within_1pct": frac}
            st.attach_surrogate(surr)
            ref = sdm.from_inputs(s)             # plain FP64 steps of the same seed, for the accuracy figures
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        step = 0
        for _ in range(args.warmup):
            st.step(s["dt"], 42, step, 1, precision=prec, golovin_b=s["golovin_b"], shuffle=shuf)
            step += 1
        st.sync()
        live0 = st.remove_zero()
        # which kernels one step launches (one profiled step, outside the timed region)
        st.set_profiling(True)
        st.step(s["dt"], 42, step, 1, precision=prec, golovin_b=s["golovin_b"], shuffle=shuf)
        step += 1
        st.sync()
        kinds = [k for k, v in st.profile().items() if v[0]]
        st.set_profiling(False)
        # a step of a single kernel kind (the large-cell kernel and the compaction launched right
        # behind it count as one) is timed by the step's own events, which bracket exactly those
        # launches; otherwise each kind is bracketed by events of its own inside the timed region
        single = len(kinds) == 1
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if args.graph:
            # G steps captured once into a CUDA graph; the device step counter advances the
            # random-number stream from replay to replay; the replays are timed
            G = args.graph
            n_rep = max(1, args.steps // G)
            n_timed = n_rep * G
            d_step = torch.full((1,), step, dtype=torch.int32, device=dev)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                st.step(s["dt"], 42, 0, G, precision=prec, golovin_b=s["golovin_b"], shuffle=shuf, d_step=d_step)
            graph.replay()                               # one untimed replay
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_rep)]
            with ClockSampler(local_rank) as clk:
                torch.cuda._sleep(int(2e8))
                for k in range(n_rep):
                    flush.fill_(float(k))
                    ev[k][0].record(stream)
                    graph.replay()
                    ev[k][1].record(stream)
                torch.cuda.synchronize()
            step = int(d_step.item())
            total = sum(a.elapsed_time(b) for a, b in ev)
            prof = {(kinds[0] if single else "cuda_graph_step"): (n_timed, total)}
            times = [total / n_timed]
        else:
            n_timed = args.steps
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            if not single:
                st.set_profiling(True)
            with ClockSampler(local_rank) as clk:
                # hold the stream briefly so that every timed iteration is queued before the first one
                # runs: the steps then run back to back and no step waits for the host to submit it
                torch.cuda._sleep(int(2e8))
                for k in range(args.steps):
                    flush.fill_(float(k))                    # evict the state from L2 between steps
                    ev[k][0].record(stream)
                    st.step(s["dt"], 42, step, 1, precision=prec, golovin_b=s["golovin_b"], shuffle=shuf)
                    ev[k][1].record(stream)
                    step += 1
                torch.cuda.synchronize()
            if single:
                prof = {kinds[0]: (args.steps, sum(a.elapsed_time(b) for a, b in ev))}
            else:
                prof = st.profile()
                st.set_profiling(False)
            times = [a.elapsed_time(b) for a, b in ev]
        st.sync()
        if dist:
            dist.barrier()
        live1 = st.remove_zero()
        ms = float(np.mean(times))
        sd_steps = 0.5 * (live0 + live1) * n_timed
        # collisions per step (for the write part of the algorithmic bytes), one extra stats step
        stats = st.step(s["dt"], 42, step, 1, precision=prec, golovin_b=s["golovin_b"], stats=True,
                        shuffle=shuf)
        step += 1
        launches = (st.launches_per_step(shuf) + (1 if args.graph else 0)) * n_timed
        if surr_info is not None:
            # accuracy against plain FP64 steps of the same seed and step indices
            for k in range(step):
                ref.step(s["dt"], 42, k, 1, precision="fp64", golovin_b=s["golovin_b"])
            edges = np.geomspace(1e-6, 5e-3, 101)
            sp_s, sp_r = st.spectrum(edges), ref.spectrum(edges)
            n_s, _, _ = st.totals()
            n_r, _, _ = ref.totals()
            surr_info.update({"steps_compared": step,
                              "spectrum_l1_vs_fp64": float(np.abs(sp_s - sp_r).sum() / max(sp_r.sum(), 1e-300)),
                              "droplet_count_rel_diff_vs_fp64": (n_s - n_r) / max(n_r, 1)})
            ref.close()

        # e2e: host (pinned) buffers in, step, host buffers out, through the C ABI
        xi_h, at_h, _ = st.get_state()
        xi_p = torch.from_numpy(xi_h.view(np.int64)).pin_memory()
        at_p = torch.from_numpy(at_h).pin_memory()
        e2e_steps = min(args.steps, 50)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            st.set_state(xi_p, at_p)
            st.step(s["dt"], 42, step, 1, precision=prec, golovin_b=s["golovin_b"], shuffle=shuf)
            st.get_state(xi_p, at_p)
            step += 1
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        bytes_io = xi_p.numel() * 8 + at_p.numel() * 8

    tot_ms, sd_total, e2e_s = combine_ranks(ms * n_timed, sd_steps, e2e_s, dist, world, dev)
    if rank != 0:
        return
    value = sd_total / (tot_ms * 1e-3)
    peak, peak_src = _peaks()
    # algorithmic bytes per SD-step of the in-place update model: read xi and v, write xi and v
    # (32 B); the bytes a step must touch at least are the reads (16 B per SD) plus 32 B per collision
    bytes_step = 32.0 * live0
    bytes_touched = 16.0 * live0 + 32.0 * stats["n_collisions"]
    kern = {k: {"launches": v[0], "ms_total": v[1], "ms_per_launch": (v[1] / v[0] if v[0] else None)}
            for k, v in prof.items() if v[0]}
    tot_k = sum(v["ms_total"] for v in kern.values()) or 1.0
    for v in kern.values():
        v["share"] = v["ms_total"] / tot_k
    dom = max(kern, key=lambda k: kern[k]["ms_total"])
    # a step of one kernel kind: one launch of it processes every SD of the step, so its algorithmic
    # bytes are the step's; a step of several kinds: the step's bytes over the whole step's time
    # (a lower figure than the dominant kernel's own)
    t_launch = kern[dom]["ms_per_launch"] if len(kern) == 1 else tot_ms / n_timed
    achieved = bytes_step / (t_launch * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                "traffic": _profiled_traffic(dom, args.workload, n),
                "algorithmic_bytes_per_launch": bytes_step, "bytes_per_unit": 32,
                "min_bytes_touched_per_launch": bytes_touched,
                "ms_per_launch": kern[dom]["ms_per_launch"],
                "time_basis": "the kernel's launches" if len(kern) == 1 else "whole step (several kernel kinds)"}
    state_mb = (16.0 + 1.0) * n / 2 ** 20
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n_timed,
        "warmup": args.warmup, "ms_per_step": tot_ms / n_timed, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "surrogate": "bf16/f32"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "n_sd": n, "n_cell": len(s["dv"]), "kernel": _kernels(s),
                   "precision": prec, "shuffle": shuf, "dt_s": s["dt"], "dV_m3": float(s["dv"][0]), "n0_m3": 1e8,
                   "l2": (f"state of {state_mb:.0f} MB " + ("larger than" if state_mb > 126 else "within")
                          + " the 126 MB L2; flushed between timed " + ("replays" if args.graph else "steps")
                          + " (256 MB write)"),
                   "parallelism": f"replicas{world}", "schedule": st.schedule,
                   "timing": (f"CUDA graph of {args.graph} steps, replays timed" if args.graph
                              else "each step timed alone")},
        "roofline": roofline,
        "kernels": kern,
        "e2e": {"value": (sd_total / n_timed) / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "stats_per_step": stats,
    }
    if surr_info is not None:
        line["surrogate"] = surr_info
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(s, shuffle=shuf, name=args.workload)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid_lognormal", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--grid-ny", type=int, default=None,
                    help="rows of a grid workload (default 256); smaller grids for profiling captures")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "surrogate"])
    ap.add_argument("--shuffle", default="prp", choices=["prp", "sort"],
                    help="Step 1 contract: keyed bijection above 256 SDs (prp) or sort by key (sort)")
    ap.add_argument("--schedule", default=None, help="JSON of sdm_schedule fields")
    ap.add_argument("--graph", type=int, default=0,
                    help="capture this many steps into one CUDA graph and time its replays")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.graph < 0 or (args.graph and args.steps < args.graph):
        ap.error("--graph G needs 0 < G <= --steps")
    if args.precision == "surrogate" and args.shuffle != "prp":
        ap.error("the surrogate precision runs under the prp contract only")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
