#!/usr/bin/env python
"""Benchmark of the fused delayed-network step on one B300 per rank.

One bench step = one simulation step of dt = 0.05 ms of the whole network: the
delayed gather over every edge, the FHN update of every node, the history write,
the low-pass readout and (every 20 steps) the noisy observation -- one launch of
the fused step kernel.

Workload (default ``roofline``): N = 1,000,000 nodes in a 1 mm cube, ~50M edges
(2.5 % hubs of in-degree 1000, the rest a radius graph of mean ~25.6), weights
lognormal(-2, 0.5) with 20 % negated, speeds U(0.05, 0.5) m/s, 5 Hz background
pulses, a 256-step history ring.  Inputs are larger than L2 (the 400 MB edge stream
is re-read every step), so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Metric: edge-updates/s (E * K / time), whole job.
With N > 1 (torchrun) every rank runs an independent replica of the workload with
its own seed (the nets are independent problems: no exchange, weak scaling).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0908_3934_b300 import netgen  # noqa: E402

METRIC = "edge-updates/s"
EDGE_BYTES = 12        # packed record (src|D 4 B + weight 4 B) + the gathered FP32 value
NODE_BYTES = 36.2      # v~ read 4, (w~,c~) read 8 + write 8, ring write 4, row_ptr 4,
                       # background counter 4 + caller id 4, readout 4 B / 20 steps
# staged kernel: per edge its weight 4 B + gather index 2 B; per distinct (source,
# delay) of a tile its packed key 4 B + the FP32 history value 4 B
STAGED_EDGE_BYTES = 6
STAGED_GATHER_BYTES = 8
KERNEL_NAMES = {1: "k_step", 2: "k_step_pipe", 3: "k_step_staged", 4: "k_resident", 5: "k_step_persist"}
RESIDENT_CHUNK = 65536  # steps per launch of the resident and persistent kernels
# format-independent bytes of one step: per edge-update a 10-byte edge record (weight 4,
# source 4, delay 2) + the gathered FP32 history value 4; per node-step NODE_BYTES
SURVEY_EDGE_BYTES = 14
E2E_MIN_STEPS = 2000   # the end-to-end leg runs at least this many steps ...
E2E_MIN_CHUNKS = 2     # ... in at least this many host round trips


def survey_bytes(E: int, N: int, node_bytes: float = NODE_BYTES) -> float:
    """Format-independent bytes of one step: 14 B per edge-update + node_bytes per node."""
    return E * SURVEY_EDGE_BYTES + N * node_bytes


def compact(x, digits: int = 4):
    """The result with every float rounded to `digits` significant digits (the
    printed line stays short; the details file keeps full precision)."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}")
    if isinstance(x, dict):
        return {k: compact(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [compact(v, digits) for v in x]
    return x


def algorithmic_bytes(info: dict, E: int, N: int) -> float:
    """Bytes one step must move under the chosen kernel's edge format (padding and
    re-reads excluded)."""
    if info["step_kernel"] == 3:
        return E * STAGED_EDGE_BYTES + info["step_gathers"] * STAGED_GATHER_BYTES + N * NODE_BYTES
    if info["step_kernel"] == 5:  # keys and entries stay in shared memory: the gathered values and node state
        return info["step_gathers"] * 4 + N * NODE_BYTES
    return E * EDGE_BYTES + N * NODE_BYTES


def workload(name: str, rank: int):
    """The seeded network of a replica (cached under the temp dir: generating the
    1M-node net takes ~40 s of host time and it is the same on every call)."""
    import pickle
    gens = {"roofline": lambda: netgen.roofline(seed=4 + 1000 * rank),
            # secondary sizes of the 1M-node net: the literal 5 % hubs beside non-hubs
            # of mean in-degree 50 (overall ~97.5) and conduction speeds x 0.1 (delays up
            # to ~410 steps, ring 512)
            "roofline_hubs5": lambda: netgen.roofline(seed=4 + 1000 * rank, hub_frac=0.05, mean_deg=97.5),
            "roofline_slow": lambda: netgen.delay_stress(netgen.roofline(seed=4 + 1000 * rank)),
            "large": lambda: netgen.large(seed=3 + 1000 * rank),
            "tiny": lambda: netgen.tiny(seed=1 + 1000 * rank),
            "batch": lambda: netgen.batch(4096, seed0=1000 + 100000 * rank)}
    if name not in gens:
        raise SystemExit(f"unknown workload {name}")
    src = open(os.path.join(ROOT, "paper_0908_3934_b300", "netgen.py"), "rb").read()
    key = hashlib.sha256(src + f"{name}:{rank}".encode()).hexdigest()[:16]
    path = os.path.join(tempfile.gettempdir(), f"geonet_{name}_{rank}_{key}.pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    spec = gens[name]()
    tmp = path + f".{os.getpid()}"
    with open(tmp, "wb") as f:
        pickle.dump(spec, f, protocol=4)
    os.replace(tmp, path)
    return spec


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_hash() -> str:
    """Hash of the step kernels' code: comments and layout do not count, so a
    profile stays tied to the code it was taken on across comment edits."""
    import re
    h = hashlib.sha256()
    for f in ("k_step.cu", "k_step_pipe.cu", "k_step_staged.cu", "staged.cu", "step_common.cuh", "ptx.cuh",
              "internal.cuh", "philox.cuh"):
        with open(os.path.join(ROOT, "paper_0908_3934_b300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)   # block comments
        src = re.sub(r"//[^\n]*", " ", src)                 # line comments
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel: str, workload_name: str, grid: int | None = None):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if
    it was taken on the current kernel source and (where the summary lists several
    tilings by grid size) on the tiling this run uses; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload_name}.json")
    try:
        with open(path) as f:
            p = json.load(f)
        if p.get("kernel_hash") != kernel_hash():
            return None
        by_grid = p.get("dram_bytes_per_launch_by_grid")
        if by_grid is not None:
            return float(by_grid[str(grid)]) if str(grid) in by_grid else None
        return float(p["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu=timestamp,{self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if uuid:
            cmd.insert(1, f"--id={uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [l.strip().split(", ") for l in self.tmp.read().splitlines() if l.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_rate(units: float, seconds: float, device="cpu"):
    """Whole-job rate of independent replicas: the units every rank processed over
    the slowest rank's timed region (sum and max over ranks; no data-path
    collective).  Returns (rate, total units, max seconds); one process returns
    its own."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units / seconds, units, seconds
    u = torch.tensor([units], dtype=torch.float64, device=device)
    sec = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(sec, op=dist.ReduceOp.MAX)
    return u.item() / sec.item(), u.item(), sec.item()


def host_cpu() -> str:
    """The host's CPU model and logical core count."""
    model = "unknown CPU"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{model}, {os.cpu_count()} logical cores"


WINDOW_STEPS = 4000  # the first 200 ms at dt = 0.05 ms: the parity window


def cpu_baseline(spec, steps: int):
    """The FP64 oracle as it stands (single-threaded C), on the first `steps` steps
    of the network from rest.  Its cost per step does not depend on the activity
    (every edge and node is visited every step), so the time of the 4000-step
    window is extrapolated from the sample and labelled as such."""
    import oracle
    D = oracle.net_delays(spec)
    t0 = time.perf_counter()
    oracle.simulate(spec, steps, delay=D, want_y=False, ev_cap=1)
    dt = time.perf_counter() - t0
    return dict(value=spec.n_edges * steps / dt, unit=METRIC, cores=1, kind="oracle",
                sample=f"first {steps} steps of the same {spec.n_nodes}-node network from rest "
                       f"(FP64 C oracle, 1 thread; delays precomputed, untimed)",
                host=host_cpu(), window_steps=WINDOW_STEPS, window_s_extrapolated=dt / steps * WINDOW_STEPS,
                seconds=dt)


def _oracle_copy(name: str, steps: int, barrier, out):
    """One core's copy of the cpu_baseline sample, in a spawned process: the network
    from the workload cache, its delays, then (all copies together) the timed steps."""
    import oracle
    spec = workload(name, 0)
    D = oracle.net_delays(spec)
    barrier.wait(timeout=900)
    t0 = time.perf_counter()
    oracle.simulate(spec, steps, delay=D, want_y=False, ev_cap=1)
    out.put((spec.n_edges * steps, time.perf_counter() - t0))


def cpu_baseline_all_cores(name: str, spec, steps: int, bytes_per_copy: float = 3e9):
    """The same oracle sample run as one independent copy per host core (as many as
    the free memory holds, 2.5 GB at peak each for the 1M-node net), all copies timed
    together: the host's aggregate oracle throughput.  The oracle itself is one
    thread; one network is not split across cores (that would change the oracle)."""
    import multiprocessing as mp
    avail = bytes_per_copy
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
                    break
    except (OSError, ValueError, IndexError):
        pass
    try:  # a container's memory limit, where one is set
        with open("/sys/fs/cgroup/memory.max") as f:
            lim = f.read().strip()
        if lim != "max":
            with open("/sys/fs/cgroup/memory.current") as f:
                avail = min(avail, int(lim) - int(f.read().strip()))
    except (OSError, ValueError):
        pass
    copies = max(1, min(os.cpu_count() or 1, int(avail // bytes_per_copy)))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(copies)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_copy, args=(name, steps, barrier, out)) for _ in range(copies)]
    for p in procs:
        p.start()
    try:
        res = [out.get(timeout=1800) for _ in range(copies)]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    units = sum(u for u, _ in res)
    t = max(s for _, s in res)
    return dict(value=units / t, unit=METRIC, cores=copies, kind="oracle",
                sample=f"{copies} independent copies of the first {steps} steps of the same "
                       f"{spec.n_nodes}-node network, one per core, timed together (edge-updates of all copies "
                       f"over the slowest copy's time)", seconds=t)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    spec = workload(args.workload, 0)
    steps = max(1, min(args.steps, args.ref_steps))
    warm = max(0, min(args.warmup, 3))  # untimed oracle steps (the oracle has no caches to warm)
    if warm:
        cpu_baseline(spec, warm)
    cb = cpu_baseline(spec, steps)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": cb["seconds"] / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, spec, world),
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "host",
                                                "window_steps", "window_s_extrapolated")},
            "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(args, spec, world):
    ring = f"ring {spec.ring_depth}" if spec.ring_depth else "ring sized to the delays"
    bg = f"{spec.background['rate_hz']:g} Hz background" if spec.background else "no background"
    return {"workload": f"{args.workload}: N={spec.n_nodes}, E={spec.n_edges} per replica, dt={spec.dt_ms:g} ms, "
                        f"FHN nodes, {bg}, {ring}",
            "nodes_per_replica": spec.n_nodes, "edges_per_replica": spec.n_edges, "replicas": world,
            "dt_ms": spec.dt_ms, "l2": "inputs larger than L2 (edge stream re-read every step)",
            "parallelism": f"replicas{world}"}


def run_batched(args, local, stream, rank):
    """4096 independent 2D networks (N log-uniform in [32, 4096]) advanced
    `batch_steps` steps by the batched form (the kernel and schedule its first
    step times), against looping the single-network path over a random sample of
    the same networks."""
    import torch
    from paper_0908_3934_b300 import geonet
    specs = workload("batch", rank)
    E = sum(sp.n_edges for sp in specs)
    N = sum(sp.n_nodes for sp in specs)
    b = geonet.Batch(specs, device=local, stream=stream.cuda_stream, obs_capacity=64)
    b.gn_batch_step(20)  # chooses the CTA size, warms up
    b.gn_batch_synchronize()
    steps = args.batch_steps
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.gn_batch_step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    info = b.gn_batch_get_info()
    b.gn_batch_destroy()
    # looping the single-network path (one network after another, each replaying its
    # own graph of step launches) over a random sample, extrapolated by count
    rng = np.random.default_rng(11)
    pick = rng.choice(len(specs), args.loop_sample, replace=False)
    t_sample = 0.0
    for i in pick:
        net = geonet.Net(specs[i], device=local, stream=stream.cuda_stream, obs_capacity=64)
        net.gn_step(20)
        net.gn_synchronize()
        ev0.record(stream)
        net.gn_step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_sample += ev0.elapsed_time(ev1) / 1e3
        net.gn_net_destroy()
    t_loop = t_sample / len(pick) * len(specs)
    return {"details_workload": f"{len(specs)} independent 2D nets, N log-uniform in [32, 4096], "
                        f"{N} nodes, {E} edges, {steps} steps ({steps * 0.05:.0f} ms)",
            "value": E * steps / t, "details_unit": METRIC, "seconds": t, "ms_per_step": t / steps * 1e3,
            "details_rtf": steps * 0.05e-3 / t, "details_cta_threads": info["cta_threads"], "details_grid": info["grid"],
            "step_kernel": info["step_kernel"],
            # kernels 3 and 5: member groups stepped a 64-step chunk at a time (L2 blocking),
            # in lanes (3: concurrent launch chains; 5: CTA lanes of one persistent launch);
            # 1 group = every member every step
            "step_groups": info["step_groups"], "step_lanes": info["step_lanes"],
            # kernel 1: one persistent launch; kernel 3: one per group and step + one advance per
            # 64-step graph (and per ragged tail); kernel 5: one cooperative launch + one advance
            # per chunk
            "details_gpu_launches": 1 if info["step_kernel"] == 1
            else 2 * ((steps + 63) // 64) if info["step_kernel"] == 5
            else steps * max(1, info["step_groups"]) + (steps + 63) // 64,
            "loop_plain": {"value": E * steps / t_loop, "details_seconds_extrapolated": t_loop,
                           "details_sample": f"{len(pick)} random nets timed one after another, "
                                     f"{t_sample:.3f} s, extrapolated by count to {len(specs)}"},
            "speedup_vs_loop": t_loop / t}


def run_size(name: str, steps: int, warmup: int, local, stream, rank):
    """Another size of the plain path (config 2's 100k-node net, the 1M-node net's
    literal 5 % hubs, its slow-conduction variant): device time per step on the
    launching stream after `warmup` untimed steps, edge-updates/s, real-time
    factor, and the step's algorithmic bytes over the measured HBM peak, both in
    the format-independent count (14 B per edge-update + 36.2 B per node) and in the
    chosen kernel's own format."""
    import torch
    from paper_0908_3934_b300 import geonet
    t0 = time.perf_counter()
    spec = workload(name, rank)
    t_gen = time.perf_counter() - t0
    net = geonet.Net(spec, device=local, stream=stream.cuda_stream, obs_capacity=64)
    net.gn_step(max(3, warmup))
    net.gn_synchronize()
    info = net.gn_net_get_info()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    net.gn_step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    net.gn_net_destroy()
    E, N = spec.n_edges, spec.n_nodes
    step_s = t / steps
    peak, _ = peaks()
    return {"details_workload": f"{name}: N={N}, E={E}, dt={spec.dt_ms:g} ms, max delay {info['max_delay']} steps, "
                        f"ring {info['ring_depth']}",
            "details_steps": steps, "ms_per_step": step_s * 1e3, "value": E * steps / t, "details_unit": METRIC,
            "rtf": spec.dt_ms * 1e-3 / step_s, "details_node_steps_per_s": N * steps / t,
            "kernel": KERNEL_NAMES[info["step_kernel"]],
            "frac_survey": survey_bytes(E, N) / step_s / 1e9 / peak,
            "frac_format": algorithmic_bytes(info, E, N) / step_s / 1e9 / peak,
            "details_gpu_launches": steps + (steps + 63) // 64, "details_generate_s": t_gen}


IZH_NODE_BYTES = 56.2  # V r/w 8, (W, c) r/w 16, (r, p) r/w 16, spike-ring write 4, piece list 4,
                       # background counter 4 + caller id 4, readout 4 B / 20 steps
HH_NODE_BYTES = 88.12  # the same + gates (m, n, h, pad) r/w 32, readout 4 B / 33 steps
PLASTIC_NODE_BYTES = 4.0  # plastic weights: the node's own ring word (s, spd) read 4
PLASTIC_SLOT_BYTES = 4.0  # per lane slot its piece's length and row
STDP_DEMO = dict(alpha=5.0, beta=0.05)  # weight units per ms, 1/ms


def run_spiking(args, spec, local, stream, model: str, plastic: bool = False):
    """The same network with spiking nodes -- Izhikevich (dt as the network's) or
    Hodgkin-Huxley (dt = 0.03 ms), both with alpha-function PSCs and calcium, the
    paper's two benchmark models -- optionally with plastic weights: step time of
    the autotuned kernel on the device, CUDA events on the stream.  The weight
    write-backs of a plastic net (edges next to a spike only) are not counted in
    its algorithmic bytes."""
    import torch
    from paper_0908_3934_b300 import geonet
    hh = model == "hh"
    ispec = netgen.hodgkin_huxley(spec) if hh else netgen.izhikevich(spec)
    if plastic:
        ispec = dataclasses.replace(ispec, stdp=dict(STDP_DEMO))
    steps = args.hh_steps if hh else args.izh_steps
    every = ispec.obs["sample_every"]
    net = geonet.Net(ispec, device=local, stream=stream.cuda_stream, obs_capacity=max(64, steps // every + 1))
    net.gn_step(max(3, args.warmup))
    net.gn_synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    net.gn_step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    info = net.gn_net_get_info()
    n_spikes = int(net.gn_get_events(cap=1 << 24)[0].size)
    nonfinite = int((~np.isfinite(net.gn_get_izh_state()["V"])).sum())
    changed = None
    if plastic:
        changed = float(np.mean(net.gn_get_weights() != np.asarray(ispec.weight, np.float32)))
    net.gn_net_destroy()
    E, N = ispec.n_edges, ispec.n_nodes
    bytes_step = (E * STAGED_EDGE_BYTES + info["step_gathers"] * STAGED_GATHER_BYTES
                  if info["step_kernel"] == 3 else E * EDGE_BYTES) + N * (HH_NODE_BYTES if hh else IZH_NODE_BYTES)
    if plastic:
        bytes_step += N * PLASTIC_NODE_BYTES + info["step_lane_slots"] * PLASTIC_SLOT_BYTES
    peak, _ = peaks()
    step_s = t / steps
    nodes = ("Hodgkin-Huxley nodes (classic squid-axon rates) with alpha-function PSCs and calcium, "
             "5 Hz background pulses of 20 uA/cm^2" if hh else
             "Izhikevich regular-spiking nodes with alpha-function PSCs and calcium, 5 Hz background pulses of 2500 pA")
    if plastic:
        nodes += (f", plastic weights (spike-time-dependent, alpha {STDP_DEMO['alpha']}/ms, "
                  f"beta {STDP_DEMO['beta']}/ms)")
    out = {"details_workload": f"the same {N}-node network, {nodes}, dt = {ispec.dt_ms} ms, max delay {info['max_delay']} steps",
            "value": E * steps / t, "details_unit": METRIC, "ms_per_step": step_s * 1e3, "details_steps": steps,
            "details_node_steps_per_s": N * steps / t,
            "rtf": ispec.dt_ms * 1e-3 / step_s, "spikes_per_node_per_s": n_spikes / N / (steps * ispec.dt_ms * 1e-3),
            "details_step_kernel": KERNEL_NAMES[info["step_kernel"]],
            "frac": bytes_step / step_s / 1e9 / peak,
            "details_roofline": {"bound": "hbm", "achieved": bytes_step / step_s / 1e9, "peak": peak, "unit": "GB/s",
                                 "algorithmic_bytes_per_launch": bytes_step},
            "details_gpu_launches": steps + steps // 64}
    out["nonfinite_nodes"] = nonfinite
    if plastic:
        out["weights_changed_frac"] = changed
    return out


def run_test_set(args, local, stream, model: str = "izh"):
    """The paper's own benchmark layout (Sec. 3.4, Sec. 3.5): the 80 networks of the
    standard test set (2 dimensions x 5 sizes x 4 classes x 2 densities) with
    Izhikevich + alpha-PSC nodes at dt = 1 ms for `test_set_steps` steps (10 s of
    simulated time by default), or Hodgkin-Huxley + alpha-PSC nodes at dt = 0.03 ms
    for `test_set_hh_steps` steps (1 s); real-time factor = simulated time / device
    time (CUDA events), one network after another, each from its own graph; then
    all 80 advanced together by the batched form (every network then runs at the
    batch's real-time factor)."""
    import statistics as st
    import torch
    from paper_0908_3934_b300 import geonet
    hh = model == "hh"
    steps = args.test_set_hh_steps if hh else args.test_set_steps
    rows = []
    ispecs = [netgen.test_set_hh(sp) if hh else netgen.test_set_izh(sp) for sp in netgen.test_set()]
    for ispec in ispecs:
        net = geonet.Net(ispec, device=local, stream=stream.cuda_stream, obs_capacity=64)
        net.gn_step(128)
        net.gn_synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        net.gn_step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        net.gn_net_destroy()
        rows.append((ispec.name, ispec.n_nodes, ispec.n_edges, steps * ispec.dt_ms * 1e-3 / t, t))
    # the same 80 networks advanced together by the batched form
    b = geonet.Batch(ispecs, device=local, stream=stream.cuda_stream, obs_capacity=64)
    b.gn_batch_step(128)
    b.gn_batch_synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.gn_batch_step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_batch = ev0.elapsed_time(ev1) / 1e3
    binfo = b.gn_batch_get_info()
    b.gn_batch_destroy()
    dt = ispecs[0].dt_ms
    rtf = [r[3] for r in rows]
    by_class = {}
    for cls in netgen.TEST_SET_CLASSES:
        big = [r[3] for r in rows if f"_{cls}_" in r[0] and r[1] == max(netgen.TEST_SET_SIZES)]
        by_class[cls] = {"min": min(big), "max": max(big)}
    nodes = ("Hodgkin-Huxley + alpha-PSC nodes, dt = 0.03 ms" if hh else "Izhikevich + alpha-PSC nodes, dt = 1 ms")
    return {"details_workload": f"the 80 test-set networks (N = 10 .. 1000, 2D / 3D, lattice / small world / scale free / "
                        f"random, low / high density), {nodes}, {steps} steps each, 20 Hz background pulses",
            "details_metric": "real-time factor (simulated time / device time)",
            "rtf_min": min(rtf), "rtf_median": st.median(rtf), "rtf_max": max(rtf),
            "details_rtf_n1000_by_class": by_class,
            "details_largest": max(rows, key=lambda r: r[2])[0],
            "batched": {"rtf_every_network": steps * dt * 1e-3 / t_batch,
                        "network_seconds_per_second": len(ispecs) * steps * dt * 1e-3 / t_batch,
                        "speedup_vs_one_after_another": sum(r[4] for r in rows) / t_batch,
                        "step_kernel": binfo["step_kernel"], "step_lanes": binfo["step_lanes"],
                        "details_gpu_launches": 2 * ((steps + 63) // 64) if binfo["step_kernel"] == 5
                        else steps * max(1, binfo["step_groups"]) + (steps + 63) // 64},
            "details_networks": [{"name": r[0], "N": r[1], "E": r[2], "rtf": round(r[3], 1)} for r in rows]}


def _host_pool():
    """A process pool for the host-side input generation (networks and their candidate
    tables), started with spawn so no worker inherits the parent's CUDA state."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))


def _estimator_set(specs, chunk: int, local, stream, pool):
    """Features [P, 33], plain scores [P] (device), labels [P] (host) and pairs per
    network of the candidate pairs of `specs`, simulated `chunk` networks at a time
    (one batched run each); rows are grouped by network in order."""
    import torch
    from paper_0908_3934_b300 import pipeline
    feats, score, label, per_net = [], [], [], []
    for c0 in range(0, len(specs), chunk):
        part = specs[c0:c0 + chunk]
        cands = pool.map(netgen.candidates, part, chunksize=32)
        r = pipeline.simulate_features(part, n_samples=500, device=local, stream=stream.cuda_stream, cands=cands)
        feats.append(r["features"])
        score.append(r["score"])
        label.append(r["label"])
        per_net.append(np.bincount(r["net"], minlength=len(part)))
        del r
    cat = (lambda xs: xs[0]) if len(feats) == 1 else torch.cat
    return cat(feats), cat(score), np.concatenate(label), np.concatenate(per_net)


def _train_score(args, tr, te, n_rows, local, stream, seed, timed=False):
    """Train a fresh MLP on the first n_rows training pairs for args.est_epochs epochs
    (visiting orders drawn on the device before the timed region) and score both
    estimators on the held-out pairs (F1 thresholds chosen on the training pairs)."""
    import torch
    from paper_0908_3934_b300 import geonet, pipeline
    Xtr, Str, Ltr = tr[0][:n_rows], tr[1][:n_rows], tr[2][:n_rows]
    dev = Xtr.device
    mlp = geonet.Mlp(netgen.mlp_init(2024), max_batch=8192, device=local, stream=stream.cuda_stream)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    orders = [torch.randperm(n_rows, generator=gen, device=dev) for _ in range(args.est_epochs)]
    yl = torch.from_numpy(Ltr.astype(np.float32)).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = pipeline.train(mlp, Xtr, yl, epochs=args.est_epochs, batch=8192, seed=seed, orders=orders)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del orders
    # F1 thresholds on the first training pairs (the first few hundred training nets)
    n_thr = min(n_rows, args.est_thr_rows)
    p_tr = torch.empty(n_thr, device=dev)
    mlp.gn_mlp_infer(Xtr[:n_thr], p_tr)
    mlp.gn_mlp_synchronize()
    thr_learned, _ = geonet.gn_score_best_f1(p_tr.cpu().numpy(), Ltr[:n_thr])
    thr_plain, _ = geonet.gn_score_best_f1(Str[:n_thr].cpu().numpy(), Ltr[:n_thr])
    p_te = torch.empty(te[0].shape[0], device=dev)
    mlp.gn_mlp_infer(te[0], p_te)
    mlp.gn_mlp_synchronize()
    learned = pipeline.scores(p_te, te[2], thr_learned)
    plain = pipeline.scores(te[1], te[2], thr_plain)
    out = {"auroc_learned": learned["auroc"], "auroc_plain": plain["auroc"], "f1_learned": learned["f1"],
           "f1_plain": plain["f1"], "details_loss_first_last": [losses[0], losses[-1]], "details_pairs": n_rows}
    if timed:
        out["train_samples_per_s"] = n_rows * args.est_epochs / t_train
    return out, mlp


def run_estimator(args, local, stream):
    """Connectivity estimation.  Workload: networks of N = 512 with config-5 laws (2D,
    kept in-degree ~20, 1-8 pulsed nodes, 500 ms observed at 1 ms), `est_train`
    training nets (seeds 10^6 + i) and `est_test` held-out ones (seeds 2 10^6 + i);
    the MLP is trained on the first 500, 2000 and all training nets (the learning
    curve) and both estimators are scored on the held-out nets.  Positive control:
    sparse, independently driven nets (netgen.estimator_control; `est_ctl_train` /
    `est_ctl_test` nets, seeds 3 10^6 + i and 4 10^6 + i), where lagged correlation
    does reveal edges.  Throughput: candidate pairs scored per second by features +
    inference from resident traces, and training samples per second."""
    import functools
    import torch
    from paper_0908_3934_b300 import geonet, pipeline
    pool = _host_pool()
    member = functools.partial(netgen.batch_member, n=512)
    t0 = time.perf_counter()
    tr_specs = pool.map(member, [10**6 + i for i in range(args.est_train)], chunksize=64)
    te_specs = pool.map(member, [2 * 10**6 + i for i in range(args.est_test)], chunksize=64)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    tr = _estimator_set(tr_specs, args.est_chunk, local, stream, pool)
    te = _estimator_set(te_specs, args.est_chunk, local, stream, pool)
    torch.cuda.synchronize()
    t_sim = time.perf_counter() - t0
    # rows of the first n training nets (rows are grouped by network in order)
    counts = np.concatenate([[0], np.cumsum(tr[3])])
    curve = {}
    full = None
    for n_nets in sorted({min(n, args.est_train) for n in (500, 2000, args.est_train)}):
        res, mlp = _train_score(args, tr, te, int(counts[n_nets]), local, stream, seed=2025,
                                timed=n_nets == args.est_train)
        curve[str(n_nets)] = {k: res[k] for k in ("auroc_learned", "auroc_plain", "f1_learned", "f1_plain")}
        if n_nets == args.est_train:
            full = res
            # throughput of scoring: features + inference from resident traces
            tab = pipeline.candidate_table(te_specs[: min(len(te_specs), args.est_chunk)])
            sim = pipeline.simulate_features(te_specs[: min(len(te_specs), args.est_chunk)], n_samples=500,
                                             device=local, stream=stream.cuda_stream)
            dev = sim["features"].device
            pos, srcd = torch.from_numpy(tab["pos"]).to(dev), torch.from_numpy(tab["src"]).to(dev)
            dstd, rad = torch.from_numpy(tab["dst"]).to(dev), torch.from_numpy(tab["radius"]).to(dev)
            P = srcd.shape[0]
            feats = torch.empty((P, 33), dtype=torch.float32, device=dev)
            sc = torch.empty(P, dtype=torch.float32, device=dev)
            p_te = torch.empty(P, device=dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            geonet.gn_xcorr_features(sim["traces"], pos, srcd, dstd, rad, feats, sc, stream=stream.cuda_stream)
            mlp.gn_mlp_infer(feats, p_te)
            ev1.record(stream)
            torch.cuda.synchronize()
            t_score = ev0.elapsed_time(ev1) / 1e3
            full["pairs_scored_per_s"] = P / t_score
            del sim, feats, sc, p_te
        mlp.gn_mlp_destroy()
    del tr, te
    # positive control
    ctl_tr = pool.map(netgen.estimator_control, [3 * 10**6 + i for i in range(args.est_ctl_train)], chunksize=64)
    ctl_te = pool.map(netgen.estimator_control, [4 * 10**6 + i for i in range(args.est_ctl_test)], chunksize=64)
    ctr = _estimator_set(ctl_tr, args.est_chunk, local, stream, pool)
    cte = _estimator_set(ctl_te, args.est_chunk, local, stream, pool)
    pool.close()
    pool.join()
    ctl, mlp = _train_score(args, ctr, cte, ctr[0].shape[0], local, stream, seed=2026)
    mlp.gn_mlp_destroy()
    out = {"details_workload": f"{args.est_train} training + {args.est_test} held-out nets of N=512 (config-5 laws), "
                               f"{int(counts[-1])} training candidate pairs, {args.est_epochs} epochs of batch 8192; "
                               f"control: {args.est_ctl_train} + {args.est_ctl_test} sparse nets driven by 5 Hz "
                               f"background pulses",
           "auroc_learned": full["auroc_learned"], "auroc_plain": full["auroc_plain"],
           "f1_learned": full["f1_learned"], "f1_plain": full["f1_plain"],
           "pairs_scored_per_s": full["pairs_scored_per_s"], "details_unit": "candidate pairs/s (features + inference)",
           "train_samples_per_s": full["train_samples_per_s"],
           "curve_auroc": {k: [v["auroc_plain"], v["auroc_learned"]] for k, v in curve.items()},
           "control_auroc": [ctl["auroc_plain"], ctl["auroc_learned"]],
           "details_curve": curve, "details_control": ctl,
           "details_seconds": {"generate_host": t_gen, "simulate_and_features": t_sim}}
    return out


def strip_details(x):
    """The result without its per-network rows and layout tables (keys starting
    with 'details_'), which go to the --details file only."""
    if isinstance(x, dict):
        return {k: strip_details(v) for k, v in x.items() if not k.startswith("details_")}
    return x


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="roofline",
                    choices=["roofline", "roofline_hubs5", "roofline_slow", "large", "tiny"])
    ap.add_argument("--cpu-steps", type=int, default=30, help="oracle steps of the cpu_baseline sample")
    ap.add_argument("--ref-steps", type=int, default=30, help="oracle steps timed by --impl reference")
    ap.add_argument("--e2e-chunk", type=int, default=1000, help="steps per host round trip in the e2e run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true", help="skip the one-copy-per-core oracle run")
    ap.add_argument("--obs-cap", type=int, default=4096, help="observation rows kept on the device")
    ap.add_argument("--batch-steps", type=int, default=10000, help="steps of the batched measurement")
    ap.add_argument("--loop-sample", type=int, default=32, help="networks timed by the looped comparison")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--sizes", default="large:4000,roofline_hubs5:2000,roofline_slow:2000",
                    help="other sizes of the plain path timed after the headline one (name:steps,...)")
    ap.add_argument("--no-sizes", action="store_true")
    ap.add_argument("--details", default=None, help="write the full result (every row, full precision) here")
    ap.add_argument("--est-train", type=int, default=20000, help="training nets of the estimator measurement")
    ap.add_argument("--est-test", type=int, default=1000, help="held-out nets of the estimator measurement")
    ap.add_argument("--est-epochs", type=int, default=4)
    ap.add_argument("--est-chunk", type=int, default=4096, help="networks simulated per batched run")
    ap.add_argument("--est-thr-rows", type=int, default=4_000_000, help="training pairs the F1 thresholds are chosen on")
    ap.add_argument("--est-ctl-train", type=int, default=2000, help="training nets of the positive control")
    ap.add_argument("--est-ctl-test", type=int, default=200, help="held-out nets of the positive control")
    ap.add_argument("--no-estimator", action="store_true")
    ap.add_argument("--no-izh", action="store_true", help="skip the Izhikevich-model measurement")
    ap.add_argument("--izh-steps", type=int, default=2000)
    ap.add_argument("--no-hh", action="store_true", help="skip the Hodgkin-Huxley-model measurements")
    ap.add_argument("--no-stdp", action="store_true", help="skip the plastic-weight measurement")
    ap.add_argument("--hh-steps", type=int, default=2000)
    ap.add_argument("--no-test-set", action="store_true", help="skip the 80-network test-set sweeps")
    ap.add_argument("--test-set-steps", type=int, default=10000, help="Izhikevich steps per test-set network")
    ap.add_argument("--test-set-hh-steps", type=int, default=33333, help="Hodgkin-Huxley steps per test-set network")
    ap.add_argument("--step-kernel", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                    help="0: autotuned, 1: one row block per CTA, 2: persistent bulk-copy pipelined kernel, "
                         "3: staged tiles (distinct gathers in shared memory), 4: the whole network in one CTA, "
                         "5: staged tiles resident in shared memory across the steps of one launch")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    from paper_0908_3934_b300 import geonet

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    spec = workload(args.workload, rank)
    stream = torch.cuda.Stream(device=dev)
    net = geonet.Net(spec, device=local, stream=stream.cuda_stream, obs_capacity=args.obs_cap,
                     step_kernel=args.step_kernel)
    info = net.gn_net_get_info()
    E, N = spec.n_edges, spec.n_nodes

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    # ---- device-resident throughput: W untimed steps, then exactly K timed steps
    net.gn_step(args.warmup)
    barrier()
    info = net.gn_net_get_info()  # the kernel is chosen on the first gn_step
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    # the W untimed steps again, right before the timed ones: the GPU idled while the
    # clock sampler started, and its first steps after an idle run below full clock
    net.gn_step(args.warmup)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    net.gn_step(args.steps)
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    if info["step_kernel"] in (4, 5):  # one resident / persistent launch and one advance per chunk
        launches = 2 * (-(-args.steps // RESIDENT_CHUNK))
    else:  # one step launch per step, one advance per 64-step graph and per ragged tail
        launches = args.steps + args.steps // 64 + (1 if args.steps % 64 else 0)
    net.gn_observe(discard=True)

    # ---- end to end through the public API: every chunk uploads a new pulse set from
    # host memory (the controls u_j), steps, and reads the observations back into a
    # pinned host buffer
    rng = np.random.default_rng(77 + rank)
    chunk = max(1, args.e2e_chunk)
    n_chunks = max(E2E_MIN_CHUNKS, -(-max(E2E_MIN_STEPS, args.steps) // chunk))
    t_sim = (net.gn_net_get_info()["step"] + chunk) * spec.dt_ms
    pulses = [[(int(j), t_sim + (c * chunk + rng.uniform(0, chunk)) * spec.dt_ms,
                t_sim + (c * chunk + rng.uniform(0, chunk)) * spec.dt_ms + 2.0, 1.0)
               for j in rng.choice(N, min(N, 1000), replace=False)] for c in range(n_chunks + 1)]
    max_rows = min(args.obs_cap, chunk // spec.obs["sample_every"] + 1)
    # two pinned buffers: the observations of one chunk are copied back while the
    # next chunk steps (gn_observe_async), each buffer reused only after its copy
    host = [torch.empty((max_rows, N), dtype=torch.float32, pin_memory=True).numpy() for _ in range(2)]
    net.gn_set_stimulus(pulses[0])
    net.gn_step(chunk)
    net.gn_observe(max_rows, out=host[0])
    barrier()
    h2d = d2h = 0
    t0 = time.perf_counter()
    for c in range(n_chunks):
        net.gn_set_stimulus(pulses[c + 1])
        h2d += 1000 * 24 + 4
        net.gn_step(chunk)
        net.gn_observe_wait()  # the copy into the other buffer (the previous chunk) is done
        rows, _, _ = net.gn_observe_async(host[c % 2], max_rows)
        d2h += rows * N * 4
    net.gn_observe_wait()
    barrier()
    t_e2e = time.perf_counter() - t0
    e2e_steps = n_chunks * chunk

    value, _, t = replica_rate(float(E) * args.steps, t, dev)
    e2e_value, _, t_e2e = replica_rate(float(E) * e2e_steps, t_e2e, dev)
    E_total = value * t / args.steps
    peak, peak_kind = peaks()
    step_s = t / args.steps
    bytes_step = algorithmic_bytes(info, E, N)
    achieved = bytes_step / step_s / 1e9
    bytes_survey = survey_bytes(E, N)
    traffic = traffic_per_launch(KERNEL_NAMES[info["step_kernel"]], args.workload, info["grid"])
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_of(args, spec, world),
        "node_steps_per_s": (value / E_total) * N * world, "rtf": spec.dt_ms * 1e-3 / step_s,
        # frac: the chosen kernel's own format (bytes it must move); frac_survey: the
        # format-independent 14 B per edge-update; frac_dram: ncu's DRAM bytes per launch
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": bytes_step, "kernel": KERNEL_NAMES[info["step_kernel"]],
                     "grid": info["grid"],
                     "bytes_survey": bytes_survey, "frac_survey": bytes_survey / step_s / 1e9 / peak,
                     "frac_dram": traffic / step_s / 1e9 / peak if traffic else None},
        "e2e": {"value": e2e_value, "unit": METRIC,
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                "steps": e2e_steps, "chunks": n_chunks},
        "gpu_launches": launches, "clocks": clocks,
        "details_layout": {"step_kernel": info["step_kernel"], "grid": info["grid"], "cta_threads": info["step_threads"],
                   "edges_per_thread": info["step_edges_per_thread"],
                   "ring_depth": info["ring_depth"], "edge_format": info["edge_format"],
                   "n_blocks": info["n_blocks"], "max_delay": info["max_delay"],
                   "device_bytes": info["device_bytes"]},
    }
    if not args.no_sizes:
        sizes = {}
        for item in args.sizes.split(","):
            name, steps = item.split(":")
            r = run_size(name, int(steps), args.warmup, local, stream, rank)
            sec = r["details_steps"] * r["ms_per_step"] / 1e3
            r["value"], _, _ = replica_rate(r["value"] * sec, sec, dev)
            sizes[name] = r
        line["sizes"] = sizes
    if not args.no_batched:
        bt = run_batched(args, local, stream, rank)
        bt["value"], _, bt["seconds"] = replica_rate(bt["value"] * bt["seconds"], bt["seconds"], dev)
        line["batched"] = bt
    if not args.no_izh and rank == 0:
        line["izhikevich"] = run_spiking(args, spec, local, stream, "izh")
    if not args.no_hh and rank == 0:
        line["hodgkin_huxley"] = run_spiking(args, spec, local, stream, "hh")
    if not args.no_stdp and rank == 0:
        line["izhikevich_stdp"] = run_spiking(args, spec, local, stream, "izh", plastic=True)
    if not args.no_test_set and rank == 0:
        line["test_set"] = run_test_set(args, local, stream)
        if not args.no_hh:
            line["test_set_hh"] = run_test_set(args, local, stream, "hh")
    if not args.no_estimator and rank == 0:
        line["estimator"] = run_estimator(args, local, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(spec, args.cpu_steps)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "host",
                                                   "window_steps", "window_s_extrapolated")}
        if not args.no_cpu_all_cores:
            ac = cpu_baseline_all_cores(args.workload, spec, args.cpu_steps)
            line["cpu_baseline"]["all_cores"] = {k: ac[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        if args.details:
            with open(args.details, "w") as f:
                json.dump(line, f, indent=1)
        print(json.dumps(compact(strip_details(line))), flush=True)
    net.gn_net_destroy()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
