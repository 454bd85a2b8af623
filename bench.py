"""Benchmark of the B300-native VMAS world step.

One "step" = one world step (all substeps fused) of every environment of the
paper-scale workload: 30,000 envs x (16 agent spheres + 4 movable boxes +
4 fixed line walls), 5 substeps, synthetic seeded scenes and uniform [-1, 1]
actions.  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Timing: W untimed warm-up steps; then K steps, each preceded by an L2 flush
(a write and then a read of a buffer twice the L2 size, outside the timed
events) and bracketed by CUDA events on the launching stream; the whole
region is bracketed by a barrier and a device synchronize.  value = env-steps
of all ranks / max over ranks of the summed event time.  Multi-GPU: one
process per GPU (torchrun), each with its own 30,000 envs (weak scaling, no
collective on the data path).

--impl reference times the FP64 oracle (the plain CPU statement of the
method) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import contextlib
import hashlib
import json
import math
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s on 1 B300, plain fused step vs surrogate at stated error; % roofline"
UNIT = "env-steps/s"
# Algorithmic bytes per env-step of the paper-scale workload: state read +
# write (2 x 24 entities x 6 FP32) + the useful action floats
# (16 agents x 2 + 4 boxes x 3).
ENTITIES, AGENTS, BOXES = 24, 16, 4
B_ALG_PER_ENV = 2 * ENTITIES * 6 * 4 + (AGENTS * 2 + BOXES * 3) * 4  # 1328


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _tensor_peak():
    """Dense bf16 TFLOP/s (burst) of the B300s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1800.0, "fallback"


def _hbm_roofline(bytes_per_env_step, env_steps_per_s, note):
    peak, kind = _peaks()
    gbs = bytes_per_env_step * env_steps_per_s / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_source": "%s hbm_gbs" % kind, "bytes_per_env_step": bytes_per_env_step,
            "note": note}


# FP32 operations of one ray against one body, counted from the closed-form
# entry distances of the LIDAR kernel as written (sqrt and divide count one,
# comparisons that feed a branch are not counted), plus one for the running
# minimum; and of one ray direction (angle, sin/cos by the library's own
# reduction and series)
LIDAR_OPS = {"sphere": 12, "box": 28, "line": 13, "ray": 22}


def _issue_roofline(figures, avg_ms, clocks):
    """The instruction-issue bound beside the HBM one: the launch's warp
    instructions (ncu, recorded for these kernel sources) over the SMs' issue
    rate (4 schedulers per SM, one warp instruction per cycle each, at the
    median SM clock sampled during the timed region), against the measured
    mean launch time."""
    if not figures or not figures.get("warp_inst_per_launch"):
        return None
    try:
        import torch

        sms = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        return None
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if not mhz:
        return None
    inst = figures["warp_inst_per_launch"]
    floor_us = inst / (sms * 4 * mhz * 1e6) * 1e6
    return {"warp_inst_per_launch": inst, "sms": sms, "sm_mhz": mhz,
            "issue_floor_us": floor_us, "measured_us": avg_ms * 1e3,
            "frac": floor_us / (avg_ms * 1e3)}


def _alu_roofline(ops_per_unit, units_per_s, note):
    """FP32 ALU roofline: one operation per lane per cycle on every FP32 lane
    (SMs x 128 lanes x the maximum SM clock, 2,032 MHz on B300)."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2.032e9 / 1e12
    achieved = ops_per_unit * units_per_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak, "peak_source": "%d SMs x 128 FP32 lanes x 2.032 GHz" % sms,
            "ops_per_unit": ops_per_unit, "note": note}


# the sources the plain step kernel is compiled from
STEP_KERNEL_SOURCES = ("contact.cuh", "mbar.cuh", "params.cuh", "step.cuh", "step_fused.cuh")


def _code_text(text):
    """C++ source without comments and with whitespace collapsed, so that a
    comment edit does not make a profile of unchanged code look stale."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _kernel_digest():
    h = hashlib.sha256()
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_03530_b300", "csrc", name)) as f:
            h.update(_code_text(f.read()).encode())
    return h.hexdigest()[:16]


def _recorded_profile():
    """(DRAM bytes per launch, headline ncu figures) of the step kernel from
    the committed ncu summary, if it was taken on the current kernel sources;
    (None, None) otherwise."""
    import re

    path = os.path.join(ROOT, "profiles", "world_step_paper30k.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    fields = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel sources sha256 prefix") != _kernel_digest():
        return None, None
    try:
        traffic = float(fields["dram bytes per launch (read+write)"])
    except (KeyError, ValueError):
        return None, None

    def pct(key, pattern):
        m = re.search(pattern, fields.get(key, ""))
        return float(m.group(1)) if m else None

    figures = {
        "dram_throughput_pct": pct("gpu__dram_throughput", r"([\d.]+) %"),
        "issue_active_pct": pct("smsp__issue_active", r"([\d.]+) %"),
        "fma_pipe_pct": pct("pipes (of active)", r"FMA ([\d.]+) %"),
        "warps_per_sm": pct("sm__warps_active", r"([\d.]+) warps"),
        "warp_inst_per_launch": (lambda v: v * 1e6 if v is not None else None)(
            pct("smsp__issue_active", r"smsp__inst_executed: ([\d.]+) M")),
        "binds": "latency: neither HBM nor the FP32 pipes are saturated",
    }
    return traffic, figures


def _recorded_traffic():
    return _recorded_profile()[0]


class ClockSampler:
    """Polls NVML (through ctypes, libnvidia-ml.so.1) for the SM clock and
    the clock-event (throttle) reasons on a background thread."""

    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
               "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}

    def __init__(self, torch_device, period=0.002):
        import ctypes

        self.samples, self.reasons = [], set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._t = None
        self.ok = False
        self.period = period
        try:
            import torch

            L = ctypes.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            h = ctypes.c_void_p()
            pr = torch.cuda.get_device_properties(torch_device)
            bus = getattr(pr, "pci_bus_id", None)
            rc = -1
            if bus is not None:
                busid = "%04x:%02x:%02x.0" % (getattr(pr, "pci_domain_id", 0), bus,
                                             getattr(pr, "pci_device_id", 0))
                rc = L.nvmlDeviceGetHandleByPciBusId_v2(busid.encode(), ctypes.byref(h))
            if rc != 0:
                rc = L.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(torch_device.index or 0),
                                                     ctypes.byref(h))
            if rc != 0:
                raise RuntimeError("no NVML handle")
            self.L, self.h, self.ct = L, h, ctypes
            v = ctypes.c_uint()
            if L.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(v)) == 0:  # NVML_CLOCK_SM
                self.max_mhz = v.value
            self._reasons_fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(L, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.ok = True
        except Exception as e:  # no NVML on this host
            self.err = str(e)

    def _run(self):
        ct, L, h = self.ct, self.L, self.h
        v, bits = ct.c_uint(), ct.c_ulonglong()
        while not self._stop.is_set():
            if L.nvmlDeviceGetClockInfo(h, 1, ct.byref(v)) == 0:
                self.samples.append(v.value)
            if self._reasons_fn(h, ct.byref(bits)) == 0:
                for n, b in self.REASONS.items():
                    if bits.value & b:
                        self.reasons.add(n)
            time.sleep(self.period)

    def __enter__(self):
        # re-entrant: each `with` block adds its samples to the same record,
        # so a form can sample only its timed loops
        if self.ok:
            self._stop = threading.Event()
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *exc):
        if self._t:
            self._stop.set()
            self._t.join()
            self._t = None

    def summary(self):
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "error": getattr(self, "err", "unavailable")}
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons),
                "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(n_envs, substeps, seed, budget_s=20.0):
    """Oracle (FP64 C, OpenMP over envs) on the host cores, on a bounded
    sample of the workload: the first E_s envs of the same scene for T_s
    steps, sized to about `budget_s` seconds."""
    import oracle
    from paper_2207_03530_b300 import scenes

    cores = oracle.max_threads()
    sc = scenes.paper_scene(n_envs, seed, substeps=substeps)
    probe = sc.subset(np.arange(min(n_envs, 4000)))
    act = scenes.make_actions(probe, 2, seed)
    oracle.step(probe, probe.init_state, act[:1], threads=cores)  # warm the thread pool
    t0 = time.perf_counter()
    oracle.step(probe, probe.init_state, act, threads=cores)
    per_env_step = (time.perf_counter() - t0) / (2 * probe.n_envs)
    E_s = min(n_envs, max(1, int(budget_s / per_env_step)))
    T_s = max(1, min(60, int(budget_s / (per_env_step * E_s))))
    sample = sc.subset(np.arange(E_s))
    act = scenes.make_actions(sample, T_s, seed)
    t0 = time.perf_counter()
    oracle.step(sample, sample.init_state, act, threads=cores)
    dt = time.perf_counter() - t0
    # one thread, on the probe sample
    act1 = scenes.make_actions(probe, 1, seed)
    t1 = time.perf_counter()
    oracle.step(probe, probe.init_state, act1, threads=1)
    single = probe.n_envs / (time.perf_counter() - t1)
    return {"value": E_s * T_s / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d of %d envs x %d steps of the same workload, FP64, %.1f s"
                      % (E_s, n_envs, T_s, dt),
            "single_thread_value": single,
            "single_thread_sample": "first %d envs x 1 step, 1 thread" % probe.n_envs}


def run_reference(args):
    """The oracle as the reference arm: each step is one FP64 world step of
    the first E_s envs of the same workload on the host cores (state carried
    across steps), E_s sized so the whole run takes about two minutes."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2207_03530_b300 import scenes

    cores = oracle.max_threads()
    sc = scenes.paper_scene(args.envs, args.seed, substeps=args.substeps)
    probe = sc.subset(np.arange(min(args.envs, 1000)))
    t0 = time.perf_counter()
    oracle.step(probe, probe.init_state, scenes.make_actions(probe, 1, args.seed), threads=cores)
    per_env_step = (time.perf_counter() - t0) / probe.n_envs
    n = args.warmup + args.steps
    budget = min(20.0, max(0.05, 120.0 / max(1, n)))
    E_s = int(min(args.envs, max(8, budget / per_env_step)))
    sample = sc.subset(np.arange(E_s))
    act = scenes.make_actions(sample, n, args.seed)
    state = sample.init_state.astype(np.float64)
    times = []
    for k in range(n):
        t0 = time.perf_counter()
        state = oracle.step(sample, state, act[k], threads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = E_s * len(times) / sum(times)
    base = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d of %d envs of the same workload, %d timed steps, FP64 C + OpenMP"
                      % (E_s, args.envs, len(times))}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * args.envs / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args), "cpu_baseline": base,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(args):
    return {"workload": "paper-scale plain step: %d envs x (16 agent spheres + 4 movable boxes "
                        "+ 4 fixed line walls), %d substeps" % (args.envs, args.substeps),
            "n_envs_per_gpu": args.envs, "entities_per_env": ENTITIES, "substeps": args.substeps,
            "seed": args.seed, "parallelism": "env-sharded replicas, no collective",
            "l2": "flushed before every timed step (write+read of 2x L2)"}


def run_native(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2207_03530_b300 import World, build, scenes

    build.build()
    sc = scenes.paper_scene(args.envs, args.seed + rank, substeps=args.substeps)
    world = World(sc)
    E, A = sc.n_envs, sc.n_actuated
    T = args.warmup + args.steps
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 + args.seed + rank)
    actions = torch.rand((T, E, A, 3), device=dev, generator=gen) * 2 - 1
    props = torch.cuda.get_device_properties(dev)
    l2 = getattr(props, "L2_cache_size", 126 << 20) or (126 << 20)
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device=dev)

    def flush_l2():
        flush.zero_()
        flush.sum()

    for t in range(args.warmup):
        flush_l2()
        world.step(actions[t])
    world.check()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with sampler:
        for k in range(args.steps):
            flush_l2()
            starts[k].record()
            world.step(actions[args.warmup + k])
            ends[k].record()
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    world.check()
    kern_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(kern_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = E * args.steps * ws / (total_ms / 1e3)

    # warm-L2 figure (no flush), for context only
    torch.cuda.synchronize()
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record()
    for k in range(args.steps):
        world.step(actions[args.warmup + k])
    w1.record()
    torch.cuda.synchronize()
    warm = E * args.steps / (w0.elapsed_time(w1) / 1e3)

    if args.stats:
        world.enable_stats(True)
        for k in range(args.steps):
            world.step(actions[args.warmup + k])
        st = world.stats(reset=True)
        world.enable_stats(False)
        n = max(1, st["env_steps"])
        print("[stats per env-step] " + " ".join("%s=%.3f" % (k, v / n) for k, v in st.items()),
              file=sys.stderr, flush=True)

    # end to end through the C ABI with host buffers: every step's actions
    # up from pinned host memory and its full state back to pinned host
    # memory (vmas_rollout_host: copies overlap the steps on copy streams)
    e2e = None
    if not args.no_e2e:
        K2 = min(args.steps, 20)
        h_act = torch.empty((K2, E, A, 3), dtype=torch.float32).pin_memory()
        h_act.copy_(actions[args.warmup:args.warmup + K2].cpu())
        h_states = torch.empty((K2, E, sc.n_entities, 6), dtype=torch.float32).pin_memory()
        world.rollout_host(h_act[:2], h_states[:2])  # allocates the streaming buffers
        # untimed warm-up over the same host buffers: the first DMA pass over
        # freshly pinned memory runs ~1.5x slower than every later one
        # (reported as cold_first_call)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        world.rollout_host(h_act, h_states)
        cold_s = time.perf_counter() - t0
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        world.rollout_host(h_act, h_states)  # returns when every state has arrived
        e2e_s = time.perf_counter() - t0
        h_state = h_states[0]
        if dist:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": E * K2 * ws / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h_act[0].numel() * 4),
               "d2h_bytes_per_step": int(h_state.numel() * 4),
               "steps": K2, "cold_first_call_value": E * K2 * ws / cold_s}

    peak, peak_kind = _peaks()
    avg_ms = statistics.mean(kern_ms)
    achieved = B_ALG_PER_ENV * E / (avg_ms / 1e3) / 1e9
    traffic, ncu_figures = _recorded_profile()
    clocks = sampler.summary()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(args),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": "%s hbm_gbs (burst copy)" % peak_kind,
                         "traffic_source": ("ncu capture of these kernel sources, read from the "
                                            "committed summary (not measured in this run)"
                                            if traffic is not None else None),
                         "bytes_per_env_step": B_ALG_PER_ENV, "kernel": "world_step_kernel",
                         "ncu": ncu_figures,
                         "issue": _issue_roofline(ncu_figures, avg_ms, clocks)},
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "warm_l2_value": warm,
            "wall_s_timed_region": wall,
        }
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.envs, args.substeps, args.seed,
                                                budget_s=args.cpu_budget)
        print(json.dumps(line), flush=True)
    world.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_adjoint(args):
    """Differentiable rollout workload: 4,096 envs x (8 agents + 2
    landmarks), 3 substeps, 50 steps, checkpoint every 10.  Times forward +
    backward (hand-written adjoint) and the plain step on the same scene,
    and checks 4 sampled envs' gradients against the FP64 oracle."""
    import torch

    from paper_2207_03530_b300 import World, build, scenes
    from paper_2207_03530_b300.diff import rollout_loss

    build.build()
    torch.cuda.set_device(0)
    E, T, K = args.envs if args.envs != 30000 else 4096, 50, 10
    sc = scenes.diff_scene(E, args.seed)
    w = World(sc)
    act = torch.from_numpy(scenes.make_actions(sc, T, args.seed + 1)).cuda()
    goals = torch.from_numpy(scenes.make_goals(sc, args.seed + 2)).cuda()

    def fwd_bwd():
        a = act.detach().requires_grad_(True)  # a fresh leaf on the same storage
        rollout_loss(w, a, goals, ckpt_every=K).sum().backward()
        return a.grad

    for _ in range(args.warmup):
        fwd_bwd()
    torch.cuda.synchronize()
    cs = ClockSampler(torch.device("cuda", 0))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with cs:
        t0.record()
        for _ in range(args.steps):
            grad = fwd_bwd()
        t1.record()
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    # the same forward + backward captured once into a CUDA graph (autograd
    # included) and replayed: no host work per iteration
    graph_ms = None
    try:
        static_a = act.detach().clone().requires_grad_(True)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                static_a.grad = None
                rollout_loss(w, static_a, goals, ckpt_every=K).sum().backward()
        torch.cuda.current_stream().wait_stream(side)
        static_a.grad = None
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            rollout_loss(w, static_a, goals, ckpt_every=K).sum().backward()
        g.replay()
        torch.cuda.synchronize()
        if not torch.equal(static_a.grad, grad):
            raise RuntimeError("graphed gradient differs")
        with cs:
            t0.record()
            for _ in range(args.steps):
                g.replay()
            t1.record()
            torch.cuda.synchronize()
        graph_ms = t0.elapsed_time(t1) / args.steps
    except Exception as exc:  # capture is an optional extra measurement
        print("graph capture of the adjoint skipped: %s" % exc, file=sys.stderr)
    # plain fused step on the same scene, same actions
    for t in range(3):
        w.step(act[t])
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    w.rollout(act)
    p1.record()
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    # accuracy on 4 sampled envs
    import oracle

    pick = np.array([0, E // 3, 2 * E // 3, E - 1])
    sub = sc.subset(pick)
    a_np, g_np = act.cpu().numpy(), goals.cpu().numpy()
    _, ref = oracle.rollout_grad(sub, sub.init_state, a_np[:, pick], g_np[pick])
    got = grad.cpu().numpy()[:, pick]
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    w.close()
    # per env-step: actions read by the forward and by the backward, the
    # action gradient written, checkpoints (x, y, vx, vy of every entity every
    # K steps) written and read back
    A_, N_ = sc.n_actuated, sc.n_entities
    b_env = 2 * A_ * 12 + A_ * 12 + 2 * N_ * 16 / K
    print(json.dumps({
        "form": "adjoint", "metric": "env-steps/s, differentiable rollout forward + backward",
        "value": E * T / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms,
        "graphed_value": E * T / (graph_ms / 1e3) if graph_ms else None,
        "graphed_ms_per_rollout": graph_ms,
        "roofline": _hbm_roofline(b_env, E * T / (ms / 1e3),
                                  "latency-bound (ncu: diff_backward_kernel)"),
        "plain_step_value": E * T / (plain_ms / 1e3), "rollout_steps": T, "ckpt_every": K,
        "grad_rel_err_vs_fp64_oracle": err, "clocks": cs.summary(),
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%d envs x (8 agent spheres + 2 landmarks), 3 substeps, %d steps"
                               % (E, T)}}), flush=True)
    return 0


def run_ragged(args):
    """Ragged batching workload: 65,536 envs of 2-64 agents,
    0-8 boxes, 0-4 walls, packed without padding; autotuned lanes per env and
    steps per launch; a 500-step rollout captured in a CUDA graph.  Also
    times the same scene padded to its largest env on the regular world."""
    import torch

    from paper_2207_03530_b300 import World, build, scenes
    from paper_2207_03530_b300.ragged import RaggedWorld

    build.build()
    torch.cuda.set_device(0)
    E = args.envs if args.envs != 30000 else 65536
    T = 500
    sc, counts = scenes.ragged_scene(E, args.seed)
    pk = scenes.pack_ragged(sc, counts)
    rw = RaggedWorld(counts, pk["shape"], pk["flags"], pk["size_a"], pk["size_b"], pk["mass"],
                     pk["inertia"], pk["init_state"], substeps=sc.substeps, dt=sc.dt, drag=sc.drag)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed + 3)
    act = torch.rand((T, rw.n_action_rows, 3), device="cuda", generator=gen) * 2 - 1
    rw.autotune(act[:64])
    lanes, tile = rw.tuning()
    schedule = rw.schedule
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps // 100)
    cs = ClockSampler(torch.device("cuda", 0))
    start = rw.state()

    def timed_rollout():
        rw.set_state(start)
        rw.rollout(act)  # captures the graph on first use
        torch.cuda.synchronize()
        with cs:
            a.record()
            for _ in range(reps):
                rw.rollout(act)
            b.record()
            torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms = timed_rollout()
    value = E * T / (ms / 1e3)
    # A/B of the two schedules: one launch per size class (autotuned lanes)
    # against one persistent launch over every class (atomic work queue), at
    # several steps per launch
    names = {0: "per-class", 1: "persistent-128reg", 2: "persistent-96reg"}
    ab = []
    for sched in (0, 1, 2):
        for t in sorted({tile, 8, 16, 32}):
            rw.schedule = sched
            rw.set_tuning(lanes, t)
            ab.append({"schedule": names[sched], "steps_per_launch": t,
                       "env_steps_per_s": E * T / (timed_rollout() / 1e3)})
    rw.schedule = schedule
    rw.set_tuning(lanes, tile)
    rw.close()
    del act
    # the same scene padded to the largest env, regular world, one step at a time
    w = World(sc)
    pact = torch.rand((20, E, sc.n_actuated, 3), device="cuda", generator=gen) * 2 - 1
    for t in range(3):
        w.step(pact[t])
    torch.cuda.synchronize()
    a.record()
    for t in range(3, 20):
        w.step(pact[t])
    b.record()
    torch.cuda.synchronize()
    padded = E * 17 / (a.elapsed_time(b) / 1e3)
    w.close()
    # per env-step: the state of every entity read and written once per
    # launch of `tile` steps (it stays on chip in between), the useful action
    # rows every step
    b_env = (int(counts.sum()) * 48 / tile + int(rw.n_action_rows) * 12) / E
    print(json.dumps({
        "form": "ragged", "metric": "env-steps/s, ragged rollout (CUDA graph, autotuned)",
        "value": value, "unit": UNIT, "ms_per_rollout": ms, "rollout_steps": T,
        "roofline": _hbm_roofline(b_env, value, "latency-bound size classes "
                                  "(ncu: the 128-entity class)"),
        "entities": int(counts.sum()), "envs": E, "lanes_per_class": [int(x) for x in lanes],
        "steps_per_launch": tile, "schedule": names[schedule],
        "schedules_ab": ab, "padded_regular_world_value": padded, "clocks": cs.summary(),
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "%d envs x (2-64 agents + 0-8 boxes + 0-4 walls), 5 substeps, "
                               "%d-step graph rollout" % (E, T)}}), flush=True)
    return 0


def _sur_rollouts(sur, sc, act, runs, World, cs=None):
    """The same 50-step rollout from sc's start with the plain step and with
    the surrogate in each inference mode; per-step CUDA events (median after
    3 steps), agent positions kept for the error."""
    import torch

    T, E = act.shape[0], sc.n_envs
    out = {}
    for name, mode in runs:
        if mode:
            sur.set_mode(mode)
        w = World(sc)
        nfb = torch.zeros(T, dtype=torch.int32, device="cuda")
        pos = torch.empty((T, E, 16, 2), device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * T)]
        with (cs if cs is not None else contextlib.nullcontext()):
            for t in range(T):
                ev[2 * t].record()
                if mode:
                    sur.step(w, act[t], n_fallback=nfb[t:t + 1])
                else:
                    w.step(act[t])
                ev[2 * t + 1].record()
                pos[t] = w.state()[:, :16, :2]
            torch.cuda.synchronize()
        ms = [ev[2 * t].elapsed_time(ev[2 * t + 1]) for t in range(T)]
        out[name] = dict(pos=pos, ms=statistics.median(ms[3:]), nfb=nfb.cpu().numpy(),
                         value=E / (statistics.median(ms[3:]) / 1e3))
        w.close()
    return out


def _pos_err(a, b):
    d = (a - b).norm(dim=-1)  # [T, E, 16]
    return float(d.mean().item()), float(d[-1].mean().item())


def run_surrogate(args):
    """Learned surrogate workload: 262,144 envs x 16 agent spheres
    (+ 4 walls), 50-step rollouts.  For each substep count S in (5, 1) the
    network is trained on the GPU with the library's own forward / backward /
    Adam kernels on transitions of the plain step at S substeps; then the
    same 50 steps run from the same start with the plain step at S (the
    reference for the error) and with the surrogate and its plain-step fallback.
    Reports env-steps/s of each and the mean agent position error; at S = 5
    also the plain step at 1 substep against the 5-substep reference (the
    cheap method without a network)."""
    import torch

    from paper_2207_03530_b300 import World, build, scenes
    from paper_2207_03530_b300.surrogate import Surrogate, train_on_plain_step

    build.build()
    torch.cuda.set_device(0)
    E = args.envs if args.envs != 30000 else 262144
    T = 50
    E_train = min(E, args.train_envs)
    sc5 = scenes.surrogate_scene(E, args.seed)
    sc1 = dataclasses_replace(sc5, substeps=1)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed + 5)
    act = torch.rand((T, E, 16, 3), device="cuda", generator=gen) * 2 - 1
    res = {}
    cs = ClockSampler(torch.device("cuda", 0))
    for S, sc in ((5, sc5), (1, sc1)):
        sur = Surrogate(max(E, E_train), seed=args.seed)
        train = train_on_plain_step(sur, E_train, args.train_steps, args.lr, args.seed + 1000,
                                    substeps=S, log=sys.stderr)
        runs = [("plain", False), ("surrogate", "fused"), ("surrogate_layered", "layered")]
        if S == 5:
            runs.append(("plain_s1", None))
        out = _sur_rollouts(sur, sc, act, [r for r in runs if r[1] is not None], World, cs)
        if S == 5:
            out.update(_sur_rollouts(sur, sc1, act, [("plain_s1", False)], World, cs))
        sur.close()
        ref = out["plain"]["pos"]
        e, e_end = _pos_err(out["surrogate"]["pos"], ref)
        res[S] = {
            "plain_value": out["plain"]["value"], "surrogate_value": out["surrogate"]["value"],
            "layered_surrogate_value": out["surrogate_layered"]["value"],
            "surrogate_ms_per_step": out["surrogate"]["ms"],
            "surrogate_mean_pos_err_50": e, "surrogate_pos_err_at_50": e_end,
            "fallback_envs_per_step": float(out["surrogate"]["nfb"].mean()),
            "train": {"seconds": train[0], "transitions": train[2], "envs": E_train,
                      "steps": args.train_steps, "final_loss": train[1], "lr": args.lr}}
        if S == 5:
            e1, e1_end = _pos_err(out["plain_s1"]["pos"], ref)
            res[S].update({"plain_s1_value": out["plain_s1"]["value"],
                           "plain_s1_mean_pos_err_50": e1, "plain_s1_pos_err_at_50": e1_end})
        del out
    # the box world (the paper-scale scene: 16 agents, 4 boxes, 4 walls), the
    # network trained on its plain-step transitions and run on the layered
    # (tcgen05) path; errors for the agents and for the boxes
    scb = scenes.paper_scene(E, args.seed)
    actb = torch.rand((T, E, scb.n_actuated, 3), device="cuda", generator=gen) * 2 - 1
    surb = Surrogate(max(E, E_train), seed=args.seed)
    trainb = train_on_plain_step(surb, E_train, args.train_steps, args.lr, args.seed + 2000,
                                 log=sys.stderr, boxes=True)
    box_res = {}
    for name, mode, sc_ in (("plain", False, scb), ("surrogate", "layered", scb),
                            ("plain_s1", False, dataclasses_replace(scb, substeps=1))):
        w = World(sc_)
        pos = torch.empty((T, E, 20, 2), device="cuda")
        nfb = torch.zeros(T, dtype=torch.int32, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * T)]
        with cs:
            for t in range(T):
                ev[2 * t].record()
                if mode:
                    surb.step(w, actb[t], n_fallback=nfb[t:t + 1])
                else:
                    w.step(actb[t])
                ev[2 * t + 1].record()
                pos[t] = w.state()[:, :20, :2]
            torch.cuda.synchronize()
        ms = statistics.median(ev[2 * t].elapsed_time(ev[2 * t + 1]) for t in range(3, T))
        box_res[name] = dict(pos=pos, value=E / (ms / 1e3), nfb=float(nfb.float().mean()))
        w.close()
    surb.check()
    surb.close()
    refb = box_res["plain"]["pos"]

    def body_err(p_):
        d = (p_ - refb).norm(dim=-1)
        return float(d[..., :16].mean()), float(d[..., 16:].mean())

    box_world = {
        "workload": "%d envs x (16 agent spheres + 4 movable boxes + 4 walls), 5 substeps, "
                    "%d steps" % (E, T),
        "plain_value": box_res["plain"]["value"],
        "surrogate_value": box_res["surrogate"]["value"],
        "surrogate_mean_pos_err_50_agents_boxes": body_err(box_res["surrogate"]["pos"]),
        "plain_s1_value": box_res["plain_s1"]["value"],
        "plain_s1_mean_pos_err_50_agents_boxes": body_err(box_res["plain_s1"]["pos"]),
        "fallback_envs_per_step": box_res["surrogate"]["nfb"],
        "train": {"seconds": trainb[0], "transitions": trainb[2], "envs": E_train,
                  "steps": args.train_steps, "final_loss": trainb[1], "lr": args.lr}}
    del box_res, refb
    r5 = res[5]
    # useful network FLOPs per env: the edge MLP on every present edge (up to
    # 6 nearest agents within 0.3, counted on the start state) and the node
    # MLP on the 16 agents
    xy = sc5.init_state[:, :16, :2].astype(np.float64)
    d = np.linalg.norm(xy[:, :, None, :] - xy[:, None, :, :], axis=-1)
    d[:, np.arange(16), np.arange(16)] = np.inf
    edges = float(np.minimum((d < 0.3).sum(-1), 6).sum(-1).mean())
    flop_env = 2.0 * (edges * (16 * 64 + 64 * 64) + 16 * (80 * 128 + 128 * 128 + 128 * 8))
    tpeak, tkind = _tensor_peak()
    tflops = flop_env * r5["surrogate_value"] / 1e12
    roof = {"bound": "tensor", "achieved": tflops, "peak": tpeak, "unit": "TFLOP/s",
            "frac": tflops / tpeak, "peak_source": "%s bf16_tflops (burst)" % tkind,
            "flop_per_env": flop_env, "edges_per_env": edges,
            "note": "instruction-issue-bound on the GELUs, not on the tensor pipe "
                    "(ncu: sur_fused_kernel)"}
    print(json.dumps({
        "form": "surrogate",
        "metric": "env-steps/s, learned surrogate step (with plain-step fallback)",
        "value": r5["surrogate_value"], "unit": UNIT, "ms_per_step": r5["surrogate_ms_per_step"],
        "roofline": roof,
        "plain_s5_value": r5["plain_value"], "plain_s1_value": r5["plain_s1_value"],
        "layered_surrogate_value": r5["layered_surrogate_value"],
        "surrogate_mean_pos_err_50": r5["surrogate_mean_pos_err_50"],
        "surrogate_pos_err_at_50": r5["surrogate_pos_err_at_50"],
        "plain_s1_mean_pos_err_50": r5["plain_s1_mean_pos_err_50"],
        "plain_s1_pos_err_at_50": r5["plain_s1_pos_err_at_50"],
        "fallback_envs_per_step": r5["fallback_envs_per_step"], "train": r5["train"],
        "substeps_1": {k: v for k, v in res[1].items()}, "box_world": box_world,
        "clocks": cs.summary(),
        "dtype": "bf16 network / f32 fallback", "data": "synthetic",
        "config": {"workload": "%d envs x (16 agent spheres + 4 walls), 5 (and 1) substeps, "
                               "%d steps" % (E, T)}}), flush=True)
    return 0


def dataclasses_replace(scene, **kw):
    import dataclasses

    return dataclasses.replace(scene, **kw)


def run_sweep(args):
    """Plain step at E in {1k, 4k, 16k, 30k, 131k, 262k} envs of the
    paper-scale scene (the larger points hold more state than L2): per-step
    CUDA events with the L2 flushed before each step, as in the headline."""
    import torch

    from paper_2207_03530_b300 import World, build, scenes

    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    props = torch.cuda.get_device_properties(dev)
    l2 = getattr(props, "L2_cache_size", 126 << 20) or (126 << 20)
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device=dev)
    peak, peak_kind = _peaks()
    points = []
    steps = min(args.steps, 50)
    cs = ClockSampler(dev)
    for E in (1000, 4000, 16000, 30000, 131072, 262144):
        sc = scenes.paper_scene(E, args.seed, substeps=args.substeps)
        w = World(sc)
        gen = torch.Generator(device=dev)
        gen.manual_seed(1000 + args.seed)
        act = torch.rand((3 + steps, E, sc.n_actuated, 3), device=dev, generator=gen) * 2 - 1
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
        with cs:
            for t in range(3 + steps):
                flush.zero_()
                flush.sum()
                if t >= 3:
                    ev[2 * (t - 3)].record()
                w.step(act[t])
                if t >= 3:
                    ev[2 * (t - 3) + 1].record()
            torch.cuda.synchronize()
        w.check()
        ms = statistics.mean(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps))
        gbs = B_ALG_PER_ENV * E / (ms / 1e3) / 1e9
        points.append({"envs": E, "state_mb": round(E * 24 * 6 * 4 / 1e6, 1),
                       "us_per_step": round(ms * 1e3, 2), "env_steps_per_s": E / (ms / 1e3),
                       "achieved_gbs": gbs, "hbm_frac": gbs / peak})
        w.close()
        del act
    print(json.dumps({"form": "sweep", "metric": "env-steps/s vs env count, plain step",
                      "unit": UNIT, "peak_gbs": peak, "peak_source": peak_kind,
                      "l2_mb": l2 / 1e6, "points": points, "clocks": cs.summary(),
                      "config": {"workload": "paper-scale scene (16 spheres + 4 boxes + 4 walls), "
                                             "5 substeps, L2 flushed before every step"}}),
          flush=True)
    return 0


def run_rollout(args):
    """Open-loop rollout of the paper-scale workload (every step's actions
    known ahead): args.steps world steps through vmas_rollout with 1, 2, 4, 8
    and 16 steps per launch, the L2 flushed before each rollout.  The state
    and the candidate lists stay on chip between the steps of a launch, so
    the state crosses HBM once per launch; the final states are checked
    bitwise equal across the tilings."""
    import torch

    from paper_2207_03530_b300 import World, build, scenes

    build.build()
    torch.cuda.set_device(0)
    sc = scenes.paper_scene(args.envs, args.seed, substeps=args.substeps)
    E, A = sc.n_envs, sc.n_actuated
    T = max(args.steps, 16)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1000 + args.seed)
    act = torch.rand((T, E, A, 3), device="cuda", generator=gen) * 2 - 1
    l2 = getattr(torch.cuda.get_device_properties(0), "L2_cache_size", 126 << 20) or (126 << 20)
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows, ref = [], None
    cs = ClockSampler(torch.device("cuda", 0))
    for tile in (1, 2, 4, 8, 16):
        w = World(sc)
        w.set_rollout_tile(tile)
        w.rollout(act[:tile])  # lazy kernel loading, off the clock
        w.set_state(sc.init_state)
        flush.zero_()
        flush.sum()
        torch.cuda.synchronize()
        with cs:
            a.record()
            w.rollout(act)
            b.record()
            torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        st = w.state().cpu().numpy()
        w.check()
        w.close()
        ref = st if ref is None else ref
        rows.append({"steps_per_launch": tile, "us_per_step": 1e3 * ms / T,
                     "env_steps_per_s": E * T / (ms / 1e3),
                     "bitwise_equal_one_step_launches": bool(np.array_equal(
                         st.view(np.uint32), ref.view(np.uint32)))})
    best = max(rows, key=lambda r: r["env_steps_per_s"])
    # per env-step: the useful action floats every step, the state read and
    # written once per launch
    state_b = 2 * ENTITIES * 6 * 4
    b_env = B_ALG_PER_ENV - state_b + state_b / best["steps_per_launch"]
    print(json.dumps({
        "form": "rollout", "metric": "env-steps/s, open-loop rollout (world steps per launch)",
        "value": best["env_steps_per_s"], "unit": UNIT, "steps_per_launch": best["steps_per_launch"],
        "tilings": rows, "rollout_steps": T, "clocks": cs.summary(),
        "roofline": _hbm_roofline(b_env, best["env_steps_per_s"],
                                  "latency-bound like the one-step launch; the state "
                                  "crosses HBM once per launch"),
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%d envs x (16 agent spheres + 4 boxes + 4 walls), %d substeps, "
                               "%d-step rollout" % (E, args.substeps, T)}}), flush=True)
    return 0


def run_small(args):
    """Small workload: 32 envs x (4 agents + 2 landmarks),
    1 substep, 100 steps: latency per step, launched one by one, replayed
    from a CUDA graph captured around the same 100 launches, and (when the
    actions are known ahead) all 100 steps in one launch.  A roofline
    fraction at 4.6 KB of state is meaningless; it is reported, labelled
    latency-bound."""
    import torch

    from paper_2207_03530_b300 import World, build, scenes

    build.build()
    torch.cuda.set_device(0)
    sc = scenes.small_scene(32, args.seed)
    T = 100
    w = World(sc)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1000 + args.seed)
    act = torch.rand((T, sc.n_envs, sc.n_actuated, 3), device="cuda", generator=gen) * 2 - 1
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for t in range(T):  # warm-up (lazy loading) off the capture
            w.step(act[t])
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    cs = ClockSampler(torch.device("cuda", 0))
    with cs:
        a.record()
        for _ in range(reps):
            for t in range(T):
                w.step(act[t])
        b.record()
        torch.cuda.synchronize()
    eager_us = a.elapsed_time(b) * 1e3 / (reps * T)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for t in range(T):
            w.step(act[t])
    g.replay()
    torch.cuda.synchronize()
    with cs:
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
    graph_us = a.elapsed_time(b) * 1e3 / (reps * T)
    # the same 100 steps as one launch (an open-loop rollout: every step's
    # actions known ahead)
    w.set_rollout_tile(T)
    w.rollout(act)
    torch.cuda.synchronize()
    with cs:
        a.record()
        for _ in range(reps):
            w.rollout(act)
        b.record()
        torch.cuda.synchronize()
    one_launch_us = a.elapsed_time(b) * 1e3 / (reps * T)
    w.check()
    w.close()
    peak, peak_kind = _peaks()
    b_env = 6 * 24 * 2 + 4 * 8  # state read + write, 4 agents x 2 action floats
    gbs = b_env * 32 / (graph_us / 1e6) / 1e9
    print(json.dumps({
        "form": "small", "metric": "us per step (latency), 100-step rollout",
        "value": graph_us, "unit": "us/step", "higher_is_better": False,
        "eager_us_per_step": eager_us, "graph_us_per_step": graph_us,
        "one_launch_rollout_us_per_step": one_launch_us,
        "env_steps_per_s_graph": 32 / (graph_us / 1e6), "clocks": cs.summary(),
        "roofline": {"bound": "latency", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "bytes_per_env_step": b_env,
                     "note": "4.6 KB of state: launch- and latency-bound"},
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "32 envs x (4 agent spheres + 2 landmarks), 1 substep, 100 steps"}}),
        flush=True)
    return 0


def run_lidar(args):
    """LIDAR on the paper-scale scene: 20 agents x 32 rays per env, with the
    culled kernel (the default) and, for comparison, every ray against every
    body."""
    import torch

    from paper_2207_03530_b300 import World, _lib, build, scenes

    build.build()
    torch.cuda.set_device(0)
    L = _lib.load()
    sc = scenes.paper_scene(args.envs, args.seed)
    w = World(sc)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cs = ClockSampler(torch.device("cuda", 0))

    def timed(cull):
        _lib.check(L.vmas_debug_lidar_cull(1 if cull else 0))
        try:
            for _ in range(max(3, args.warmup)):
                w.lidar(32, 1.0)
            torch.cuda.synchronize()
            with cs:
                a.record()
                for _ in range(args.steps):
                    w.lidar(32, 1.0)
                b.record()
                torch.cuda.synchronize()
        finally:
            _lib.check(L.vmas_debug_lidar_cull(1))
        return a.elapsed_time(b) / args.steps

    ms_full = timed(False)
    ms = timed(True)
    rays = args.envs * sc.n_actuated * 32
    w.close()
    # every-ray kernel: bodies each ray is tested against (every other
    # collidable entity; the casters are spheres or boxes)
    coll = (np.asarray(sc.flags[0]) & scenes.COLLIDABLE) != 0
    shape = np.asarray(sc.shape[0])
    ops = (LIDAR_OPS["ray"] + LIDAR_OPS["sphere"] * (int((coll & (shape == 0)).sum()) - 1)
           + LIDAR_OPS["box"] * int((coll & (shape == 1)).sum())
           + LIDAR_OPS["line"] * int((coll & (shape == 2)).sum()))
    value, full_value = rays / (ms / 1e3), rays / (ms_full / 1e3)
    # algorithmic bytes per ray: its reading, and its share of the env's
    # inputs (x, y, angle, packed parameters, kind byte of every entity)
    b_ray = 4.0 + sc.n_entities * (3 * 4 + 16 + 1) / (sc.n_actuated * 32)
    print(json.dumps({"form": "lidar", "metric": "rays/s", "value": value,
                      "unit": "rays/s", "ms_per_call": ms, "env_scans_per_s": args.envs / (ms / 1e3),
                      "roofline": _hbm_roofline(b_ray, value, "culled kernel; instruction-issue-"
                                                "bound, not HBM-bound (ncu: lidar_cull_kernel)"),
                      "every_ray": {"value": full_value, "ms_per_call": ms_full,
                                    "roofline": _alu_roofline(ops, full_value,
                                                              "instruction-issue-bound (ncu: "
                                                              "lidar_kernel)")},
                      "clocks": cs.summary(), "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "%d envs x 20 agents x 32 rays vs 24 bodies"
                                             % args.envs}}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--form", choices=["plain", "adjoint", "lidar", "ragged", "surrogate",
                                       "sweep", "small", "rollout"],
                    default="plain",
                    help="plain: the fused world step (the headline); adjoint: "
                         "differentiable rollout forward + backward")
    ap.add_argument("--envs", type=int, default=30000)
    ap.add_argument("--substeps", type=int, default=5)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--train-envs", type=int, default=65536, help="surrogate form")
    ap.add_argument("--train-steps", type=int, default=1500, help="surrogate form")
    ap.add_argument("--lr", type=float, default=2e-3, help="surrogate form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of host work the CPU-baseline sample is sized to")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling)")
    ap.add_argument("--stats", action="store_true",
                    help="print step counters per env-step to stderr (extra pass)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.steps > 2:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "adjoint":
        return run_adjoint(args)
    if args.form == "lidar":
        return run_lidar(args)
    if args.form == "ragged":
        return run_ragged(args)
    if args.form == "surrogate":
        return run_surrogate(args)
    if args.form == "sweep":
        return run_sweep(args)
    if args.form == "small":
        return run_small(args)
    if args.form == "rollout":
        return run_rollout(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
