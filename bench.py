"""Benchmark of the VOPP planning hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vopp|reference]
                    [--workload nav1024_d4 | nav256_d3 | grid2048_d5]

One step = one full plan (root preparation, every level's expansion, the fused leaf
expansion and backup, the FP64 root and the action choice) of the default workload: a
2-D navigation POMDP with 1024 root particles uniform in [0,10]^2, depth 4, 4 actions x 4
observation branches (65,536 leaves, 7.16e7 particle-steps by the sum_l (A W)^l N rule),
eta = 0.5, gamma = 0.95, distance-softmax reference policy of temperature 2.  Inputs are
synthetic and seeded; the root particles are resident in HBM when the timed region starts.

`value` is particle-steps/s over the device-timed steps (CUDA events on the library's
stream: the start event before the plan, the end event right after vopp_plan_submit has
enqueued it, so the interval is the plan on the device; L2 flushed before each step by
writing 256 MB).  `e2e` repeats the
measurement through the same C ABI with host root buffers (host->device copy of the inputs
and device->host copy of the result inside the timed region).  N > 1 runs independent
plans per rank (different seeds; no collective on the data path) and reports the
whole-job aggregate over max-over-ranks time.

`--impl reference` times the FP64 CPU oracle (the only reference this method has) on a
bounded sample of the same workload, on the host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_27191_b300 import workloads as WL  # noqa: E402

METRIC = "particle-steps/s and plans/s at <=1e-4 rel err; p50/p99 plan latency (served vs plain)"
UNIT = "particle-steps/s"

WORKLOADS = {
    "nav1024_d4": WL.CONFIG2,
    "nav256_d3": WL.CONFIG1,
    "grid2048_d5": WL.CONFIG3,
    # smaller grid plan (depth 4) used for kernel profiles
    "grid2048_d4": WL.PlanSpec(kind=WL.GRID, N=2048, D=4, W=3, eta=1.0, gamma=0.95, seed=1,
                               layout_seed=1, root_seed=1),
    # crowd navigation shaped like the paper's CrowdNav (gamma 0.97), wide particle state
    "crowd1024_d4": WL.PlanSpec(kind=WL.CROWD, N=1024, D=4, W=2, eta=1.0, gamma=0.97, seed=1,
                                layout_seed=1, root_seed=1),
}

# Leaf-kernel roofline: issue-bound FP32/INT/SFU arithmetic.  Algorithmic operations per
# particle-step of the fused leaf step, counted operation by operation: NAV2D 83 (Philox 22,
# Box-Muller 14, transition 18, likelihood in linear form 11, heuristic 7, the linear sums
# with their compensation 8.5, loads 2), GRID 18.5 (no Philox; averaged over the 13 actions:
# a sense step 18, a move 19, collect 19), TOY2 16, CROWD 525 (five Philox calls 220, six
# Box-Muller pairs 84, the six people's reactions, moves and tests 180, robot, likelihood,
# heuristic, sums and loads 41); and the issue peak of the B300: 148 SMs x 4 schedulers x
# 32 lanes per clock at the maximum SM clock.
ALG_INSTR_PER_STEP = {WL.NAV2D: 83.0, WL.GRID: 18.5, WL.TOY2: 16.0, WL.CROWD: 525.0}
SMS = 148
LANES_PER_CLK = 128
DATA = "synthetic (seeded root particles; no datasets)"   # both arms' lines


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("vopp_kernels.cu", "vopp_device.cuh"):
        with open(os.path.join(ROOT, "paper_2510_27191_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def leaf_traffic(workload: str):
    """DRAM bytes per leaf launch from the committed ncu capture of this workload, or None
    when there is none or the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", f"k_leaf_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d["dram_bytes_per_launch"] if d.get("source_hash") == kernel_source_hash() else None


# Bytes per particle of a materialised level store: NAV2D x, y, log w; GRID / TOY2 packed
# state, log w; CROWD robot x, y, flags, 12 people coordinates, log w.
STORE_BYTES = {WL.NAV2D: 12, WL.GRID: 8, WL.TOY2: 8, WL.CROWD: 64}


def expand_alg_bytes(spec, level: int) -> int:
    """Algorithmic DRAM bytes of the expansion launch that writes `level`: every child's
    particle store (written), every parent's store (read once), and 12 B of statistics per
    child (mean reward, branch weight, completion counter)."""
    AW = spec.A * spec.W
    per = STORE_BYTES[spec.kind] * spec.N
    return (AW ** level + AW ** (level - 1)) * per + 12 * AW ** level


def expand_traffic(workload: str, level: int):
    """DRAM bytes of that launch from the committed ncu capture, or None when there is none
    or the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", f"k_expand_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash() or d.get("level") != level:
        return None
    return d["dram_bytes_per_launch"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [v.strip() for v in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        finally:
            os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest of every rank's value (the slowest rank's time); the value itself when
    running alone."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n_gpus and world > 1:
        raise SystemExit(f"WORLD_SIZE {world} != --gpus {n_gpus}")
    return rank, world, local


def run_reference(args, spec, rank, world):
    """FP64 oracle on the host cores: each step plans one wave of level-1 subtrees, one per
    host thread (each 1/(A W) of the tree; the ctypes calls release the interpreter lock)."""
    import concurrent.futures as cf
    import oracle as O
    if rank != 0:
        return
    m = O.make_model(spec.kind, pi_mode=spec.pi_mode, pi_temp=spec.pi_temp,
                     rock_x=WL.grid_layout(spec.layout_seed)[0] if spec.kind == WL.GRID else None,
                     rock_y=WL.grid_layout(spec.layout_seed)[1] if spec.kind == WL.GRID else None)
    root = _root_arrays(spec)
    AW = spec.A * spec.W
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = max(1, min(threads or 1, AW))
    steps_per_subtree = sum(AW ** l for l in range(1, spec.D)) * spec.N + spec.N

    def subtree(i):
        kw = dict(root_x=root.get("x"), root_y=root.get("y"), root_s=root.get("s"),
                  root_pf=root.get("pf"))
        r = O.plan(m, spec.N, spec.D, spec.W, spec.eta, spec.gamma, spec.seed, path=(i % AW,),
                   outputs=False, **kw)
        return r["particle_steps"]

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        def sample(i):
            return sum(ex.map(subtree, range(i * threads, (i + 1) * threads)))

        for i in range(args.warmup):
            sample(i)
        t0 = time.perf_counter()
        done = 0
        for i in range(args.steps):
            done += sample(args.warmup + i)
        dt = time.perf_counter() - t0
    value = done / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": DATA, "config": _config(spec, args),
           "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": threads,
                            "sample": f"{threads} level-1 subtrees per step, one per thread "
                                      f"({steps_per_subtree} particle-steps each, 1/{AW} of "
                                      f"the plan)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def _root_arrays(spec):
    if spec.kind == WL.NAV2D:
        x, y, _ = WL.nav_root(spec.N, spec.root_seed)
        return dict(x=x, y=y)
    if spec.kind == WL.CROWD:
        r = WL.crowd_root(spec.N, spec.root_seed)
        return dict(x=r["x"], y=r["y"], s=r["s"], pf=r["pf"])
    s, _ = WL.grid_root(spec.N, spec.root_seed)
    return dict(s=s)


def _host_states(spec, root):
    """The C ABI's root layout of the workload's particles."""
    if spec.kind == WL.NAV2D:
        return np.concatenate([root["x"], root["y"]]).astype(np.float32)
    if spec.kind == WL.CROWD:
        return WL.pack_crowd_states(root)
    return root["s"].astype(np.int32)


def _config(spec, args):
    return {"workload": f"{WL.KIND_NAMES[spec.kind]} N={spec.N} D={spec.D} A={spec.A} W={spec.W} "
                        f"eta={spec.eta} gamma={spec.gamma} pi={'softmax(-dist/2)' if spec.pi_mode == WL.PI_NAV_SOFTMAX_DIST else 'uniform'}",
            "particle_steps_per_plan": spec.steps, "leaves": (spec.A * spec.W) ** spec.D,
            "root_particles": spec.N, "depth": spec.D, "branches": spec.A * spec.W,
            "l2": "flushed before every step (256 MB write)",
            "parallelism": f"replicas{args.gpus if args else 1}"}


def cpu_baseline(spec, budget_s=20.0, gpu=None):
    """The oracle timed as it stands on the host over a bounded sample: level-1 subtrees of
    the same plan (independent, so they spread over the host's cores with one thread per
    core; the ctypes calls release the interpreter lock).  Reports the all-cores rate, with
    the single-thread rate beside it.  The single-thread sample is the whole plan of the
    GPU's last timed seed when it fits half the budget (gpu = (result, seed)); the
    GPU result's error against it is reported as `accuracy`."""
    import concurrent.futures as cf
    import oracle as O
    m = O.make_model(spec.kind, pi_mode=spec.pi_mode, pi_temp=spec.pi_temp,
                     rock_x=WL.grid_layout(spec.layout_seed)[0] if spec.kind == WL.GRID else None,
                     rock_y=WL.grid_layout(spec.layout_seed)[1] if spec.kind == WL.GRID else None)
    root = _root_arrays(spec)
    AW = spec.A * spec.W

    def subtree(n):
        r = O.plan(m, spec.N, spec.D, spec.W, spec.eta, spec.gamma, spec.seed, path=(n % AW,),
                   outputs=False, root_x=root.get("x"), root_y=root.get("y"),
                   root_s=root.get("s"), root_pf=root.get("pf"))
        return r["particle_steps"]

    # single thread: the whole plan of the GPU's last timed seed if it fits half the budget
    # (about 1e7 FP64 particle-steps/s on one core), else subtrees one after another
    accuracy, whole = None, gpu is not None and spec.steps <= 1e7 * budget_s / 2
    t0 = time.perf_counter()
    done1, n1 = 0, 0
    if whole:
        res, seed = gpu
        o = O.plan(m, spec.N, spec.D, spec.W, spec.eta, spec.gamma, seed, outputs=False,
                   root_x=root.get("x"), root_y=root.get("y"), root_s=root.get("s"),
                   root_pf=root.get("pf"))
        done1, n1 = o["particle_steps"], AW
        q_o, q_g = np.asarray(o["q_root"], dtype=np.float64), np.asarray(res["q"], dtype=np.float64)
        rel = lambda g, r: np.abs(g - r) / np.maximum(np.abs(r), 1.0)
        top = np.sort(q_o)[::-1]
        accuracy = {"oracle": f"FP64, seed {seed}, whole plan", "tolerance": 1e-4,
                    "max_err_q_root": float(rel(q_g, q_o).max()),
                    "err_v_root": float(rel(np.float64(res["v_root"]), np.float64(o["v_root"]))),
                    "action": int(res["action"]), "oracle_action": int(o["action"]),
                    "action_match": int(res["action"]) == int(o["action"]),
                    "oracle_top2_q_gap": float(top[0] - top[1]) if len(top) > 1 else None,
                    "near_threshold_particles": int(o["near_threshold"])}
    else:
        while time.perf_counter() - t0 < budget_s / 3 and n1 < AW:
            done1 += subtree(n1)
            n1 += 1
    dt1 = time.perf_counter() - t0
    # all cores: waves of one subtree per thread, every subtree of the plan at least once
    # when the budget allows
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = max(1, threads or 1)
    done, n = 0, 0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        while time.perf_counter() - t0 < budget_s * 2 / 3 and n < max(AW, threads):
            wave = list(range(n, n + threads))
            done += sum(ex.map(subtree, wave))
            n += len(wave)
    dt = time.perf_counter() - t0
    return {"kind": "oracle", "value": done / dt, "unit": UNIT, "cores": threads,
            "single_thread_value": done1 / dt1,
            "sample": f"{n} level-1 subtrees (of {AW}; indices taken modulo {AW}) of the same "
                      f"plan, {done} particle-steps, FP64, {threads} threads, {dt:.1f} s; "
                      f"single thread: " + (f"the whole plan" if whole else f"{n1} subtrees") +
                      f", {done1} particle-steps, {dt1:.1f} s",
            "accuracy": accuracy}


def config_leg(V, ctx, name, steps, warmup=1):
    """One configured workload at full size on this context: event-timed plans (L2 flushed
    before each), then the same plans with per-kernel events for its leaf kernel's roofline."""
    import torch
    spec = WORKLOADS[name]
    rx, ry = WL.grid_layout(spec.layout_seed)
    model = V.vopp_create_model(ctx, V.make_desc(spec.kind, pi_mode=spec.pi_mode,
                                                 pi_temp=spec.pi_temp,
                                                 rock_x=rx if spec.kind == WL.GRID else None,
                                                 rock_y=ry if spec.kind == WL.GRID else None))
    states = torch.from_numpy(_host_states(spec, _root_arrays(spec))).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def run(n):
        ts = []
        for i in range(n):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            V.vopp_plan_submit(model, states, None, spec.N, spec.D, spec.W, spec.eta, spec.gamma,
                               None, spec.seed + i)
            b.record(stream)                 # the plan's device time (see timed_pass)
            V.vopp_plan_finish(ctx)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    run(warmup)
    ts = run(steps)
    V.vopp_ctx_set_timing(ctx, True)
    V.vopp_ctx_reset_kernel_times(ctx)
    run(steps)
    kt = V.vopp_ctx_kernel_times(ctx)
    V.vopp_ctx_set_timing(ctx, False)
    V.vopp_model_destroy(model)
    leaf_ms, leaf_n = kt["leaf"]
    leaf_s = leaf_ms / max(leaf_n, 1) / 1e3
    AW = spec.A * spec.W
    leaf_steps = (AW ** spec.D + (AW ** (spec.D - 1) if spec.D >= 2 else 0)) * spec.N
    pk, pk_src = peaks()
    peak_ops = SMS * LANES_PER_CLK * float(pk.get("sm_max_mhz", 2032.0)) * 1e6
    ms = float(np.median(ts))
    fam_total = sum(v[0] for k, v in kt.items() if not k.startswith("expand_to_"))
    out = {"workload": _config(spec, None)["workload"], "plans": steps,
           "ms_per_plan": ms, "particle_steps": spec.steps,
           "particle_steps_per_s": spec.steps / (ms / 1e3),
           "leaf": {"avg_launch_ms": leaf_s * 1e3, "per_unit": f"{ALG_INSTR_PER_STEP[spec.kind]:g} instr per particle-step",
                    "frac": ALG_INSTR_PER_STEP[spec.kind] * leaf_steps / leaf_s / peak_ops,
                    "share_of_plan": leaf_ms / max(fam_total, 1e-9)}}
    # the deepest materialised level's expansion (K2): HBM-bound, algorithmic bytes = the
    # child particle stores written + the parent stores read + the per-child statistics
    deep = spec.D - 2
    if deep >= 1 and kt.get(f"expand_to_l{deep}", (0.0, 0))[1]:
        ems, en = kt[f"expand_to_l{deep}"]
        e_s = ems / en / 1e3
        nbytes = expand_alg_bytes(spec, deep)
        out["expand"] = {"kernel": "k_expand", "level": deep, "bound": "hbm",
                         "avg_launch_ms": e_s * 1e3, "alg_bytes_per_launch": nbytes,
                         "achieved": nbytes / e_s / 1e9, "peak": float(pk["hbm_gbs"]),
                         "unit": "GB/s", "frac": nbytes / e_s / 1e9 / float(pk["hbm_gbs"]),
                         "peak_source": f"{pk_src} STREAM-style copy",
                         "traffic": expand_traffic(name, deep),
                         "share_of_plan": ems / max(fam_total, 1e-9)}
    return out


def modes_run(V, ctx, spec, dev_states):
    """The other planning modes on the same device: anytime deepening of the workload's plan
    (to its depth, and under 2 ms and 50 ms budgets), episode mode at 60,000 parallel
    episodes (the paper's largest batch) on both models, and one closed-loop grid episode."""
    import torch
    out = {}
    rx, ry = WL.grid_layout(spec.layout_seed)
    model = V.vopp_create_model(ctx, V.make_desc(spec.kind, pi_mode=spec.pi_mode,
                                                 pi_temp=spec.pi_temp,
                                                 rock_x=rx if spec.kind == WL.GRID else None,
                                                 rock_y=ry if spec.kind == WL.GRID else None))

    def timed(fn, reps=3):
        fn()
        ts, r = [], None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts)), r

    t, r = timed(lambda: V.vopp_plan_anytime(model, dev_states, None, spec.N, spec.D, spec.W,
                                             spec.eta, spec.gamma, spec.seed))
    out["anytime"] = {"max_depth": spec.D, "depth_reached": r["depth_reached"], "ms": 1e3 * t,
                      "particle_steps": r["particle_steps"],
                      "particle_steps_per_s": r["particle_steps"] / t}
    for budget in (0.002, 0.05):   # the next iteration starts while under budget (Alg. 1)
        t, r = timed(lambda: V.vopp_plan_anytime(model, dev_states, None, spec.N, spec.D + 2,
                                                 spec.W, spec.eta, spec.gamma, spec.seed,
                                                 budget_s=budget))
        out[f"anytime_budget_{int(budget * 1e3)}ms"] = {
            "max_depth": spec.D + 2, "depth_reached": r["depth_reached"], "ms": 1e3 * t,
            "particle_steps": r["particle_steps"]}
    V.vopp_model_destroy(model)
    eps = {}
    rx, ry = WL.grid_layout(1)
    for name, kind in (("grid", WL.GRID), ("nav", WL.NAV2D)):
        m = V.vopp_create_model(ctx, V.make_desc(kind, rock_x=rx if kind == WL.GRID else None,
                                                 rock_y=ry if kind == WL.GRID else None))
        if kind == WL.GRID:
            st, _ = WL.grid_root(2048, 1)
            st = torch.from_numpy(st.astype(np.int32)).cuda()
        else:
            x, y, _ = WL.nav_root(2048, 1)
            st = torch.from_numpy(np.concatenate([x, y]).astype(np.float32)).cuda()
        t, r = timed(lambda: V.vopp_plan_episodes(m, st, None, 2048, 60000, 6, 1.0, 0.95, 5))
        eps[name] = {"episodes": 60000, "depth_reached": r["depth_reached"], "ms": 1e3 * t,
                     "nodes": r["n_nodes"], "model_steps": r["particle_steps"],
                     "model_steps_per_s": r["particle_steps"] / t}
        V.vopp_model_destroy(m)
    out["episodes"] = eps
    cs = WORKLOADS["crowd1024_d4"]
    mc = V.vopp_create_model(ctx, V.make_desc(WL.CROWD))
    cst = torch.from_numpy(_host_states(cs, _root_arrays(cs))).cuda()
    t, r = timed(lambda: V.vopp_plan(mc, cst, None, cs.N, cs.D, cs.W, cs.eta, cs.gamma, None, cs.seed))
    out["crowd1024_d4"] = {"ms": 1e3 * t, "particle_steps": r["particle_steps"],
                           "particle_steps_per_s": r["particle_steps"] / t,
                           "state_bytes_per_particle": 60}
    V.vopp_model_destroy(mc)
    m = V.vopp_create_model(ctx, V.make_desc(WL.GRID, rock_x=rx, rock_y=ry))
    st, _ = WL.grid_root(1024, 2)
    g = V.vopp_agent_create(m, st.astype(np.int32), None, 1024, 2)
    env = V.vopp_env_create(m, int(WL.pack_grid_state(np.array([0b10110101]), *WL.GRID_START)[0]),
                            9, WL.GRID)
    t0 = time.perf_counter()
    ep, acts, rews = V.vopp_run_episode(g, env, 4, 3, 1.0, 0.95, 100, 60)
    dt = time.perf_counter() - t0
    out["closed_loop_grid"] = {"steps": ep["steps"], "terminated": ep["terminated"],
                               "discounted_return": ep["discounted_return"],
                               "plan_depth": 4, "particles": 1024, "wall_s": dt,
                               "plan_s": ep["plan_seconds"], "status": ep["status"]}
    V.vopp_env_destroy(env)
    V.vopp_agent_destroy(g)
    V.vopp_model_destroy(m)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="vopp", choices=["vopp", "reference"])
    ap.add_argument("--workload", default="nav1024_d4", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-serve", action="store_true",
                    help="skip the batched (512 mixed plans), served (Poisson requests) and "
                         "other-mode (anytime, episodes, closed loop) legs")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served and plain legs at the serving workload's rate "
                         "(2,000 requests/s; 60 s as the workload specifies)")
    ap.add_argument("--overload-seconds", type=float, default=4.0,
                    help="length of the legs at 16,000 requests/s (overload)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every plan's kernels one by one instead of replaying the "
                         "captured CUDA graph of the plan's shape")
    args = ap.parse_args()
    spec = WORKLOADS[args.workload]
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, spec, rank, world)
        return

    import torch
    from paper_2510_27191_b300 import vopp as V
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    ctx = V.vopp_ctx_create(local, 0, stream.cuda_stream)
    # plans of one shape replay one captured CUDA graph (metadata upload, every kernel, result
    # copy): the per-plan host work is a memcpy into pinned memory and one graph launch
    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, 0 if args.no_graphs else 1)
    model = V.vopp_create_model(ctx, V.make_desc(spec.kind, pi_mode=spec.pi_mode,
                                                 pi_temp=spec.pi_temp,
                                                 rock_x=WL.grid_layout(spec.layout_seed)[0] if spec.kind == WL.GRID else None,
                                                 rock_y=WL.grid_layout(spec.layout_seed)[1] if spec.kind == WL.GRID else None))
    root = _root_arrays(spec)
    host_states = _host_states(spec, root)
    dev_states = torch.from_numpy(host_states).cuda()
    pinned = torch.from_numpy(host_states).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    seeds = [spec.seed + 1000 * rank + i for i in range(args.warmup + args.steps)]

    def plan(states, seed):
        return V.vopp_plan(model, states, None, spec.N, spec.D, spec.W, spec.eta, spec.gamma,
                           None, seed)

    def timed_pass(states, n_steps, seed0, device_timed=False):
        """device_timed: the end event is recorded as soon as the plan is enqueued
        (vopp_plan_submit), so the time is the plan's on the device; otherwise after the
        synchronous vopp_plan returns (its stream synchronisation and result collection on
        the host included, as a caller of vopp_plan sees it)."""
        times, res = [], None
        for i in range(n_steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            seed = seeds[(seed0 + i) % len(seeds)]
            a.record(stream)
            if device_timed:
                V.vopp_plan_submit(model, states, None, spec.N, spec.D, spec.W, spec.eta,
                                   spec.gamma, None, seed)
                b.record(stream)
                res = V.vopp_plan_finish(ctx)
            else:
                res = plan(states, seed)
                b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        return times, res

    for i in range(args.warmup):
        plan(dev_states, seeds[i])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    V.vopp_ctx_reset_kernel_times(ctx)
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        times, last = timed_pass(dev_states, args.steps, args.warmup, device_timed=True)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    counters = V.vopp_ctx_counters(ctx)
    total_ms = max_over_ranks(float(sum(times)), dist, "cuda")
    units = spec.steps * args.steps * world
    value = weak_scaling_rate(spec.steps * args.steps, world, total_ms)
    lat = np.array(times)

    # roofline of the dominant kernel (the fused leaf expansion), per-kernel events
    V.vopp_ctx_set_timing(ctx, True)
    V.vopp_ctx_reset_kernel_times(ctx)
    timed_pass(dev_states, args.steps, args.warmup)
    kt = V.vopp_ctx_kernel_times(ctx)
    V.vopp_ctx_set_timing(ctx, False)
    leaf_ms, leaf_n = kt["leaf"]
    leaf_avg_s = leaf_ms / max(leaf_n, 1) / 1e3
    AW = spec.A * spec.W
    leaf_steps = (AW ** spec.D + (AW ** (spec.D - 1) if spec.D >= 2 else 0)) * spec.N
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2032.0))
    peak_ops = SMS * LANES_PER_CLK * sm_max * 1e6
    achieved_ops = ALG_INSTR_PER_STEP[spec.kind] * leaf_steps / leaf_avg_s
    total_kernel_ms = sum(v[0] for k, v in kt.items() if not k.startswith("expand_to_"))

    # end to end through the C ABI with host buffers
    V.vopp_ctx_reset_kernel_times(ctx)
    e2e_times, _ = timed_pass(pinned.numpy(), args.steps, args.warmup)
    c2 = V.vopp_ctx_counters(ctx)
    e2e_ms = max_over_ranks(float(sum(e2e_times)), dist, "cuda")

    # the other legs mix plan shapes: one captured graph per context would be re-captured at
    # every shape change, so they launch stage by stage
    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, 0)

    # issue rates of the leaf kernel's arithmetic, per SM cycle (outside every timed region)
    pipes = V.vopp_pipe_rates(local)
    fma_per_clk = pipes.get("fma.rn.f32", (LANES_PER_CLK, 0.0))[0]

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": DATA,
            "config": _config(spec, args),
            "plans_per_s": args.steps * world / (total_ms / 1e3),
            "nodes_per_s": (sum(AW ** l for l in range(spec.D + 1))) * args.steps * world / (total_ms / 1e3),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean())},
            "wall_s": t_wall,
            "gpu_launches": int(counters["launches"]),
            "e2e": {"value": units / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(c2["h2d_bytes"] // max(args.steps, 1)),
                    "d2h_bytes_per_step": int(c2["d2h_bytes"] // max(args.steps, 1))},
            "roofline": {"kernel": "k_leaf", "bound": "alu", "achieved": achieved_ops / 1e12,
                         "peak": peak_ops / 1e12, "unit": "Tinstr/s",
                         "frac": achieved_ops / peak_ops, "traffic": leaf_traffic(args.workload),
                         "traffic_unit": "DRAM bytes per launch (ncu capture, profiles/)",
                         "peak_source": f"148 SMs x 128 lanes/clk x {sm_max:.0f} MHz ({pk_src} max clock)",
                         "per_unit": f"{ALG_INSTR_PER_STEP[spec.kind]:g} instr per particle-step",
                         "units_per_launch": leaf_steps, "avg_launch_ms": leaf_avg_s * 1e3,
                         "share_of_step": leaf_ms / max(total_kernel_ms, 1e-9),
                         "frac_of_measured_fp32_issue":
                             achieved_ops / (SMS * fma_per_clk * sm_max * 1e6)},
            "pipe_rates": {"unit": "thread ops per SM cycle (microbenchmark, clock64)",
                           **{k: round(v[0], 3) for k, v in pipes.items()}},
            "kernels_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in kt.items() if v[1]},
            "clocks": clk.summary(),
            "result": {"action": int(last["action"]), "v_root": last["v_root"]},
        }
        if not args.no_batch_serve:
            from paper_2510_27191_b300 import loadgen as LG
            out["batched"] = LG.batch_run(V, ctx)
            out["batched_small"] = LG.small_batch_run(V, ctx)
            served = {}
            # served: continuous batching, batched belief updates, agents with subtree reuse
            # (the workload as specified); served_noreuse: the same without kept trees; plain:
            # one synchronous plan per request, then its own belief update
            legs = [(2000.0, "served", True), (2000.0, "plain", False),
                    (2000.0, "served_noreuse", False), (16000.0, "served", True),
                    (16000.0, "plain", False)]
            for rate, name, reuse in legs:
                mode = "plain" if name == "plain" else "served"
                secs = args.serve_seconds if rate == 2000.0 else args.overload_seconds
                r = LG.serve_run(V, ctx, seconds=secs, rate=rate, mode=mode,
                                 drain_factor=2.0, reuse=reuse)
                served[f"{name}_{int(rate)}"] = {k: r[k] for k in (
                    "plans_per_s", "particle_steps_per_s", "p50_ms", "p99_ms",
                    "deadline_misses", "completed", "requests", "unfinished",
                    "subtree_reuse", "reused_plans", "seconds", "hbm_budget_bytes")}
                if mode == "served":
                    served[f"{name}_{int(rate)}"]["mean_batch"] = r.get("mean_batch")
            out["served"] = served
        if not args.no_batch_serve:
            out["modes"] = modes_run(V, ctx, spec, dev_states)
            # the other single-plan configurations at full size (C1, C3)
            out["configs"] = {"nav256_d3": config_leg(V, ctx, "nav256_d3", 20, 3),
                              "grid2048_d5": config_leg(V, ctx, "grid2048_d5", 3, 1)}
            if "expand" in out["configs"]["grid2048_d5"]:
                # the materialising kernel's HBM roofline, on the workload that writes the
                # most (GridSense N=2048 D=5: level 3 is 0.97 GB)
                out["roofline_expand"] = {"workload": "grid2048_d5",
                                          **out["configs"]["grid2048_d5"]["expand"]}
        if not args.no_cpu_baseline and world == 1:
            last_seed = seeds[(args.warmup + args.steps - 1) % len(seeds)]
            out["cpu_baseline"] = cpu_baseline(spec, gpu=(last, last_seed))
        print(json.dumps(out))
    V.vopp_model_destroy(model)
    V.vopp_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
