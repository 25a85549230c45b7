"""Workload drivers for the batched and served planning paths (used by bench.py and tests).

batch_run: one batch of mixed plans through vopp_plan_batch against the same plans run one
           at a time through vopp_plan (the plain path).
serve_run: Poisson plan requests from device-resident agents against the serving loop
           (continuous batching) or the plain path, with a belief update after every plan.

Only argument marshalling and timing happen here; every plan runs in libvopp's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as WL


def _root(ps: WL.PlanSpec):
    if ps.kind == WL.NAV2D:
        x, y, _ = WL.nav_root(ps.N, ps.root_seed)
        return np.concatenate([x, y]).astype(np.float32)
    s, _ = WL.grid_root(ps.N, ps.root_seed)
    return np.asarray(s, dtype=np.int32)


def make_models(V, ctx, layout_seed: int = 1):
    rx, ry = WL.grid_layout(layout_seed)
    return {WL.NAV2D: V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D)),
            WL.GRID: V.vopp_create_model(ctx, V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry))}


def batch_run(V, ctx, n_plans: int = 512, seed: int = 7, reps: int = 2, sequential: bool = True,
              autotune: bool = True):
    """Returns a dict with the batched and sequential times (CUDA events around each)."""
    import torch
    specs = WL.draw_mixed_plans(n_plans, seed)
    models = make_models(V, ctx)
    roots = [torch.from_numpy(_root(ps)).cuda() for ps in specs]
    reqs = [dict(model=models[ps.kind], states=r, weights=None, n=ps.N, depth=ps.D, width=ps.W,
                 eta=ps.eta, gamma=ps.gamma, seed=ps.seed, A=ps.A) for ps, r in zip(specs, roots)]
    steps = float(sum(ps.steps for ps in specs))
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3, out

    tune = V.vopp_autotune(ctx, reqs[::8], reps=1) if autotune else None   # tiles from the tuner
    V.vopp_plan_batch(ctx, reqs[:8])          # warm-up
    t_batch = []
    for _ in range(reps):
        t, (outs, keep) = timed(lambda: V.vopp_plan_batch(ctx, reqs))
        t_batch.append(t)
    res = {"plans": n_plans, "particle_steps": steps, "batched_s": min(t_batch),
           "autotune": tune,
           "batched_particle_steps_per_s": steps / min(t_batch),
           "batched_plans_per_s": n_plans / min(t_batch)}
    if sequential:
        def seq():
            return [V.vopp_plan(q["model"], q["states"], None, q["n"], q["depth"], q["width"],
                                q["eta"], q["gamma"], None, q["seed"]) for q in reqs]
        t_seq, singles = timed(seq)
        same = all(a["q"].tolist() == b["q"].tolist() for a, b in zip(outs, singles))
        res.update({"sequential_s": t_seq, "sequential_particle_steps_per_s": steps / t_seq,
                    "sequential_plans_per_s": n_plans / t_seq, "speedup": t_seq / min(t_batch),
                    "batched_equals_sequential": bool(same)})
    for m in models.values():
        V.vopp_model_destroy(m)
    return res


def serve_run(V, ctx, seconds: float = 5.0, rate: float = 2000.0, n_agents: int = 1024,
              seed: int = 11, mode: str = "served", deadline_s: float = 0.05, max_batch: int = 64,
              n_slots: int = 3, drain_factor: float = 3.0):
    """Poisson arrivals at `rate` per second over `n_agents` agents for `seconds`; each
    agent's requests are served in order, a belief update follows every completed plan."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x73657276]))
    specs = WL.draw_mixed_plans(n_agents, seed, WL.SERVE_CAP_STEPS)
    models = make_models(V, ctx)
    agents = [V.vopp_agent_create(models[ps.kind], _root(ps), None, ps.N, 1000003 * (i + 1))
              for i, ps in enumerate(specs)]
    n_req = rng.poisson(rate * seconds)
    arrivals = np.sort(rng.uniform(0.0, seconds, n_req))
    who = [int(v) for v in rng.integers(0, n_agents, n_req)]
    queues = [[] for _ in range(n_agents)]
    busy = np.zeros(n_agents, dtype=bool)
    lat, steps_done, updates = [], 0, 0
    plan_count = np.zeros(n_agents, dtype=np.int64)
    srv = V.vopp_server_create(ctx, max_batch, n_slots) if mode == "served" else None
    inflight = {}          # ticket -> (agent, arrival)

    def obs_for(ps, action):
        if ps.kind == WL.NAV2D:
            return (float(rng.uniform(2, 8)), float(rng.uniform(2, 8)))
        return 0 if action < 5 else int(rng.integers(1, 3))

    def after_plan(i, res):
        nonlocal updates
        ps = specs[i]
        a = max(int(res["action"]), 0)
        try:
            V.vopp_belief_update(agents[i], a, obs_for(ps, a), ps.kind)
            updates += 1
        except V.VoppError:
            pass                      # impossible observation: belief left unchanged

    resets = 0

    def reset(i):
        # every particle of agent i is terminal: its episode is over, start a new one
        nonlocal resets
        ps = specs[i]
        V.vopp_agent_destroy(agents[i])
        agents[i] = V.vopp_agent_create(models[ps.kind], _root(ps), None, ps.N,
                                        1000003 * (i + 1) + 17 * resets)
        resets += 1

    def issue(i):
        ps = specs[i]
        plan_count[i] += 1
        seed_i = (i + 1) * 7919 + int(plan_count[i])
        return V.vopp_submit_agent(srv, agents[i], ps.D, ps.W, ps.eta, ps.gamma, seed_i)

    t0 = time.perf_counter()
    k = 0
    if mode == "served":
        # event-driven: a request is submitted the moment it arrives (or, if its agent has a
        # plan in flight, the moment that plan's belief update is done); between events the
        # loop polls for completions and arrivals
        def finish(t, rc, res):
            if rc not in (V.VOPP_OK, V.VOPP_E_DEGENERATE):
                V.check(rc)
            i, arr = inflight.pop(t)
            lat.append(time.perf_counter() - t0 - arr)
            nonlocal_steps[0] += res["particle_steps"] if res is not None else 0
            if res is None:
                reset(i)
            else:
                after_plan(i, res)
            busy[i] = False
            if queues[i]:
                inflight[issue(i)] = (i, queues[i].pop(0))
                busy[i] = True

        nonlocal_steps = [0]
        while True:
            now = time.perf_counter() - t0
            while k < n_req and arrivals[k] <= now:
                i = who[k]
                if busy[i]:
                    queues[i].append(arrivals[k])
                else:
                    inflight[issue(i)] = (i, arrivals[k])
                    busy[i] = True
                k += 1
            if k >= n_req and not inflight:
                break
            if now > seconds * drain_factor:
                break                                  # overloaded: stop draining
            # poll: a completion or an arrival is picked up within microseconds (a blocking
            # wait would add a thread wake-up to every request)
            got = V.vopp_wait_any(srv, 0.0) if inflight else None
            if got is None:
                if not inflight and k < n_req:
                    while time.perf_counter() - t0 < arrivals[k]:
                        pass                           # idle until the next arrival
                continue
            finish(got[0], got[1], got[2])
            while inflight:                            # everything else already finished
                got = V.vopp_wait_any(srv, 0.0)
                if got is None:
                    break
                finish(got[0], got[1], got[2])
        steps_done = nonlocal_steps[0]
    else:
        # plain path: requests run alone, synchronously, in arrival order (an agent's earlier
        # request has always finished, with its belief update, before its next one starts)
        while k < n_req:
            while time.perf_counter() - t0 < arrivals[k]:
                pass                                   # idle until the next arrival
            i, arr = who[k], arrivals[k]
            k += 1
            ps = specs[i]
            plan_count[i] += 1
            try:
                res = V.vopp_agent_plan(agents[i], models[ps.kind], ps.D, ps.W, ps.eta,
                                        ps.gamma, (i + 1) * 7919 + int(plan_count[i]))
            except V.VoppError as e:
                if e.code != V.VOPP_E_DEGENERATE:
                    raise
                res = None
            lat.append(time.perf_counter() - t0 - arr)
            if res is None:
                reset(i)
            else:
                steps_done += res["particle_steps"]
                after_plan(i, res)
            if time.perf_counter() - t0 > seconds * drain_factor:
                break                                  # overloaded: stop draining
    wall = time.perf_counter() - t0
    stats = V.vopp_server_get_stats(srv) if srv else {}
    if srv:
        V.vopp_server_destroy(srv)
    for g in agents:
        V.vopp_agent_destroy(g)
    for m in models.values():
        V.vopp_model_destroy(m)
    lat = np.array(lat)
    out = {"mode": mode, "requests": int(n_req), "completed": int(len(lat)), "wall_s": wall,
           "unfinished": int(n_req - len(lat)),
           "plans_per_s": len(lat) / wall, "particle_steps_per_s": steps_done / wall,
           "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
           "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
           "deadline_misses": int(np.sum(lat > deadline_s)), "belief_updates": updates,
           "episodes_restarted": resets,
           "offered_rate": rate, "agents": n_agents, "seconds": seconds}
    if stats:
        out["batches"] = int(stats["batches"])
        out["mean_batch"] = stats["batched_plans"] / max(stats["batches"], 1)
        out["peak_in_flight_bytes"] = int(stats["peak_in_flight_bytes"])
    return out
