"""Workload drivers for the batched and served planning paths (used by bench.py and tests).

batch_run: one batch of mixed plans through vopp_plan_batch against the same plans run one
           at a time through vopp_plan (the plain path).
serve_run: Poisson plan requests from device-resident agents against the serving loop
           (continuous batching) or the plain path, with a belief update after every plan.

Only argument marshalling and timing happen here; every plan runs in libvopp's kernels.
"""
from __future__ import annotations

import gc
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
              autotune: bool = True, graphs: bool = True):
    """Returns a dict with the batched and sequential times (CUDA events around each).
    graphs: the batch replays its recorded launch sequence (the sequential plans always
    launch stage by stage); the context's graph option is left off.  autotune: both times use
    the leaf CTA size and scheduling the tuner picks for this batch; the context's defaults
    (128 threads, per-model scheduling) are put back afterwards, so that later single plans
    on the context do not inherit a choice made for the mixed batch."""
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
    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, int(graphs))
    V.vopp_plan_batch(ctx, reqs)              # warm-up (and the recorded sequence)
    t_batch = []
    for _ in range(reps):
        t, (outs, keep) = timed(lambda: V.vopp_plan_batch(ctx, reqs))
        t_batch.append(t)
    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, 0)
    res = {"plans": n_plans, "particle_steps": steps, "batched_s": min(t_batch),
           "autotune": tune, "graphs": bool(graphs),
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
    if autotune:
        V.vopp_ctx_set_option(ctx, V.VOPP_OPT_LEAF_THREADS, 128)
        V.vopp_ctx_set_option(ctx, V.VOPP_OPT_PERSISTENT, 2)
    return res


def small_batch_run(V, ctx, n_plans: int = 512, reps: int = 3, graphs: bool = True):
    """n_plans small navigation plans (N=256, depth 3, 4x4 branches: the latency-bound shape)
    with different seeds and roots, one batch against one plan at a time (CUDA events); the
    batch replays its recorded launch sequence when graphs is set."""
    import torch
    model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D))
    ps = WL.CONFIG1
    roots = []
    for i in range(n_plans):
        x, y, _ = WL.nav_root(ps.N, 100 + i)
        roots.append(torch.from_numpy(np.concatenate([x, y]).astype(np.float32)).cuda())
    reqs = [dict(model=model, states=r, weights=None, n=ps.N, depth=ps.D, width=ps.W,
                 eta=ps.eta, gamma=ps.gamma, seed=1000 + i, A=4) for i, r in enumerate(roots)]
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3, out

    def seq():
        return [V.vopp_plan(q["model"], q["states"], None, q["n"], q["depth"], q["width"],
                            q["eta"], q["gamma"], None, q["seed"]) for q in reqs]

    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, int(graphs))
    V.vopp_plan_batch(ctx, reqs)              # warm-up (and the recorded sequence)
    t_b = min(timed(lambda: V.vopp_plan_batch(ctx, reqs))[0] for _ in range(reps))
    outs, _ = V.vopp_plan_batch(ctx, reqs)
    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, 0)
    seq()
    t_s, singles = min((timed(seq) for _ in range(reps)), key=lambda r: r[0])
    same = all(a["q"].tolist() == b["q"].tolist() for a, b in zip(outs, singles))
    V.vopp_model_destroy(model)
    steps = float(ps.steps) * n_plans
    return {"plans": n_plans, "workload": "nav2d N=256 D=3 A=4 W=4 (different roots and seeds)",
            "batched_s": t_b, "sequential_s": t_s, "speedup": t_s / t_b,
            "batched_plans_per_s": n_plans / t_b, "sequential_plans_per_s": n_plans / t_s,
            "batched_particle_steps_per_s": steps / t_b, "batched_equals_sequential": bool(same),
            "graphs": bool(graphs)}


SERVE_HBM_BUDGET = 120 * (1 << 30)   # the serving workload's admission budget: 120 GB


def serve_run(V, ctx, seconds: float = 5.0, rate: float = 2000.0, n_agents: int = 1024,
              seed: int = 11, mode: str = "served", deadline_s: float = 0.05, max_batch: int = 64,
              n_slots: int = 3, drain_factor: float = 3.0, reuse: bool = False,
              hbm_budget_bytes: int = SERVE_HBM_BUDGET, graphs: bool = True):
    """Poisson arrivals at `rate` per second over `n_agents` agents for `seconds`; each
    agent's requests are served in order, a belief update follows every completed plan.
    Served mode updates the agents of all plans that finished together in one batched call
    and admits batches by the HBM budget; reuse: agents keep their trees (subtree reuse);
    graphs: the server replays the recorded launch sequences of batch shapes it has seen (it
    reads the context's graph option when it is created; the option is left off)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x73657276]))
    specs = WL.draw_mixed_plans(n_agents, seed, WL.SERVE_CAP_STEPS)
    models = make_models(V, ctx)

    def new_agent(i, salt=0):
        ps = specs[i]
        g = V.vopp_agent_create(models[ps.kind], _root(ps), None, ps.N, 1000003 * (i + 1) + salt)
        if reuse:
            V.vopp_agent_set_reuse(g, True)
        return g

    agents = [new_agent(i) for i in range(n_agents)]
    reused = 0
    n_req = rng.poisson(rate * seconds)
    arrivals = np.sort(rng.uniform(0.0, seconds, n_req))
    who = [int(v) for v in rng.integers(0, n_agents, n_req)]
    queues = [[] for _ in range(n_agents)]
    busy = np.zeros(n_agents, dtype=bool)
    lat, steps_done, updates = [], 0, 0
    plan_count = np.zeros(n_agents, dtype=np.int64)
    srv = None
    if mode == "served":
        V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, int(graphs))
        srv = V.vopp_server_create(ctx, max_batch, n_slots, hbm_budget_bytes)
        V.vopp_ctx_set_option(ctx, V.VOPP_OPT_GRAPHS, 0)
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
        agents[i] = new_agent(i, 17 * resets)
        resets += 1

    def issue(i):
        ps = specs[i]
        plan_count[i] += 1
        seed_i = (i + 1) * 7919 + int(plan_count[i])
        return V.vopp_submit_agent(srv, agents[i], ps.D, ps.W, ps.eta, ps.gamma, seed_i)

    # the timed loop runs with Python's cyclic garbage collector off (its pauses would show
    # up as request latency); reference counting still frees everything the loop drops
    gc_was_on = gc.isenabled()
    gc.disable()
    t0 = time.perf_counter()
    k = 0
    if mode == "served":
        # event-driven: a request is submitted the moment it arrives (or, if its agent has a
        # plan in flight, the moment that plan's belief update is done); between events the
        # loop polls for completions and arrivals
        def finish(done):
            """Completed plans: latencies, one batched belief update, next requests."""
            nonlocal updates, reused
            upd, freed = [], []
            for t, rc, res in done:
                if rc not in (V.VOPP_OK, V.VOPP_E_DEGENERATE):
                    V.check(rc)
                i, arr = inflight.pop(t)
                freed.append(i)
                lat.append(time.perf_counter() - t0 - arr)
                if res is None:
                    reset(i)
                else:
                    nonlocal_steps[0] += res["particle_steps"]
                    reused += bool(res["flags"] & V.VOPP_FLAG_REUSED)
                    a = max(int(res["action"]), 0)
                    upd.append((i, a, obs_for(specs[i], a)))
            if upd:
                st, _, _ = V.vopp_belief_update_batch(
                    ctx, [agents[i] for i, _, _ in upd], [a for _, a, _ in upd],
                    [o for _, _, o in upd], [specs[i].kind for i, _, _ in upd])
                updates += int(np.sum(st == V.VOPP_OK))   # impossible observation: unchanged
            for i in freed:
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
            # wait for a completion until the next arrival is due: the library spins for such
            # short waits, so a completion or an arrival is picked up within a microsecond
            # (a sleeping wait would add a thread wake-up to every request)
            if inflight:
                # (the clock read again: the submissions above take time)
                wait = (arrivals[k] - (time.perf_counter() - t0)) if k < n_req else 1e-3
                got = V.vopp_wait_any(srv, min(max(wait, 0.0), 1e-3))
            else:
                got = None
            if got is None:
                if not inflight and k < n_req:
                    while time.perf_counter() - t0 < arrivals[k]:
                        pass                           # idle until the next arrival
                continue
            done = [got[:3]]
            while len(done) < len(inflight):           # everything else already finished
                got = V.vopp_wait_any(srv, 0.0)
                if got is None:
                    break
                done.append(got[:3])
            finish(done)
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
                reused += bool(res["flags"] & V.VOPP_FLAG_REUSED)
                after_plan(i, res)
            if time.perf_counter() - t0 > seconds * drain_factor:
                break                                  # overloaded: stop draining
    wall = time.perf_counter() - t0
    if gc_was_on:
        gc.enable()
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
           "reused_plans": int(reused), "subtree_reuse": bool(reuse),
           "episodes_restarted": resets,
           "offered_rate": rate, "agents": n_agents, "seconds": seconds,
           "hbm_budget_bytes": int(hbm_budget_bytes) if mode == "served" else None,
           "graphs": bool(graphs) if mode == "served" else False}
    if stats:
        out["batches"] = int(stats["batches"])
        out["mean_batch"] = stats["batched_plans"] / max(stats["batches"], 1)
        out["peak_in_flight_bytes"] = int(stats["peak_in_flight_bytes"])
    return out
