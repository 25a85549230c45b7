"""Serving loop (continuous batching) on the GPU: results alone vs in the mix, admission by
the HBM budget, overlap of batches (needs a GPU)."""
import dataclasses
import time

import numpy as np
import pytest

from paper_2510_27191_b300 import workloads as WL
import oracle as O
from tests.parity import Spec, action_agrees, assert_close

pytestmark = pytest.mark.gpu


def _models(V, ctx):
    rx, ry = WL.grid_layout(1)
    return {WL.NAV2D: V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D)),
            WL.GRID: V.vopp_create_model(ctx, V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry))}


def test_served_results_equal_alone_results():
    """Every plan's result is bit-identical whether it ran alone (vopp_plan) or inside a
    batch of the serving loop, for requests from agents and from raw root particles."""
    import torch
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    models = _models(V, ctx)
    srv = V.vopp_server_create(ctx, max_batch=16, n_slots=2)
    try:
        specs = WL.draw_mixed_plans(48, 11, 1 << 22)
        agents, tickets, inputs = [], [], []
        V.vopp_server_set_paused(srv, True)      # queue the whole burst, then release it
        for i, ps in enumerate(specs):
            sp = Spec.from_plan(ps)
            st = sp.states()
            if i % 2 == 0:
                g = V.vopp_agent_create(models[ps.kind], st, None, ps.N, 1234 + i)
                agents.append(g)
                t = V.vopp_submit_agent(srv, g, ps.D, ps.W, ps.eta, ps.gamma, ps.seed)
            else:
                t = V.vopp_submit(srv, models[ps.kind], st, None, ps.N, ps.D, ps.W, ps.eta,
                                  ps.gamma, ps.seed)
            tickets.append(t)
            inputs.append((ps, st))
        V.vopp_server_set_paused(srv, False)
        served = [V.vopp_wait(srv, t, {WL.NAV2D: 4, WL.GRID: 13}[ps.kind], 20.0)
                  for t, (ps, _) in zip(tickets, inputs)]
        stats = V.vopp_server_get_stats(srv)
        assert stats["completed"] == 48 and stats["rejected"] == 0
        assert stats["batches"] <= 4 and stats["max_batch_seen"] == 16   # batches of <= 16
        for (res, lat), (ps, st) in zip(served, inputs):
            alone = V.vopp_plan(models[ps.kind], st, None, ps.N, ps.D, ps.W, ps.eta, ps.gamma,
                                None, ps.seed)
            assert res["q"].tolist() == alone["q"].tolist()
            assert res["action"] == alone["action"] and res["v_root"] == alone["v_root"]
            assert lat > 0
        for g in agents:
            V.vopp_agent_destroy(g)
    finally:
        V.vopp_server_destroy(srv)
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)


def test_admission_refuses_plans_beyond_the_budget():
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    models = _models(V, ctx)
    srv = V.vopp_server_create(ctx, max_batch=8, n_slots=2, hbm_budget_bytes=4 << 20)
    try:
        x, y, _ = WL.nav_root(1024, 1)
        st = np.concatenate([x, y]).astype(np.float32)
        big = V.vopp_submit(srv, models[WL.NAV2D], st, None, 1024, 5, 4, 1.0, 0.95, 1)
        small = [V.vopp_submit(srv, models[WL.NAV2D], np.concatenate([x[:64], y[:64]]), None,
                               64, 2, 2, 1.0, 0.95, s)
                 for s in range(6)]
        with pytest.raises(V.VoppError) as e:
            V.vopp_wait(srv, big, 4, 20.0)
        assert e.value.code == V.VOPP_E_BUDGET
        for t in small:
            res, _ = V.vopp_wait(srv, t, 4, 20.0)
            assert res["action"] >= 0
        st_ = V.vopp_server_get_stats(srv)
        assert st_["rejected"] == 1 and st_["peak_in_flight_bytes"] <= 4 << 20
        with pytest.raises(V.VoppError) as e:
            V.vopp_wait(srv, 10**9, 4, 0.05)
        assert e.value.code == V.VOPP_E_TIMEOUT
    finally:
        V.vopp_server_destroy(srv)
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)


def _observation(kind, action, st, lw):
    """An observation the agent's own belief makes possible: from its heaviest particle (moved
    by the action's mean displacement for the navigation model; the sensed rock's bit for the
    grid model, NULL for moves and collect)."""
    i = int(np.argmax(lw))
    if kind == WL.NAV2D:
        n = lw.size
        d = [(1, 0), (-1, 0), (0, 1), (0, -1)][action]
        return (float(np.clip(st[i] + d[0], 0, 10)), float(np.clip(st[n + i] + d[1], 0, 10)))
    if action >= 5:
        return 1 if (int(st[i]) >> (action - 5)) & 1 else 2
    return 0


def _replay(kind, st, lw, N, D, W, eta, gamma, seed, res, what):
    """Run the oracle on the particles a request carried and compare the served result."""
    w = np.exp(lw.astype(np.float64) - float(np.max(lw)))
    n = lw.size
    root = (dict(x=st[:n], y=st[n:], w=w) if kind == WL.NAV2D else dict(s=st, w=w))
    sp = Spec(kind, N, D, W, eta=eta, gamma=gamma, seed=seed, root=root, weights="random")
    orc = sp.run_oracle(outputs=False)
    assert orc["status"] == O.OK, what
    assert_close(res["q"][:sp.A], orc["q_root"], f"{what} root Q")
    assert_close([res["v_root"]], [orc["v_root"]], f"{what} root V")
    assert action_agrees(dict(res, q=res["q"][:sp.A]), orc, sp), what


def test_tagged_agents_and_sampled_requests_replayed_by_the_oracle():
    """Eight tagged agents run short episodes through the serving loop (plan, act, observe,
    belief update) among untagged traffic.  Every plan of a tagged agent is replayed by the
    oracle from the particles the agent held when the plan was submitted, and so is every
    eighth untagged request."""
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    models = _models(V, ctx)
    srv = V.vopp_server_create(ctx, max_batch=16, n_slots=3)
    agents = []
    try:
        rng = np.random.default_rng(5)
        for i in range(8):
            kind = WL.NAV2D if i % 2 == 0 else WL.GRID
            sp = Spec(kind, 192 + 32 * i, 2, 2, root_seed=40 + i)
            agents.append((kind, V.vopp_agent_create(models[kind], sp.states(), None, sp.N,
                                                     900 + i)))
        untagged = WL.draw_mixed_plans(48, 23, 1 << 20)
        replayed = 0
        for step in range(3):
            # one untagged burst per step, submitted before the tagged agents' plans
            burst = []
            for j, ps in enumerate(untagged[16 * step:16 * (step + 1)]):
                ps = dataclasses.replace(ps, layout_seed=1)   # the served grid model's layout
                sp = Spec.from_plan(ps)
                t = V.vopp_submit(srv, models[ps.kind], sp.states(), None, ps.N, ps.D, ps.W,
                                  ps.eta, ps.gamma, ps.seed)
                burst.append((t, ps, sp))
            tagged = []
            for i, (kind, g) in enumerate(agents):
                st, lw, _ = V.vopp_agent_get_particles(g, kind)
                D, W = 2 + (i + step) % 2, 2
                eta, gamma, seed = float(rng.uniform(0.3, 2.0)), 0.95, 7000 + 10 * i + step
                t = V.vopp_submit_agent(srv, g, D, W, eta, gamma, seed)
                tagged.append((t, kind, g, st, lw, D, W, eta, gamma, seed))
            for t, kind, g, st, lw, D, W, eta, gamma, seed in tagged:
                res, _ = V.vopp_wait(srv, t, V.VOPP_MAX_ACTIONS, 30.0)
                _replay(kind, st, lw, lw.size, D, W, eta, gamma, seed, res,
                        f"tagged agent {g:#x} step {step}")
                replayed += 1
                a = res["action"]
                V.vopp_belief_update(g, a, _observation(kind, a, st, lw), kind)
            for j, (t, ps, sp) in enumerate(burst):
                res, _ = V.vopp_wait(srv, t, V.VOPP_MAX_ACTIONS, 30.0)
                if j % 8 == step % 8:
                    orc = sp.run_oracle(outputs=False)
                    assert_close(res["q"][:sp.A], orc["q_root"], f"untagged {j} root Q")
                    assert_close([res["v_root"]], [orc["v_root"]], f"untagged {j} root V")
                    assert action_agrees(dict(res, q=res["q"][:sp.A]), orc, sp)
                    replayed += 1
        assert replayed == 24 + 6
        assert V.vopp_server_get_stats(srv)["completed"] == 24 + 48
    finally:
        V.vopp_server_destroy(srv)
        for _, g in agents:
            V.vopp_agent_destroy(g)
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)


def test_served_crowd_requests_equal_alone():
    """CROWD requests and agents through the serving loop, mixed with navigation requests."""
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    mc = V.vopp_create_model(ctx, V.make_desc(V.VOPP_CROWD))
    mn = V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D))
    srv = V.vopp_server_create(ctx, max_batch=8, n_slots=2)
    try:
        V.vopp_server_set_paused(srv, True)
        sub = []
        for i in range(6):
            if i % 2 == 0:
                st = WL.pack_crowd_states(WL.crowd_root(96 + 16 * i, 20 + i))
                n, m, A = 96 + 16 * i, mc, 5
            else:
                x, y, _ = WL.nav_root(128, 20 + i)
                st, n, m, A = np.concatenate([x, y]).astype(np.float32), 128, mn, 4
            if i == 4:
                g = V.vopp_agent_create(mc, st, None, n, 7)
                t = V.vopp_submit_agent(srv, g, 2, 2, 1.0, 0.97, 100 + i)
            else:
                g = None
                t = V.vopp_submit(srv, m, st, None, n, 2, 2, 1.0, 0.97, 100 + i)
            sub.append((t, m, st, n, A, g, 100 + i))
        V.vopp_server_set_paused(srv, False)
        for t, m, st, n, A, g, seed in sub:
            res, _ = V.vopp_wait(srv, t, A, 20.0)
            alone = V.vopp_plan(m, st, None, n, 2, 2, 1.0, 0.97, None, seed)
            assert res["q"].tolist() == alone["q"].tolist() and res["action"] == alone["action"]
            if g is not None:
                V.vopp_agent_destroy(g)
    finally:
        V.vopp_server_destroy(srv)
        V.vopp_model_destroy(mc)
        V.vopp_model_destroy(mn)
        V.vopp_ctx_destroy(ctx)



def test_agents_come_and_go_while_plans_run():
    """Agents created and destroyed (device memory from the stream-ordered pool, no device
    synchronisation) while the server runs other agents' plans leave those plans' results
    unchanged; the zero-timeout poll answers while they run."""
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    models = _models(V, ctx)
    srv = V.vopp_server_create(ctx, max_batch=8, n_slots=3)
    try:
        specs = WL.draw_mixed_plans(24, 5, 1 << 24)
        agents = [V.vopp_agent_create(models[ps.kind], Spec.from_plan(ps).states(), None, ps.N,
                                      900 + i) for i, ps in enumerate(specs)]
        tickets = [V.vopp_submit_agent(srv, g, ps.D, ps.W, ps.eta, ps.gamma, ps.seed)
                   for g, ps in zip(agents, specs)]
        churn = 0
        while V.vopp_server_get_stats(srv)["completed"] < len(tickets) and churn < 200:
            ps = specs[churn % len(specs)]
            g = V.vopp_agent_create(models[ps.kind], Spec.from_plan(ps).states(), None, ps.N, 7)
            V.vopp_agent_destroy(g)
            churn += 1
        got = {}
        while len(got) < len(tickets):
            r = V.vopp_wait_any(srv, 20.0)
            assert r is not None and r[1] == V.VOPP_OK
            got[r[0]] = r[2]
        assert V.vopp_wait_any(srv, 0.0) is None          # nothing left: answers at once
        for t, g, ps in zip(tickets, agents, specs):
            alone = V.vopp_agent_plan(g, models[ps.kind], ps.D, ps.W, ps.eta, ps.gamma, ps.seed)
            assert got[t]["q"][:len(alone["q"])].tolist() == alone["q"].tolist()
            assert got[t]["action"] == alone["action"]
        for g in agents:
            V.vopp_agent_destroy(g)
    finally:
        V.vopp_server_destroy(srv)
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)


@pytest.mark.parametrize("direct", [1, 0])
def test_direct_dispatch_matches_alone(direct):
    """An idle server's submitting thread launches the request itself (VOPP_OPT_SERVER_DIRECT
    1) or hands every request to the worker (0): one request at a time and in a burst, every
    result equals the plan run alone, bit for bit, and every request is accounted for."""
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    models = _models(V, ctx)
    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_SERVER_DIRECT, direct)
    srv = V.vopp_server_create(ctx, max_batch=8, n_slots=3)
    V.vopp_ctx_set_option(ctx, V.VOPP_OPT_SERVER_DIRECT, 1)
    try:
        specs = WL.draw_mixed_plans(24, 5, 1 << 21)
        inputs = [(ps, Spec.from_plan(ps).states()) for ps in specs]
        A = {WL.NAV2D: 4, WL.GRID: 13}
        one_by_one = []
        for ps, st in inputs[:12]:
            t = V.vopp_submit(srv, models[ps.kind], st, None, ps.N, ps.D, ps.W, ps.eta,
                              ps.gamma, ps.seed)
            one_by_one.append(V.vopp_wait(srv, t, A[ps.kind], 20.0)[0])
        stats = V.vopp_server_get_stats(srv)
        assert stats["completed"] == 12 and stats["batches"] == 12   # each ran alone
        tickets = [V.vopp_submit(srv, models[ps.kind], st, None, ps.N, ps.D, ps.W, ps.eta,
                                 ps.gamma, ps.seed) for ps, st in inputs[12:]]
        burst = []
        for t, (ps, _) in zip(tickets, inputs[12:]):
            burst.append(V.vopp_wait(srv, t, A[ps.kind], 20.0)[0])
        stats = V.vopp_server_get_stats(srv)
        assert stats["completed"] == 24 and stats["rejected"] == 0 and stats["pending"] == 0
        for res, (ps, st) in zip(one_by_one + burst, inputs):
            alone = V.vopp_plan(models[ps.kind], st, None, ps.N, ps.D, ps.W, ps.eta, ps.gamma,
                                None, ps.seed)
            assert res["q"].tolist() == alone["q"].tolist()
            assert res["action"] == alone["action"] and res["v_root"] == alone["v_root"]
        # stress: tiny plans kept three in flight, each next one submitted the moment one
        # finishes (submitting threads and the worker race for the slots); every ticket
        # completes exactly once and the in-flight reservation returns to zero
        x, y, _ = WL.nav_root(64, 9)
        st = np.concatenate([x, y])
        nav = models[WL.NAV2D]
        live, seen, n_sub = set(), set(), 0
        while n_sub < 3000 or live:
            while n_sub < 3000 and len(live) < 3:
                live.add(V.vopp_submit(srv, nav, st, None, 64, 2, 2, 1.0, 0.95, n_sub + 1))
                n_sub += 1
            got = V.vopp_wait_any(srv, 2.0)
            assert got is not None, "a submitted plan never completed"
            t, rc, _, _ = got
            assert rc == V.VOPP_OK and t in live and t not in seen
            live.discard(t)
            seen.add(t)
        stats = V.vopp_server_get_stats(srv)
        assert stats["completed"] == stats["submitted"] == 24 + 3000
        assert stats["pending"] == 0 and stats["in_flight_bytes"] == 0
    finally:
        V.vopp_server_destroy(srv)
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)
