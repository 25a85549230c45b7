"""Serving loop (continuous batching) on the GPU: results alone vs in the mix, admission by
the HBM budget, overlap of batches (needs a GPU)."""
import time

import numpy as np
import pytest

from paper_2510_27191_b300 import workloads as WL
from tests.parity import Spec

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
        small = [V.vopp_submit(srv, models[WL.NAV2D], st[:2 * 64] if False else
                               np.concatenate([x[:64], y[:64]]), None, 64, 2, 2, 1.0, 0.95, s)
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
