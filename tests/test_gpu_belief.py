"""SIR belief update (Sec. III-B) of the CUDA path vs the FP64 oracle (needs a GPU).

Two updates in a row on an agent: propagated states (NAV2D within 1e-4 max(|x|,1), GRID
bit-exact), normalised log weights within the same tolerance, ESS, the resampling decision
and the ancestor indices (exact unless the oracle flags a CDF position or the ESS test
within 1e-5 of a tie, where FP32 weights may decide differently).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import assert_close

pytestmark = pytest.mark.gpu


def _run(kind, N, steps, seed=9, weights="uniform"):
    """Each step starts the oracle from the GPU's current particles (identical inputs)."""
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        if kind == WL.NAV2D:
            x, y, w = WL.nav_root(N, 3, weights)
            x = (8.0 + 2.0 * (x / 10.0)).astype(np.float32)
            st = np.concatenate([x, y]).astype(np.float32)
            desc = V.make_desc(V.VOPP_NAV2D)
            om = O.make_model(O.NAV2D)
        else:
            rx, ry = WL.grid_layout(2)
            s, w = WL.grid_root(N, 3, weights)
            st = np.asarray(s, dtype=np.int32)
            desc = V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry)
            om = O.make_model(O.GRID, rock_x=rx, rock_y=ry)
        model = V.vopp_create_model(ctx, desc)
        agent = V.vopp_agent_create(model, st, w, N, seed)
        resampled_any = False
        for t, (a, obs) in enumerate(steps):
            gst0, glw0, _ = V.vopp_agent_get_particles(agent, kind)
            kw = (dict(x=gst0[:N], y=gst0[N:]) if kind == WL.NAV2D else dict(s=gst0))
            ess, res = V.vopp_belief_update(agent, a, obs, kind)
            rc, o = O.belief_update(om, glw0.astype(np.float64), a, obs, seed, t, **kw)
            assert rc == O.OK
            gst, glw, ganc = V.vopp_agent_get_particles(agent, kind)
            assert_close([ess], [o["ess"]], "ESS")
            if not o["ess_tie"]:
                assert res == o["resampled"]
            resampled_any |= res
            # ancestors: exact away from CDF ties, a neighbouring index at a flagged tie
            same = ganc == o["ancestors"]
            assert np.all(same | o["ties"]), np.flatnonzero(~(same | o["ties"]))[:5]
            assert np.all(np.abs(ganc.astype(np.int64) - o["ancestors"]) <= 1)
            # every output particle is the propagated state of the ancestor the GPU chose
            if kind == WL.NAV2D:
                assert_close(gst[:N], o["prop_x"][ganc], "x")
                assert_close(gst[N:], o["prop_y"][ganc], "y")
            else:
                np.testing.assert_array_equal(gst, o["prop_s"][ganc])
            lw_ref = o["lw"] if not res else np.full(N, -math.log(N))
            assert_close(glw, lw_ref, "log weights")
        V.vopp_agent_destroy(agent)
        V.vopp_model_destroy(model)
        return resampled_any
    finally:
        V.vopp_ctx_destroy(ctx)


def test_nav_belief_update_two_steps():
    assert _run(WL.NAV2D, 2500, [(0, (8.9, 4.2)), (3, (9.1, 3.0))])


def test_nav_belief_update_weighted_no_resample():
    _run(WL.NAV2D, 777, [(2, (5.0, 5.0))], weights="random")


def test_grid_belief_update_two_steps():
    # repeated senses of rocks 0 and 1 push the ESS below N/2 on the sixth update
    assert _run(WL.GRID, 4096, [(5, 1), (5, 1), (6, 2), (0, 0), (6, 2), (5, 1)])


def test_belief_update_degenerate_is_reported():
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        rx, ry = WL.grid_layout(2)
        model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry))
        st = WL.pack_grid_state(np.zeros(16, dtype=np.int64), rx[0], ry[0])   # rock 0 bad
        agent = V.vopp_agent_create(model, st, None, 16, 1)
        with pytest.raises(V.VoppError) as e:
            V.vopp_belief_update(agent, 5, 1, WL.GRID)      # "good" at distance 0: impossible
        assert e.value.code == V.VOPP_E_DEGENERATE
        s2, lw2, _ = V.vopp_agent_get_particles(agent, WL.GRID)
        np.testing.assert_array_equal(s2, st)
        np.testing.assert_allclose(lw2, math.log(1 / 16), rtol=1e-6)
        V.vopp_agent_destroy(agent)
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_batched_update_equals_single_updates():
    """vopp_belief_update_batch over mixed agents (NAV2D and GRID, several N, one agent with
    an impossible observation, one with subtree reuse that adopts) equals the same updates
    made one by one, bit for bit, and leaves the failing agent's belief unchanged."""
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        rx, ry = WL.grid_layout(2)
        nav = V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D))
        grid = V.vopp_create_model(ctx, V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry))
        specs = []          # (kind, model, states, N, action, obs, reuse)
        for i, n in enumerate((128, 1000, 4096)):
            x, y, _ = WL.nav_root(n, 10 + i)
            specs.append((WL.NAV2D, nav, np.concatenate([x, y]).astype(np.float32), n, i % 4,
                          (2.0 + i, 3.0), False))
        for i, n in enumerate((256, 2048)):
            s, _ = WL.grid_root(n, 20 + i)
            specs.append((WL.GRID, grid, np.asarray(s, np.int32), n, 5 + i, 1 + i, False))
        s, _ = WL.grid_root(300, 30)
        specs.append((WL.GRID, grid, np.asarray(s, np.int32), 300, 0, 1, False))  # move: obs 1 impossible
        s, _ = WL.grid_root(512, 31)
        specs.append((WL.GRID, grid, np.asarray(s, np.int32), 512, 2, 0, True))   # reuse: adopts

        def make():
            out = []
            for j, (kind, model, st, n, a, o, reuse) in enumerate(specs):
                g = V.vopp_agent_create(model, st, None, n, 500 + j)
                if reuse:
                    V.vopp_agent_set_reuse(g, True)
                    V.vopp_agent_plan(g, model, 3, 2, 1.0, 0.95, 8)
                out.append(g)
            return out

        single, batched = make(), make()
        st_single = []
        for g, (kind, model, st, n, a, o, reuse) in zip(single, specs):
            try:
                ess, res = V.vopp_belief_update(g, a, o, kind)
                st_single.append((V.VOPP_OK, ess, res))
            except V.VoppError as e:
                st_single.append((e.code, 0.0, False))
        status, ess, res = V.vopp_belief_update_batch(ctx, batched, [p[4] for p in specs],
                                                      [p[5] for p in specs], [p[0] for p in specs])
        for j, (g1, g2, sp) in enumerate(zip(single, batched, specs)):
            assert status[j] == st_single[j][0], j
            if status[j] == V.VOPP_OK:
                assert ess[j] == st_single[j][1] and res[j] == st_single[j][2], j
            p1, p2 = V.vopp_agent_get_particles(g1, sp[0]), V.vopp_agent_get_particles(g2, sp[0])
            for a1, a2 in zip(p1[:2], p2[:2]):
                np.testing.assert_array_equal(a1, a2)
            if status[j] == V.VOPP_OK and ess[j] > 0:
                np.testing.assert_array_equal(p1[2], p2[2])
        assert status[5] == V.VOPP_E_DEGENERATE
        assert ess[6] == -1.0 and V.vopp_agent_reuse_info(batched[6])["adopted_slot"] >= 0
        for g in single + batched:
            V.vopp_agent_destroy(g)
        V.vopp_model_destroy(nav)
        V.vopp_model_destroy(grid)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_batched_update_rejects_bad_batches_without_updating():
    """An agent listed twice, or an agent of another context, makes the whole batch
    VOPP_E_INVALID with no belief touched."""
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    ctx2 = V.vopp_ctx_create(0, 0, 0)
    try:
        nav = V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D))
        nav2 = V.vopp_create_model(ctx2, V.make_desc(V.VOPP_NAV2D))
        x, y, _ = WL.nav_root(64, 3)
        st = np.concatenate([x, y]).astype(np.float32)
        g1 = V.vopp_agent_create(nav, st, None, 64, 1)
        g2 = V.vopp_agent_create(nav2, st, None, 64, 2)
        before = V.vopp_agent_get_particles(g1, WL.NAV2D)
        for agents in ([g1, g1], [g1, g2]):
            with pytest.raises(V.VoppError) as e:
                V.vopp_belief_update_batch(ctx, agents, [0] * len(agents),
                                           [(5.0, 5.0)] * len(agents), [WL.NAV2D] * len(agents))
            assert e.value.code == V.VOPP_E_INVALID
        after = V.vopp_agent_get_particles(g1, WL.NAV2D)
        for a, b in zip(before[:2], after[:2]):
            np.testing.assert_array_equal(a, b)
        V.vopp_agent_destroy(g1)
        V.vopp_agent_destroy(g2)
        V.vopp_model_destroy(nav)
        V.vopp_model_destroy(nav2)
    finally:
        V.vopp_ctx_destroy(ctx)
        V.vopp_ctx_destroy(ctx2)
