"""Subtree reuse on the CUDA path (needs a GPU).

An agent with reuse on keeps its plan's tree; a belief update whose observation equals the
sampled observation of a root branch (a, k) adopts that branch's particle set and subtree,
and the agent's next plans continue it.  A reused plan of depth D after adopting the branch
path (c1, ..., cP) must equal the subtree below that path in the oracle's tree of depth
P + D built from the original root with the original seed (the oracle's path mode): the
adopted particles bit for bit (GRID states) and within 1e-4 (log weights), every node's V
and the root's Q within 1e-4 max(|oracle|, 1), the action whenever the oracle's top-two gap
exceeds that tolerance.  The copied levels must equal the same levels expanded again under
the same keys bit for bit, and a served reused plan must equal the synchronous one.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import RTOL, assert_close

pytestmark = pytest.mark.gpu

N, W, ETA, GAMMA, SEED = 256, 3, 1.0, 0.95, 5
SENSE_A1, SENSE_A2 = 6, 9          # sense actions: their branches sample "good" / "bad"
MIXED_SEED = 4321


def _grid():
    rx, ry = WL.grid_layout(3)
    s, _ = WL.grid_root(N, 4)
    return rx, ry, np.asarray(s, dtype=np.int32)


def _pick_obs(obs_level, a):
    """An observation sampled by some branch of action a (the second branch's), and the
    slot the update must adopt: the lowest k of a whose observation equals it."""
    vals = [int(obs_level[a * W + k][0]) for k in range(W)]
    o = vals[1]
    return o, a * W + vals.index(o)


def _check_action(res, q_oracle):
    order = np.argsort(-q_oracle, kind="stable")
    gap = q_oracle[order[0]] - q_oracle[order[1]]
    if gap > RTOL * max(abs(q_oracle[order[0]]), 1.0):
        assert res["action"] == int(order[0])


def _run_chain(V, ctx, model, s, obs_fn, **kw):
    agent = V.vopp_agent_create(model, s, None, N, 77)
    V.vopp_agent_set_reuse(agent, True)
    served = kw.get("served", False)
    mixed = kw.get("mixed", False)   # each served plan batched with a depth-2 plan from s
    srv = V.vopp_server_create(ctx, 8, 2) if served else None
    depths = kw.get("depths", (4, 3, 3))

    def plan(d, seed):
        if not served:
            return V.vopp_agent_plan(agent, model, d, W, ETA, GAMMA, seed)
        if mixed:
            V.vopp_server_set_paused(srv, True)
        t = V.vopp_submit_agent(srv, agent, d, W, ETA, GAMMA, seed)
        if mixed:
            t2 = V.vopp_submit(srv, model, s, None, N, 2, W, ETA, GAMMA, MIXED_SEED)
            V.vopp_server_set_paused(srv, False)
            out["extra"].append(V.vopp_wait(srv, t2, 13, 30.0)[0])
        return V.vopp_wait(srv, t, 13, 30.0)[0]

    out = dict(res=[], particles=[], info=[], slots=[], trees=[], extra=[])
    try:
        out["res"].append(plan(depths[0], SEED))
        for step, a in enumerate((SENSE_A1, SENSE_A2)):
            o, slot = obs_fn(step, a)
            out["slots"].append(slot)
            ess, resampled = V.vopp_belief_update(agent, a, o, WL.GRID)
            assert ess == -1.0 and not resampled
            out["info"].append(V.vopp_agent_reuse_info(agent))
            st, lw, _ = V.vopp_agent_get_particles(agent, WL.GRID)
            out["particles"].append((st.copy(), lw.copy()))
            out["res"].append(plan(depths[step + 1], 1234 + step))   # the seed is not used
            if not served:
                d = depths[step + 1]
                out["trees"].append([V.vopp_tree_read(ctx, V.VOPP_FIELD_V, l, (W * 13) ** l)
                                     for l in range(d + 1)])
    finally:
        if srv:
            V.vopp_server_destroy(srv)
        V.vopp_agent_destroy(agent)
    return out


@pytest.fixture(scope="module")
def grid_chain():
    from paper_2510_27191_b300 import vopp as V
    rx, ry, s = _grid()
    om = O.make_model(O.GRID, rock_x=rx, rock_y=ry)
    # oracle: level-1 observations of the first tree, then the two reused plans as subtrees
    o1 = O.plan(om, N, 1, W, ETA, GAMMA, SEED, root_s=s)
    oracle_obs = {0: o1["obs"][1]}
    picks = {}

    def obs_fn(step, a):
        if step not in picks:
            picks[step] = _pick_obs(oracle_obs[step], a)
        return picks[step]

    o_plans = []
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        V.vopp_ctx_set_tree_detail(ctx, V.VOPP_TREE_FULL)
        model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry))

        # the second adoption needs the first reused plan's level-2 observations: take them
        # from the oracle's subtree below the first adopted slot
        def obs_fn_chain(step, a):
            if step == 1 and 1 not in oracle_obs:
                path = [picks[0][1]]
                op = O.plan(om, N, 1 + 3, W, ETA, GAMMA, SEED, root_s=s, path=path, dump_levels=2)
                o_plans.append(op)
                oracle_obs[1] = op["obs"][2]
            return obs_fn(step, a)

        copy = _run_chain(V, ctx, model, s, obs_fn_chain)
        V.vopp_ctx_set_option(ctx, V.VOPP_OPT_REUSE_COPY, 0)
        recompute = _run_chain(V, ctx, model, s, obs_fn_chain)
        V.vopp_ctx_set_option(ctx, V.VOPP_OPT_REUSE_COPY, 1)
        served = _run_chain(V, ctx, model, s, obs_fn_chain, served=True)
        # the same chain with a plan that needs a root preparation in every batch (the
        # continued plans' copies then run in that launch)
        mixed = _run_chain(V, ctx, model, s, obs_fn_chain, served=True, mixed=True)
        mixed_ref = V.vopp_plan(model, s, None, N, 2, W, ETA, GAMMA, None, MIXED_SEED)
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)
    path2 = [picks[0][1], picks[1][1]]
    o3 = O.plan(om, N, 2 + 3, W, ETA, GAMMA, SEED, root_s=s, path=path2, dump_levels=2)
    return dict(copy=copy, recompute=recompute, served=served, mixed=mixed, mixed_ref=mixed_ref,
                oracle=[o_plans[0], o3], picks=picks)


def test_adoption_takes_the_matching_branch_and_its_particles(grid_chain):
    c = grid_chain["copy"]
    picks = grid_chain["picks"]
    for step in range(2):
        info = c["info"][step]
        assert info["adopted_slot"] == picks[step][1]
        assert info["key_level"] == step + 1
        assert info["kept_levels"] >= 1
        # the belief is the oracle's node at the adopted path (dumped at level step + 1)
        op = grid_chain["oracle"][step]
        st, lw = c["particles"][step]
        lev = step + 1
        np.testing.assert_array_equal(st, op["ps"][lev][0])
        assert_close(lw, op["plw"][lev][0], f"adopted log weights, step {step}")


def test_reused_plans_equal_the_oracle_subtree(grid_chain):
    c = grid_chain["copy"]
    for step in range(2):
        res = c["res"][step + 1]
        op = grid_chain["oracle"][step]
        P = step + 1
        assert res["flags"] & 4                       # VOPP_FLAG_REUSED
        q_or = op["Q"][P][0]
        assert_close(res["q"], q_or, f"root Q of reused plan {step}")
        assert_close([res["v_root"]], [op["V"][P][0]], f"root V of reused plan {step}")
        _check_action(res, q_or)
        # every level's V (level l of the reused plan = level P + l below the path)
        for l, v in enumerate(c["trees"][step]):
            if l == 0:
                continue
            assert_close(v, op["V"][P + l], f"V level {l} of reused plan {step}")
    assert c["res"][1]["reused_levels"] == 1          # depth-4 tree: level 1 of the subtree
    assert c["res"][2]["reused_levels"] == 0          # depth-3 tree: nothing below its root


def test_copied_levels_equal_recomputed_levels(grid_chain):
    a, b = grid_chain["copy"], grid_chain["recompute"]
    for ra, rb in zip(a["res"], b["res"]):
        np.testing.assert_array_equal(ra["q"], rb["q"])
        assert ra["v_root"] == rb["v_root"] and ra["action"] == rb["action"]
    assert b["res"][1]["reused_levels"] == 0
    for ta, tb in zip(a["trees"], b["trees"]):
        for va, vb in zip(ta, tb):
            np.testing.assert_array_equal(va, vb)


def test_served_reused_plans_equal_synchronous(grid_chain):
    a, b = grid_chain["copy"], grid_chain["served"]
    for ra, rb in zip(a["res"], b["res"]):
        np.testing.assert_array_equal(ra["q"], rb["q"])
        assert ra["v_root"] == rb["v_root"] and ra["action"] == rb["action"]
        assert ra["flags"] == rb["flags"] and ra["reused_levels"] == rb["reused_levels"]
    assert [i["adopted_slot"] for i in a["info"]] == [i["adopted_slot"] for i in b["info"]]


def test_reused_plans_batched_with_a_root_preparation(grid_chain):
    """Continued plans batched with a plan that needs a root preparation (their copies then
    ride in the root preparation launch) equal the synchronous chain bit for bit, and so does
    the other plan its plain run."""
    a, b = grid_chain["copy"], grid_chain["mixed"]
    for ra, rb in zip(a["res"], b["res"]):
        np.testing.assert_array_equal(ra["q"], rb["q"])
        assert ra["v_root"] == rb["v_root"] and ra["action"] == rb["action"]
        assert ra["flags"] == rb["flags"] and ra["reused_levels"] == rb["reused_levels"]
    assert len(b["extra"]) == 3
    for r in b["extra"]:
        np.testing.assert_array_equal(r["q"], grid_chain["mixed_ref"]["q"])
        assert r["v_root"] == grid_chain["mixed_ref"]["v_root"]


def test_unmatched_observation_falls_back_to_the_sir_update():
    """NAV2D observations are continuous: no branch matches, the SIR update runs, nothing is
    kept, and the next plan equals that of an agent without reuse."""
    from paper_2510_27191_b300 import vopp as V
    x, y, _ = WL.nav_root(N, 3)
    st = np.concatenate([x, y]).astype(np.float32)
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D))
        res = []
        for reuse in (True, False):
            g = V.vopp_agent_create(model, st, None, N, 11)
            V.vopp_agent_set_reuse(g, reuse)
            r0 = V.vopp_agent_plan(g, model, 3, 2, 0.5, 0.95, 3)
            ess, _ = V.vopp_belief_update(g, r0["action"], (4.0, 5.0), WL.NAV2D)
            assert ess > 0.0
            info = V.vopp_agent_reuse_info(g)
            assert info["adopted_slot"] == -1 and info["kept_levels"] == 0
            r1 = V.vopp_agent_plan(g, model, 3, 2, 0.5, 0.95, 4)
            assert not (r1["flags"] & 4)
            res.append(r1)
            V.vopp_agent_destroy(g)
        np.testing.assert_array_equal(res[0]["q"], res[1]["q"])
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_shallow_tree_or_width_change_plans_afresh():
    """A depth-2 tree keeps no level-1 particle sets, so even a matching observation runs the
    SIR update; after an adoption, a plan of another width does not continue the subtree: it
    plans afresh from the adopted particles (equal, within tolerance, to vopp_plan from them
    with that seed)."""
    from paper_2510_27191_b300 import vopp as V
    rx, ry, s = _grid()
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry))
        g = V.vopp_agent_create(model, s, None, N, 31)
        V.vopp_agent_set_reuse(g, True)
        V.vopp_agent_plan(g, model, 2, W, ETA, GAMMA, 3)
        ess, _ = V.vopp_belief_update(g, 2, 0, WL.GRID)          # move N: NULL matches
        assert ess > 0.0 and V.vopp_agent_reuse_info(g)["adopted_slot"] == -1
        V.vopp_agent_plan(g, model, 3, W, ETA, GAMMA, 4)
        ess, _ = V.vopp_belief_update(g, 2, 0, WL.GRID)
        assert ess == -1.0 and V.vopp_agent_reuse_info(g)["adopted_slot"] >= 0
        r = V.vopp_agent_plan(g, model, 3, W - 1, ETA, GAMMA, 5)  # another width: fresh
        assert not (r["flags"] & 4) and r["reused_levels"] == 0
        st, lw, _ = V.vopp_agent_get_particles(g, WL.GRID)
        w = np.exp(lw.astype(np.float64) - lw.max()).astype(np.float32)
        ref = V.vopp_plan(model, st, w, N, 3, W - 1, ETA, GAMMA, None, 5)
        assert_close(r["q"], ref["q"], "fresh plan after a width change")
        V.vopp_agent_destroy(g)
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_reuse_keeps_no_tree_for_continuous_observations_unless_forced():
    """enable = 1 keeps no tree for a NAV2D agent (continuous observations practically never
    match) and its plans equal an agent's without reuse bit for bit; enable = 2 keeps the tree
    for NAV2D too: the observation a root branch sampled, fed back, is adopted."""
    from paper_2510_27191_b300 import vopp as V
    x, y, _ = WL.nav_root(N, 3)
    st = np.concatenate([x, y]).astype(np.float32)
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        V.vopp_ctx_set_tree_detail(ctx, V.VOPP_TREE_FULL)
        model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D))
        with pytest.raises(V.VoppError):
            g = V.vopp_agent_create(model, st, None, N, 11)
            try:
                V.vopp_agent_set_reuse(g, 3)
            finally:
                V.vopp_agent_destroy(g)
        out = {}
        for enable in (0, 1, 2):
            g = V.vopp_agent_create(model, st, None, N, 11)
            V.vopp_agent_set_reuse(g, enable)
            r0 = V.vopp_agent_plan(g, model, 3, 2, 0.5, 0.95, 3)
            a = int(r0["action"])
            obs = V.vopp_tree_read(ctx, V.VOPP_FIELD_OBS, 1, 2 * 4 * 2)   # level 1: (x, y) per child
            slot = a * 2 + 1                                   # the second branch of action a
            o = (float(obs[2 * slot]), float(obs[2 * slot + 1]))
            V.vopp_belief_update(g, a, o, WL.NAV2D)
            info = V.vopp_agent_reuse_info(g)
            r1 = V.vopp_agent_plan(g, model, 3, 2, 0.5, 0.95, 4)
            out[enable] = (info["adopted_slot"], r1)
            V.vopp_agent_destroy(g)
        assert out[0][0] == -1 and out[1][0] == -1
        np.testing.assert_array_equal(out[0][1]["q"], out[1][1]["q"])
        assert not (out[1][1]["flags"] & V.VOPP_FLAG_REUSED)
        assert out[2][0] >= 0 and (out[2][1]["flags"] & V.VOPP_FLAG_REUSED)
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)
