"""Closed loop (Alg. 1: plan, execute, perceive, belief update) on the GPU: the environment
step against the oracle's, and the episode runner against the same calls made one by one,
with every decision checked against the oracle planning from the agent's own particles
(needs a GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import Spec, action_agrees, close

pytestmark = pytest.mark.gpu


def _model(V, ctx, kind):
    rx, ry = WL.grid_layout(1)
    return V.vopp_create_model(ctx, V.make_desc(kind, rock_x=rx if kind == WL.GRID else None,
                                                rock_y=ry if kind == WL.GRID else None))


def _omodel(kind):
    rx, ry = WL.grid_layout(1)
    return O.make_model(kind, rock_x=rx if kind == WL.GRID else None,
                        rock_y=ry if kind == WL.GRID else None)


def _start(kind):
    if kind == WL.NAV2D:
        return (5.0, 5.0)
    if kind == WL.GRID:
        return int(WL.pack_grid_state(np.array([0b01101001]), *WL.GRID_START)[0])
    return 1


def _check_env_step(kind, om, prev, a, seed, t, obs, rew, term, nxt, what):
    rc, onxt, oobs, orew, oterm = O.env_step(om, prev, a, seed, t)
    assert rc == O.OK
    if kind == WL.NAV2D:
        near = abs(onxt[0] ** 2 + onxt[1] ** 2 - 0.25) < 1e-5
        assert close(np.array(nxt), np.array(onxt)).all(), (what, nxt, onxt)
        assert close(np.array(obs), np.array(oobs)).all(), (what, obs, oobs)
        if not near:
            assert rew == np.float32(orew) and term == oterm, (what, rew, orew)
    else:   # rewards are FP32 on the device (e.g. -0.1 of TOY2)
        assert (nxt, obs, rew, term) == (onxt, oobs, np.float32(orew), oterm), what


@pytest.mark.parametrize("kind", [WL.NAV2D, WL.GRID, WL.TOY2])
def test_env_step_equals_oracle(kind):
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = _model(V, ctx, kind)
        om = _omodel(kind)
        A = V.vopp_model_num_actions(m)
        seed = 0x5EED + kind
        env = V.vopp_env_create(m, _start(kind), seed, kind)
        rng = np.random.default_rng(kind)
        prev = V.vopp_env_get_state(env, kind)
        for t in range(96):
            a = int(rng.integers(A))
            obs, rew, term = V.vopp_env_step(env, a, kind)
            nxt = V.vopp_env_get_state(env, kind)
            _check_env_step(kind, om, prev, a, seed, t, obs, rew, term, nxt, f"t={t}")
            prev = nxt
        with pytest.raises(V.VoppError):
            V.vopp_env_step(env, A, kind)
        V.vopp_env_destroy(env)
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)


@pytest.mark.parametrize("kind", [WL.NAV2D, WL.GRID])
def test_runner_equals_stepwise_loop_and_oracle_decisions(kind):
    from paper_2510_27191_b300 import vopp as V
    N, D, W, eta, gamma, seed, steps = 192, 2, 2, 0.7, 0.95, 4242, 12
    sp = Spec(kind, N, D, W, root_seed=31)
    om = _omodel(kind)
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = _model(V, ctx, kind)
        env_seed = 77 + kind
        # one call at a time, each decision and environment step checked against the oracle
        g = V.vopp_agent_create(m, sp.states(), None, N, 9)
        env = V.vopp_env_create(m, _start(kind), env_seed, kind)
        acts, rews = [], []
        for t in range(steps):
            st, lw, _ = V.vopp_agent_get_particles(g, kind)
            res = V.vopp_agent_plan(g, m, D, W, eta, gamma, seed + t)
            w = np.exp(lw.astype(np.float64) - lw.max())
            root = (dict(x=st[:N], y=st[N:], w=w) if kind == WL.NAV2D else dict(s=st, w=w))
            osp = Spec(kind, N, D, W, eta=eta, gamma=gamma, seed=seed + t, root=root)
            orc = osp.run_oracle(outputs=False)
            assert orc["status"] == O.OK
            # (a goal-boundary crossing inside the tree may flip a decision between FP32 and
            # FP64; the oracle flags those trees)
            assert action_agrees(res, orc, osp) or orc["near_threshold"] > 0, t
            prev = V.vopp_env_get_state(env, kind)
            obs, rew, term = V.vopp_env_step(env, res["action"], kind)
            _check_env_step(kind, om, prev, res["action"], env_seed, t, obs, rew, term,
                            V.vopp_env_get_state(env, kind), f"t={t}")
            acts.append(res["action"])
            rews.append(rew)
            if term:
                break
            V.vopp_belief_update(g, res["action"], obs, kind)
        V.vopp_agent_destroy(g)
        V.vopp_env_destroy(env)
        # the runner makes the same calls: identical trajectory
        g = V.vopp_agent_create(m, sp.states(), None, N, 9)
        env = V.vopp_env_create(m, _start(kind), env_seed, kind)
        ep, racts, rrews = V.vopp_run_episode(g, env, D, W, eta, gamma, seed, steps)
        assert ep["rc"] == V.VOPP_OK and ep["status"] == V.VOPP_OK
        assert racts.tolist() == acts and rrews.tolist() == rews
        assert ep["steps"] == len(acts) and ep["terminated"] == int(len(acts) < steps or term)
        disc = sum(gamma ** t * r for t, r in enumerate(rews))
        assert ep["discounted_return"] == pytest.approx(disc, rel=1e-6, abs=1e-6)
        assert ep["total_reward"] == pytest.approx(sum(rews), rel=1e-6, abs=1e-6)
        AW = V.vopp_model_num_actions(m) * W
        assert ep["particle_steps"] == len(acts) * sum(AW ** l * N for l in range(1, D + 1))
        V.vopp_agent_destroy(g)
        V.vopp_env_destroy(env)
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_anytime_episode_and_model_mismatch():
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = _model(V, ctx, WL.GRID)
        m2 = _model(V, ctx, WL.NAV2D)
        sp = Spec(WL.GRID, 256, 3, 2, root_seed=3)
        g = V.vopp_agent_create(m, sp.states(), None, 256, 1)
        env = V.vopp_env_create(m, _start(WL.GRID), 5, WL.GRID)
        ep, acts, rews = V.vopp_run_episode(g, env, 3, 2, 1.0, 0.95, 100, 30, anytime=True,
                                            budget_s=10.0)
        assert ep["rc"] == V.VOPP_OK and ep["steps"] == len(acts) >= 1
        assert ep["min_depth"] == 3          # a generous budget reaches the maximum depth
        if ep["terminated"]:
            assert rews[-1] == 10.0          # the grid episode ends by exiting east
        env2 = V.vopp_env_create(m2, (5.0, 5.0), 5, WL.NAV2D)
        ep2, _, _ = V.vopp_run_episode(g, env2, 2, 2, 1.0, 0.95, 1, 3)
        assert ep2["rc"] == V.VOPP_E_INVALID and ep2["steps"] == 0
        V.vopp_env_destroy(env2)
        V.vopp_env_destroy(env)
        V.vopp_agent_destroy(g)
        V.vopp_model_destroy(m2)
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)
