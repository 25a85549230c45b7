"""The CROWD model (the paper's CrowdNav as a synthetic model) on the GPU against the
oracle: whole small trees node by node, the SIR belief update, the environment step, anytime
deepening and episode mode (needs a GPU).  People coordinates within the tolerance, flags
and observations bit-exact away from oracle-flagged near-threshold events (reaction radius,
bump radius, closer-bit ties)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import Gpu, Spec, action_agrees, assert_close, close, compare_full_tree

pytestmark = pytest.mark.gpu


def _full(spec, leaf_gen=True):
    g = Gpu(spec, leaf_gen=leaf_gen)
    try:
        res = g.plan()
        top = spec.D - 1 if not leaf_gen or spec.D < 2 else spec.D - 2
        orc = spec.run_oracle(dump_levels=max(top, 0))
        assert orc["status"] == O.OK
        compare_full_tree(spec, g, res, orc, max(top, 0))
        assert action_agrees(res, orc, spec)
        assert res["particle_steps"] == orc["particle_steps"]
        return res, orc
    finally:
        g.close()


@pytest.mark.parametrize("N,D,W,leaf_gen", [(48, 2, 2, True), (48, 2, 2, False), (33, 3, 1, True),
                                            (200, 1, 4, True)])
def test_crowd_full_tree(N, D, W, leaf_gen):
    _full(Spec(WL.CROWD, N, D, W, eta=1.0, gamma=0.97, seed=71, root_seed=N), leaf_gen=leaf_gen)


def test_crowd_weighted_root_near_people():
    """Robot among the people (reactions, YELL and bumps all occur) with random weights."""
    root = WL.crowd_root(64, 9, weights="random", robot=(25.0, 4.0))
    sp = Spec(WL.CROWD, 64, 2, 2, eta=0.5, gamma=0.97, seed=5, root=root, weights="random")
    res, orc = _full(sp)
    assert np.isfinite(res["v_root"])


def test_crowd_belief_update():
    from paper_2510_27191_b300 import vopp as V
    N, seed = 600, 13
    root = WL.crowd_root(N, 5, robot=(25.0, 3.0))
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_CROWD))
        om = O.make_model(O.CROWD)
        agent = V.vopp_agent_create(model, WL.pack_crowd_states(root), None, N, seed)
        for t, (a, obs) in enumerate([(0, 0b000011), (4, 0), (1, 0b110000), (0, 0b000111)]):
            g0, lw0, _ = V.vopp_agent_get_particles(agent, V.VOPP_CROWD)
            st0 = g0.reshape(15, N)
            ess, res = V.vopp_belief_update(agent, a, obs, V.VOPP_CROWD)
            rc, o = O.belief_update(om, lw0.astype(np.float64), a, obs, seed, t, x=st0[0], y=st0[1],
                                    s=st0[14].view(np.int32), pf=st0[2:14])
            assert rc == O.OK
            g, glw, ganc = V.vopp_agent_get_particles(agent, V.VOPP_CROWD)
            st = g.reshape(15, N)
            assert_close([ess], [o["ess"]], "ESS")
            if not o["ess_tie"]:
                assert res == o["resampled"]
            same = ganc == o["ancestors"]
            assert np.all(same | o["ties"])
            keep = same
            assert_close(st[0][keep], o["x"][keep], "robot x")
            assert_close(st[1][keep], o["y"][keep], "robot y")
            np.testing.assert_array_equal(st[14].view(np.int32)[keep], o["s"][keep])
            assert_close(st[2:14][:, keep], o["pf"][:, keep], "people")
            lw_ref = o["lw"] if not res else np.full(N, -math.log(N))
            assert_close(glw, lw_ref, "log weights")
        V.vopp_agent_destroy(agent)
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_crowd_env_step_and_anytime_and_episodes():
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        model = V.vopp_create_model(ctx, V.make_desc(V.VOPP_CROWD))
        om = O.make_model(O.CROWD)
        root = WL.crowd_root(1, 2, robot=(25.0, 2.0))
        state = (25.0, 2.0, int(0b011010), root["pf"][:, 0].astype(np.float64))
        env = V.vopp_env_create(model, state, 44, V.VOPP_CROWD)
        prev = V.vopp_env_get_state(env, V.VOPP_CROWD)
        rng = np.random.default_rng(3)
        for t in range(40):
            a = int(rng.integers(5))
            obs, rew, term = V.vopp_env_step(env, a, V.VOPP_CROWD)
            nxt = V.vopp_env_get_state(env, V.VOPP_CROWD)
            rc, onxt, oobs, orew, oterm = O.env_step(om, (prev[0], prev[1], prev[2],
                                                         prev[3].astype(np.float64)), a, 44, t)
            assert rc == O.OK
            assert close(np.array(nxt[:2]), np.array(onxt[:2])).all()
            assert close(nxt[3], onxt[3]).all()
            assert (nxt[2], obs, rew, term) == (onxt[2], oobs, np.float32(orew), oterm), t
            prev = nxt
            if term:
                break
        V.vopp_env_destroy(env)
        # anytime deepening on the CROWD root
        sp = Spec(WL.CROWD, 40, 2, 2, eta=1.0, gamma=0.97, seed=8, root_seed=7)
        r = V.vopp_plan_anytime(model, sp.states(), None, 40, 2, 2, 1.0, 0.97, 8)
        orc = O.plan_anytime(sp.oracle_model(), 40, 2, 2, 1.0, 0.97, 8, root_x=sp.root["x"],
                             root_y=sp.root["y"], root_s=sp.root["s"], root_pf=sp.root["pf"])
        assert orc["status"] == O.OK and orc["near_threshold"] == 0
        assert_close(r["q"], orc["q_root"], "anytime Q")
        assert_close([r["v_root"]], [orc["v_root"]], "anytime V")
        # episode mode on the CROWD root, node by node
        M, K = 96, 3
        oe = O.plan_episodes(om, M, K, 1.0, 0.97, 19, root_x=sp.root["x"], root_y=sp.root["y"],
                             root_s=sp.root["s"], root_pf=sp.root["pf"])
        assert oe["status"] == O.OK and oe["near_decisions"] == 0 and oe["near_threshold"] == 0
        ge = V.vopp_plan_episodes(model, sp.states(), None, 40, M, K, 1.0, 0.97, 19)
        n = oe["n_nodes"]
        assert ge["n_nodes"] == n and ge["particle_steps"] == oe["particle_steps"]
        assert V.vopp_episode_tree_read(ctx, V.VOPP_EP_PARENT, n).tolist() == oe["parent_an"].tolist()
        vis = V.vopp_episode_tree_read(ctx, V.VOPP_EP_VISITS, n * 5).reshape(n, 5)
        assert vis.astype(np.int64).tolist() == oe["N"].tolist()
        assert_close(V.vopp_episode_tree_read(ctx, V.VOPP_EP_PSI, n * 5).reshape(n, 5), oe["psi"], "psi")
        assert ge["action"] == oe["action"]
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)
