"""Episode mode (Alg. 1-3 as printed) on the GPU against the oracle, node by node: the
tree's structure and visit counts exactly, reward sums, preferences and values within the
tolerance (needs a GPU).  Fixtures are chosen so that the oracle flags no sampled decision
within 1e-5 of a boundary (where FP32 simulation and FP64 could choose differently)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import assert_close

pytestmark = pytest.mark.gpu

RX, RY = WL.grid_layout(1)


def _case(kind, seed=1):
    if kind == WL.GRID:
        s, _ = WL.grid_root(200, seed)
        return dict(states=s.astype(np.int32), N=200, M=256, K=4, okw=dict(root_s=s),
                    omodel=O.make_model(O.GRID, rock_x=RX, rock_y=RY), desc=dict(rock_x=RX, rock_y=RY))
    if kind == WL.NAV2D:
        x, y, _ = WL.nav_root(200, seed)
        return dict(states=np.concatenate([x, y]).astype(np.float32), N=200, M=256, K=3,
                    okw=dict(root_x=x, root_y=y), omodel=O.make_model(O.NAV2D), desc={})
    s, _ = WL.toy2_root_sampled(100, seed)
    return dict(states=s.astype(np.int32), N=100, M=300, K=4, okw=dict(root_s=s),
                omodel=O.make_model(O.TOY2, pi_mode=O.PI_FIXED, pi_fixed=(0.6, 0.4)),
                desc=dict(pi_mode=WL.PI_FIXED, pi_fixed=(0.6, 0.4)))


@pytest.mark.parametrize("kind", [WL.GRID, WL.NAV2D, WL.TOY2])
def test_episode_tree_equals_oracle(kind):
    from paper_2510_27191_b300 import vopp as V
    c = _case(kind)
    eta, gamma, seed = 0.8, 0.95, 1004
    orc = O.plan_episodes(c["omodel"], c["M"], c["K"], eta, gamma, seed, **c["okw"])
    assert orc["status"] == O.OK and orc["near_decisions"] == 0 and orc["near_threshold"] == 0
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = V.vopp_create_model(ctx, V.make_desc(kind, **c["desc"]))
        A = V.vopp_model_num_actions(m)
        res = V.vopp_plan_episodes(m, c["states"], None, c["N"], c["M"], c["K"], eta, gamma, seed)
        n = orc["n_nodes"]
        assert res["depth_reached"] == c["K"] and res["n_nodes"] == n
        assert res["particle_steps"] == orc["particle_steps"]
        par = V.vopp_episode_tree_read(ctx, V.VOPP_EP_PARENT, n)
        dep = V.vopp_episode_tree_read(ctx, V.VOPP_EP_DEPTH, n)
        vis = V.vopp_episode_tree_read(ctx, V.VOPP_EP_VISITS, n * A).reshape(n, A)
        assert par.tolist() == orc["parent_an"].tolist()
        assert dep.tolist() == orc["depth"].tolist()
        assert vis.astype(np.int64).tolist() == orc["N"].tolist()
        rew = V.vopp_episode_tree_read(ctx, V.VOPP_EP_REWARD, n * A).reshape(n, A)
        psi = V.vopp_episode_tree_read(ctx, V.VOPP_EP_PSI, n * A).reshape(n, A)
        val = V.vopp_episode_tree_read(ctx, V.VOPP_EP_V, n)
        assert_close(rew, orc["C"], "reward sums")
        assert_close(psi, orc["psi"], "preferences")
        assert_close(val, orc["V"], "values")
        assert res["action"] == orc["action"]
        assert_close(res["q"], orc["q_root"], "root Q")
        assert_close([res["v_root"]], [orc["v_root"]], "root V")
        assert_close(res["policy"], orc["policy"], "root policy")
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_episode_agent_budget_capacity_and_refusals():
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        c = _case(WL.GRID)
        m = V.vopp_create_model(ctx, V.make_desc(WL.GRID, **c["desc"]))
        plain = V.vopp_plan_episodes(m, c["states"], None, c["N"], 512, 3, 1.0, 0.95, 7)
        g = V.vopp_agent_create(m, c["states"], None, c["N"], 3)
        ag = V.vopp_agent_plan_episodes(g, m, 512, 3, 1.0, 0.95, 7)
        assert ag["q"].tolist() == plain["q"].tolist() and ag["action"] == plain["action"]
        assert ag["n_nodes"] == plain["n_nodes"]
        V.vopp_agent_destroy(g)
        early = V.vopp_plan_episodes(m, c["states"], None, c["N"], 512, 6, 1.0, 0.95, 7,
                                     budget_s=1e-9)
        assert early["depth_reached"] == 1
        with pytest.raises(V.VoppError) as e:
            V.vopp_plan_episodes(m, c["states"], None, c["N"], 512, 3, 1.0, 0.95, 7, max_nodes=3)
        assert e.value.code == V.VOPP_E_NOMEM
        with pytest.raises(V.VoppError) as e:
            V.vopp_plan_episodes(m, c["states"], None, c["N"], 0, 3, 1.0, 0.95, 7)
        assert e.value.code == V.VOPP_E_INVALID
        mn = V.vopp_create_model(ctx, V.make_desc(WL.NAV2D, pi_mode=WL.PI_NAV_SOFTMAX_DIST))
        x, y, _ = WL.nav_root(16, 1)
        with pytest.raises(V.VoppError) as e:
            V.vopp_plan_episodes(mn, np.concatenate([x, y]), None, 16, 8, 2, 1.0, 0.95, 7)
        assert e.value.code == V.VOPP_E_INVALID
        V.vopp_model_destroy(mn)
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)
