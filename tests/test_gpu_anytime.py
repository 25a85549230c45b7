"""Anytime iterative deepening with persistent preferences (Alg. 1 planning loop, Eq. 3) on
the GPU against the oracle: the root result and, at every internal level, each node's
preferences, value and Q after the last iteration (needs a GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import RTOL, Spec, assert_close

pytestmark = pytest.mark.gpu


def _oracle_anytime(sp: Spec, K: int):
    m = sp.oracle_model()
    w = sp.root.get("w")
    w = None if w is None else np.asarray(w, dtype=np.float64)
    kw = (dict(root_x=sp.root["x"], root_y=sp.root["y"]) if sp.kind == WL.NAV2D
          else dict(root_s=sp.root["s"]))
    return O.plan_anytime(m, sp.N, K, sp.W, sp.eta, sp.gamma, sp.seed, root_w=w,
                          outputs=True, **kw)


def _psi_action_agrees(action, psi):
    top = np.sort(psi)[::-1]
    if len(top) < 2 or top[0] - top[1] > RTOL * max(abs(top[0]), 1.0):
        return action == int(np.argmax(psi))
    return action in np.flatnonzero(psi >= top[0] - RTOL * max(abs(top[0]), 1.0))


CASES = [
    # kind, N, K, W, eta, extra Spec arguments
    (WL.NAV2D, 96, 4, 2, 0.5, dict(pi_mode=WL.PI_NAV_SOFTMAX_DIST, root_seed=4)),
    (WL.NAV2D, 200, 3, 3, 1.5, dict(weights="random", root_seed=5)),
    (WL.GRID, 64, 3, 2, 1.0, dict(root_seed=6)),
    (WL.GRID, 33, 2, 3, 0.3, dict(weights="random", root_seed=7)),
    (WL.TOY2, 50, 5, 2, 0.7, dict(branch_mode=WL.BRANCH_ENUMERATE, pi_fixed=(0.7, 0.3),
                                  pi_mode=WL.PI_FIXED)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_anytime_equals_oracle(case):
    from paper_2510_27191_b300 import vopp as V
    kind, N, K, W, eta, kw = CASES[case]
    sp = Spec(kind, N, K, W, eta=eta, seed=1000 + case, **kw)
    orc = _oracle_anytime(sp, K)
    assert orc["status"] == O.OK
    assert orc["near_threshold"] == 0, "fixture crosses the goal boundary; pick another seed"
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = V.vopp_create_model(ctx, V.make_desc(kind, sp.branch_mode, sp.pi_mode,
                                                 pi_temp=sp.pi_temp, pi_fixed=sp.pi_fixed,
                                                 rock_x=sp.rock_x, rock_y=sp.rock_y))
        w = sp.root.get("w")
        res = V.vopp_plan_anytime(m, sp.states(), None if w is None else np.asarray(w, np.float32),
                                  N, K, W, eta, sp.gamma, sp.seed)
        assert res["depth_reached"] == K
        A = sp.A
        assert_close(res["q"], orc["q_root"], "root Q (last iteration)")
        assert_close([res["v_root"]], [orc["v_root"]], "root V")
        assert_close(res["policy"], orc["policy"], "root policy")
        assert _psi_action_agrees(res["action"], orc["psi_root"])
        for l in range(K):
            n = (A * W) ** l
            psi = V.vopp_tree_read(ctx, V.VOPP_FIELD_PSI, l, n * A).reshape(n, A)
            assert_close(psi, orc["psi_levels"][l], f"Psi level {l}")
            q = V.vopp_tree_read(ctx, V.VOPP_FIELD_Q, l, n * A).reshape(n, A)
            assert_close(q, orc["Q"][l], f"Q level {l}")
            v = V.vopp_tree_read(ctx, V.VOPP_FIELD_V, l, n)
            assert_close(v, orc["V"][l], f"V level {l}")
        # steps: each iteration k adds level k-2, rebuilds level k-1 and expands level k
        AW = A * W
        steps = sum(AW ** k * N for k in range(1, K + 1))
        steps += sum(AW ** (k - 1) * N for k in range(2, K + 1))
        steps += sum(AW ** l * N for l in range(1, K - 1))
        assert res["particle_steps"] == steps
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_first_iteration_is_the_depth_one_plan_and_budget_stops_early():
    from paper_2510_27191_b300 import vopp as V
    sp = Spec(WL.NAV2D, 256, 1, 4, eta=0.8, seed=9)
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = V.vopp_create_model(ctx, V.make_desc(WL.NAV2D))
        one = V.vopp_plan(m, sp.states(), None, sp.N, 1, 4, 0.8, 0.95, None, 9)
        a1 = V.vopp_plan_anytime(m, sp.states(), None, sp.N, 1, 4, 0.8, 0.95, 9)
        assert_close(a1["q"], one["q"], "Q")
        assert_close([a1["v_root"]], [one["v_root"]], "V")
        # a budget that is over after the first iteration stops there
        early = V.vopp_plan_anytime(m, sp.states(), None, sp.N, 6, 4, 0.8, 0.95, 9,
                                    budget_s=1e-9)
        assert early["depth_reached"] == 1 and early["q"].tolist() == a1["q"].tolist()
        # no time limit: runs to the maximum depth; a generous budget does too
        full = V.vopp_plan_anytime(m, sp.states(), None, sp.N, 3, 4, 0.8, 0.95, 9)
        gen = V.vopp_plan_anytime(m, sp.states(), None, sp.N, 3, 4, 0.8, 0.95, 9, budget_s=60.0)
        assert full["depth_reached"] == gen["depth_reached"] == 3
        assert full["q"].tolist() == gen["q"].tolist() and full["action"] == gen["action"]
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_agent_anytime_equals_plain_anytime():
    from paper_2510_27191_b300 import vopp as V
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        rx, ry = WL.grid_layout(1)
        m = V.vopp_create_model(ctx, V.make_desc(WL.GRID, rock_x=rx, rock_y=ry))
        sp = Spec(WL.GRID, 300, 3, 2, seed=21)
        g = V.vopp_agent_create(m, sp.states(), None, sp.N, 5)
        a = V.vopp_agent_plan_anytime(g, m, 3, 2, 1.0, 0.95, 21)
        b = V.vopp_plan_anytime(m, sp.states(), None, sp.N, 3, 2, 1.0, 0.95, 21)
        assert a["q"].tolist() == b["q"].tolist() and a["v_root"] == b["v_root"]
        assert a["action"] == b["action"] and a["depth_reached"] == 3
        V.vopp_agent_destroy(g)
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)
