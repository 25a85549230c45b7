"""Batched plans (one launch per stage covering every plan) and the full-size grid plan
(needs a GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import workloads as WL
from tests.parity import Gpu, Spec, action_agrees, assert_close, compare_full_tree

pytestmark = pytest.mark.gpu


def _mixed_specs(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = [WL.NAV2D, WL.GRID, WL.TOY2][i % 3]
        N = int(rng.integers(1, 700))
        W = int(rng.integers(1, 4)) + (1 if kind == WL.TOY2 else 0)
        A = {WL.NAV2D: 4, WL.GRID: 13, WL.TOY2: 2}[kind]
        D = int(rng.integers(0, 4))
        while D > 1 and (A * W) ** D * N > 3e6:
            D -= 1
        bm = WL.BRANCH_ENUMERATE if (kind == WL.TOY2 and i % 2) else WL.BRANCH_SAMPLE
        if bm == WL.BRANCH_ENUMERATE:
            W = max(W, 2)
        out.append(Spec(kind, N, D, W, eta=float(rng.uniform(0.2, 2.0)), gamma=0.95,
                        seed=int(rng.integers(1, 2**40)), root_seed=i + 1, branch_mode=bm,
                        weights="random" if i % 4 == 1 else "uniform"))
    return out


def test_batch_equals_individual_plans_and_oracle():
    from paper_2510_27191_b300 import vopp as V
    specs = _mixed_specs(24, 3)
    ctx = V.vopp_ctx_create(0, 0, 0)
    models = {}
    try:
        reqs, singles = [], []
        for s in specs:
            key = (s.kind, s.branch_mode)
            if key not in models:
                models[key] = V.vopp_create_model(ctx, V.make_desc(
                    s.kind, s.branch_mode, rock_x=WL.grid_layout(1)[0] if s.kind == WL.GRID else None,
                    rock_y=WL.grid_layout(1)[1] if s.kind == WL.GRID else None))
            s.rock_x, s.rock_y = (WL.grid_layout(1) if s.kind == WL.GRID else (None, None))
            w = s.root.get("w")
            reqs.append(dict(model=models[key], states=s.states(),
                             weights=None if w is None else np.asarray(w, np.float32), n=s.N,
                             depth=s.D, width=s.W, eta=s.eta, gamma=s.gamma, seed=s.seed, A=s.A))
        outs, keep = V.vopp_plan_batch(ctx, reqs)
        for r, s in zip(reqs, specs):
            singles.append(V.vopp_plan(r["model"], r["states"], r["weights"], s.N, s.D, s.W, s.eta,
                                       s.gamma, None, s.seed))
        for i, (a, b, s) in enumerate(zip(outs, singles, specs)):
            assert a["q"].tolist() == b["q"].tolist(), i
            assert a["v_root"] == b["v_root"] and a["action"] == b["action"], i
            orc = s.run_oracle(outputs=False)
            assert orc["status"] == O.OK
            assert_close(a["q"], orc["q_root"], f"plan {i} root Q")
            assert_close([a["v_root"]], [orc["v_root"]], f"plan {i} root V")
            assert action_agrees(a, orc, s)
            assert a["particle_steps"] == orc["particle_steps"]
        del keep
    finally:
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)


def test_batch_tree_read_per_plan():
    from paper_2510_27191_b300 import vopp as V
    specs = [Spec(WL.NAV2D, 64, 2, 2, seed=1), Spec(WL.GRID, 100, 2, 2, seed=2)]
    ctx = V.vopp_ctx_create(0, 0, 0)
    V.vopp_ctx_set_tree_detail(ctx, V.VOPP_TREE_FULL)
    try:
        ms = [V.vopp_create_model(ctx, V.make_desc(s.kind, rock_x=s.rock_x, rock_y=s.rock_y))
              for s in specs]
        reqs = [dict(model=m, states=s.states(), weights=None, n=s.N, depth=s.D, width=s.W,
                     eta=s.eta, gamma=s.gamma, seed=s.seed, A=s.A) for m, s in zip(ms, specs)]
        outs, keep = V.vopp_plan_batch(ctx, reqs)
        for p, s in enumerate(specs):
            orc = s.run_oracle()
            n = (s.A * s.W) ** 2
            assert_close(V.vopp_tree_read(ctx, V.VOPP_FIELD_V, 2, n, plan=p), orc["V"][2], "V2")
            np.testing.assert_array_equal(V.vopp_tree_read(ctx, V.VOPP_FIELD_REP, 2, n, plan=p),
                                          orc["rep"][2])
        for m in ms:
            V.vopp_model_destroy(m)
        del keep
    finally:
        V.vopp_ctx_destroy(ctx)


def test_config3_grid_sampled_subtrees_bit_exact():
    """GRID 11x11, 8 rocks, N=2048, depth 5, 13 actions x 3 branches (9.0e7 leaves,
    1.9e11 particle-steps): one whole level-2 subtree (1.25e8 particle-steps of FP64 oracle:
    the node's particles, Q and V, and every node and branch below it) and three level-3
    subtrees against the oracle's path mode, integers exact.  The root and level 1 are too
    large for the oracle here (the root is 1.9e11 particle-steps, a level-1 node 4.9e9): the
    root's Q and V are checked against the closed-form backup (Alg. 3, Eq. 1) of the GPU's
    own level-1 statistics, so the upper tree's arithmetic, not its inputs, is what that
    check covers."""
    from paper_2510_27191_b300 import vopp as V
    spec = Spec.from_plan(WL.CONFIG3)
    g = Gpu(spec)
    try:
        res = g.plan()
        AW = 39
        rng = np.random.default_rng(1)
        for _ in range(3):
            path = tuple(int(v) for v in rng.integers(0, AW, 3))
            sub = spec.run_oracle(path=path)
            assert sub["status"] == O.OK
            n3 = (path[0] * AW + path[1]) * AW + path[2]
            assert_close(g.read(V.VOPP_FIELD_V, 3, 1, n3), sub["V"][3], f"V3 {path}")
            assert_close(g.read(V.VOPP_FIELD_Q, 3, 13, n3 * 13), sub["Q"][3][0], f"Q3 {path}")
            assert_close(g.read(V.VOPP_FIELD_V, 4, AW, n3 * AW), sub["V"][4], f"V4 {path}")
            assert_close(g.read(V.VOPP_FIELD_Q, 4, AW * 13, n3 * AW * 13), sub["Q"][4].ravel(),
                         f"Q4 {path}")
            assert_close(g.read(V.VOPP_FIELD_RBAR, 4, AW, n3 * AW), sub["rbar"][4], f"rbar4 {path}")
            assert_close(g.read(V.VOPP_FIELD_LOMEGA, 4, AW, n3 * AW), sub["lomega"][4], f"lom4 {path}")
            np.testing.assert_array_equal(g.read(V.VOPP_FIELD_REP, 4, AW, n3 * AW), sub["rep"][4])
            n5 = AW * AW
            o5 = n3 * n5
            assert_close(g.read(V.VOPP_FIELD_V, 5, n5, o5), sub["V"][5], f"V5 {path}")
            assert_close(g.read(V.VOPP_FIELD_RBAR, 5, n5, o5), sub["rbar"][5], f"rbar5 {path}")
            assert_close(g.read(V.VOPP_FIELD_LOMEGA, 5, n5, o5), sub["lomega"][5], f"lom5 {path}")
            np.testing.assert_array_equal(g.read(V.VOPP_FIELD_REP, 5, n5, o5), sub["rep"][5])
            np.testing.assert_array_equal(g.read(V.VOPP_FIELD_OBS, 5, 2 * n5, 2 * o5),
                                          sub["obs"][5].ravel())
            # the level-3 particle store (materialised), bit-exact states
            ps = g.read(V.VOPP_FIELD_PS, 3, 2048, n3 * 2048)
            sub_d = spec.run_oracle(path=path, dump_levels=3, outputs=False)
            np.testing.assert_array_equal(ps, sub_d["ps"][3][0])
            assert_close(g.read(V.VOPP_FIELD_PLW, 3, 2048, n3 * 2048), sub_d["plw"][3][0], "plw3")
        # one level-2 node and its whole subtree (depth 3 below it)
        path2 = (int(rng.integers(0, AW)), int(rng.integers(0, AW)))
        n2 = path2[0] * AW + path2[1]
        sub2 = spec.run_oracle(path=path2, dump_levels=2)
        assert sub2["status"] == O.OK
        assert_close(g.read(V.VOPP_FIELD_V, 2, 1, n2), sub2["V"][2], f"V2 {path2}")
        assert_close(g.read(V.VOPP_FIELD_Q, 2, 13, n2 * 13), sub2["Q"][2][0], f"Q2 {path2}")
        assert_close(g.read(V.VOPP_FIELD_RBAR, 2, 1, n2), sub2["rbar"][2], f"rbar2 {path2}")
        assert_close(g.read(V.VOPP_FIELD_LOMEGA, 2, 1, n2), sub2["lomega"][2], f"lom2 {path2}")
        np.testing.assert_array_equal(g.read(V.VOPP_FIELD_PS, 2, 2048, n2 * 2048), sub2["ps"][2][0])
        assert_close(g.read(V.VOPP_FIELD_PLW, 2, 2048, n2 * 2048), sub2["plw"][2][0], "plw2")
        assert_close(g.read(V.VOPP_FIELD_V, 3, AW, n2 * AW), sub2["V"][3], f"V3 below {path2}")
        assert_close(g.read(V.VOPP_FIELD_Q, 3, AW * 13, n2 * AW * 13), sub2["Q"][3].ravel(),
                     f"Q3 below {path2}")
        np.testing.assert_array_equal(g.read(V.VOPP_FIELD_REP, 3, AW, n2 * AW), sub2["rep"][3])
        n4 = AW * AW
        assert_close(g.read(V.VOPP_FIELD_V, 4, n4, n2 * n4), sub2["V"][4], f"V4 below {path2}")
        assert_close(g.read(V.VOPP_FIELD_LOMEGA, 4, n4, n2 * n4), sub2["lomega"][4],
                     f"lom4 below {path2}")
        n5 = AW ** 3
        assert_close(g.read(V.VOPP_FIELD_V, 5, n5, n2 * n5), sub2["V"][5], f"V5 below {path2}")
        assert_close(g.read(V.VOPP_FIELD_RBAR, 5, n5, n2 * n5), sub2["rbar"][5],
                     f"rbar5 below {path2}")
        # root: the FP64 root backup of the level-1 stats (closed form, any size)
        q1 = np.zeros(13)
        rb = g.read(V.VOPP_FIELD_RBAR, 1, AW).astype(np.float64).reshape(13, 3)
        lo = g.read(V.VOPP_FIELD_LOMEGA, 1, AW).astype(np.float64).reshape(13, 3)
        v1 = g.read(V.VOPP_FIELD_V, 1, AW).astype(np.float64).reshape(13, 3)
        for a in range(13):
            om = np.exp(lo[a] - lo[a].max())
            q1[a] = rb[a].mean() + 0.95 * (om @ v1[a]) / om.sum()
        assert_close(res["q"], q1, "root Q from level-1 stats")
        v = 1.0 * np.log(np.mean(np.exp((q1 - q1.max()) / 1.0))) + q1.max()
        assert_close([res["v_root"]], [v], "root V")
        assert res["particle_steps"] == WL.CONFIG3.steps
    finally:
        g.close()


def test_graph_replay_equals_direct_launches():
    """With VOPP_OPT_GRAPHS the launch sequence is captured once per shape and replayed; the
    results equal those of direct launches bit for bit, across seeds and a shape change."""
    from paper_2510_27191_b300 import vopp as V
    spec = Spec(WL.NAV2D, 300, 3, 2, seed=1, pi_mode=WL.PI_NAV_SOFTMAX_DIST)
    spec2 = Spec(WL.GRID, 128, 3, 2, seed=1)
    ctx_a = V.vopp_ctx_create(0, 0, 0)
    ctx_b = V.vopp_ctx_create(0, 0, 0)
    V.vopp_ctx_set_option(ctx_b, V.VOPP_OPT_GRAPHS, 1)
    try:
        ma = V.vopp_create_model(ctx_a, V.make_desc(WL.NAV2D, pi_mode=WL.PI_NAV_SOFTMAX_DIST))
        mb = V.vopp_create_model(ctx_b, V.make_desc(WL.NAV2D, pi_mode=WL.PI_NAV_SOFTMAX_DIST))
        ga = V.vopp_create_model(ctx_a, V.make_desc(WL.GRID, rock_x=spec2.rock_x, rock_y=spec2.rock_y))
        gb = V.vopp_create_model(ctx_b, V.make_desc(WL.GRID, rock_x=spec2.rock_x, rock_y=spec2.rock_y))
        for seed in (1, 2, 3, 4):
            for (m1, m2, s) in ((ma, mb, spec), (ga, gb, spec2)):
                a = V.vopp_plan(m1, s.states(), None, s.N, s.D, s.W, 0.7, 0.95, None, seed)
                b = V.vopp_plan(m2, s.states(), None, s.N, s.D, s.W, 0.7, 0.95, None, seed)
                assert a["q"].tolist() == b["q"].tolist() and a["action"] == b["action"]
        orc = spec.run_oracle(outputs=False)
        b = V.vopp_plan(mb, spec.states(), None, spec.N, spec.D, spec.W, spec.eta, spec.gamma,
                        None, spec.seed)
        assert_close(b["q"], orc["q_root"], "graph-replayed root Q")
        for m in (ma, mb, ga, gb):
            V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx_a)
        V.vopp_ctx_destroy(ctx_b)


def test_autotune_picks_a_configuration_without_changing_results():
    from paper_2510_27191_b300 import vopp as V
    specs = _mixed_specs(12, 9)
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        models = {}
        reqs = []
        for s in specs:
            key = (s.kind, s.branch_mode)
            if key not in models:
                models[key] = V.vopp_create_model(ctx, V.make_desc(
                    s.kind, s.branch_mode, rock_x=WL.grid_layout(1)[0] if s.kind == WL.GRID else None,
                    rock_y=WL.grid_layout(1)[1] if s.kind == WL.GRID else None))
            reqs.append(dict(model=models[key], states=s.states(), weights=None, n=s.N, depth=s.D,
                             width=s.W, eta=s.eta, gamma=s.gamma, seed=s.seed, A=s.A))
        before, k1 = V.vopp_plan_batch(ctx, reqs)
        tune = V.vopp_autotune(ctx, reqs, reps=1)
        assert tune["leaf_threads"] in (64, 128, 256) and len(tune["tried"]) == 6
        after, k2 = V.vopp_plan_batch(ctx, reqs)
        for a, b in zip(before, after):
            assert_close(b["q"], a["q"], "Q after tuning")
        for m in models.values():
            V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_batch_with_crowd_plans_equals_individual_plans_and_oracle():
    """CROWD plans (their own leaf kernel and shared-memory class) batched with the other
    models: every result equals the plan run alone bit for bit and the oracle within the
    tolerance."""
    from paper_2510_27191_b300 import vopp as V
    specs = [Spec(WL.CROWD, 64, 2, 2, eta=0.8, gamma=0.97, seed=31, root_seed=1),
             Spec(WL.NAV2D, 300, 2, 3, eta=0.6, seed=32, root_seed=2),
             Spec(WL.CROWD, 150, 1, 4, eta=1.2, gamma=0.97, seed=33, root_seed=3, weights="random"),
             Spec(WL.GRID, 200, 2, 2, seed=34, root_seed=4),
             Spec(WL.CROWD, 33, 3, 1, eta=0.5, gamma=0.97, seed=35, root_seed=5)]
    ctx = V.vopp_ctx_create(0, 0, 0)
    models = {}
    try:
        reqs = []
        for s in specs:
            if s.kind not in models:
                models[s.kind] = V.vopp_create_model(ctx, V.make_desc(s.kind, rock_x=s.rock_x,
                                                                      rock_y=s.rock_y))
            w = s.root.get("w")
            reqs.append(dict(model=models[s.kind], states=s.states(),
                             weights=None if w is None else np.asarray(w, np.float32), n=s.N,
                             depth=s.D, width=s.W, eta=s.eta, gamma=s.gamma, seed=s.seed, A=s.A))
        outs, keep = V.vopp_plan_batch(ctx, reqs)
        for i, (r, s) in enumerate(zip(reqs, specs)):
            alone = V.vopp_plan(r["model"], r["states"], r["weights"], s.N, s.D, s.W, s.eta,
                                s.gamma, None, s.seed)
            assert outs[i]["q"].tolist() == alone["q"].tolist(), i
            orc = s.run_oracle(outputs=False)
            assert orc["status"] == O.OK
            assert_close(outs[i]["q"], orc["q_root"], f"plan {i} root Q")
            assert action_agrees(outs[i], orc, s)
        del keep
    finally:
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)


def test_config4_mixed_batch_at_full_size_against_oracle():
    """The 512-plan mixed batch of the batching workload (NAV2D and GRID, N log-uniform in
    [128, 4096], depth 3-6, width 2 or 4: 9.2e10 particle-steps) in one vopp_plan_batch call
    with every plan's tree kept: each of its 82 plans of at most 1e7 particle-steps equals the
    oracle node by node (root, every node's Q and V, every branch's statistics, the
    representatives and discrete observations exact), and three of the largest plans equal
    the oracle's subtree below a level-(D-2) node.  The FP64 oracle cannot run the larger
    plans' roots in test time (up to 1e9 particle-steps each)."""
    import concurrent.futures as cf
    import os
    import torch
    from paper_2510_27191_b300 import vopp as V
    specs = WL.draw_mixed_plans(512, 7)
    ctx = V.vopp_ctx_create(0, 0, 0)
    V.vopp_ctx_set_tree_detail(ctx, V.VOPP_TREE_FULL)
    rx, ry = WL.grid_layout(7)
    models = {WL.NAV2D: V.vopp_create_model(ctx, V.make_desc(V.VOPP_NAV2D)),
              WL.GRID: V.vopp_create_model(ctx, V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry))}
    try:
        pspecs = [Spec.from_plan(ps) for ps in specs]
        reqs = [dict(model=models[s.kind], states=torch.from_numpy(s.states()).cuda(),
                     weights=None, n=s.N, depth=s.D, width=s.W, eta=s.eta, gamma=s.gamma,
                     seed=s.seed, A=s.A) for s in pspecs]
        outs, keep = V.vopp_plan_batch(ctx, reqs)
        small = [i for i, ps in enumerate(specs) if ps.steps <= 1e7]
        assert len(small) == 82
        threads = max(1, min(16, len(os.sched_getaffinity(0))))
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            orcs = list(ex.map(lambda i: pspecs[i].run_oracle(dump_levels=max(pspecs[i].D - 2, 0)),
                               small))
        for i, orc in zip(small, orcs):
            s = pspecs[i]
            assert orc["status"] == O.OK
            g = Gpu.__new__(Gpu)           # read plan i's tree through the batch's context
            g.V, g.spec, g.ctx = V, s, ctx
            g.read = (lambda f, l, c, o=0, p=i: V.vopp_tree_read(ctx, f, l, c, o, p))
            compare_full_tree(s, g, outs[i], orc, max(s.D - 2, 0))
            assert action_agrees(outs[i], orc, s), i
            assert outs[i]["particle_steps"] == orc["particle_steps"]
        rng = np.random.default_rng(4)
        for i in sorted(range(len(specs)), key=lambda k: -specs[k].steps)[:3]:
            s = pspecs[i]
            AW = s.A * s.W
            path = tuple(int(v) for v in rng.integers(0, AW, s.D - 2))
            sub = s.run_oracle(path=path)
            assert sub["status"] == O.OK
            n = 0
            for c in path:
                n = n * AW + c
            assert_close(V.vopp_tree_read(ctx, V.VOPP_FIELD_V, s.D - 2, 1, n, i), sub["V"][s.D - 2],
                         f"plan {i} V at {path}")
            assert_close(V.vopp_tree_read(ctx, V.VOPP_FIELD_Q, s.D - 2, s.A, n * s.A, i),
                         sub["Q"][s.D - 2][0], f"plan {i} Q at {path}")
            assert_close(V.vopp_tree_read(ctx, V.VOPP_FIELD_V, s.D - 1, AW, n * AW, i),
                         sub["V"][s.D - 1], f"plan {i} V below {path}")
            assert_close(V.vopp_tree_read(ctx, V.VOPP_FIELD_V, s.D, AW * AW, n * AW * AW, i),
                         sub["V"][s.D], f"plan {i} leaves below {path}")
            np.testing.assert_array_equal(
                V.vopp_tree_read(ctx, V.VOPP_FIELD_REP, s.D, AW * AW, n * AW * AW, i), sub["rep"][s.D])
        del keep
    finally:
        for m in models.values():
            V.vopp_model_destroy(m)
        V.vopp_ctx_destroy(ctx)
