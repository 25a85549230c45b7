"""Helpers shared by the GPU parity tests: run a plan through the C ABI with the whole
tree kept on the device, run the FP64 oracle on the same seeded inputs, compare."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2510_27191_b300 import workloads as WL

# |gpu - oracle| <= RTOL * max(|oracle|, 1): the value tolerance of the FP32 path
# (relative 1e-4, measured in reward units below magnitude 1).
RTOL = 1e-4

KIND_A = {WL.NAV2D: 4, WL.GRID: 13, WL.TOY2: 2, WL.CROWD: 5}


def close(g, o, rtol=RTOL):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    both_inf = np.isneginf(g) & np.isneginf(o)
    with np.errstate(invalid="ignore"):
        err = np.abs(g - o)
    tol = rtol * np.maximum(np.abs(o), 1.0)
    ok = both_inf | (err <= tol)
    return ok


def assert_close(g, o, what, mask=None, rtol=RTOL):
    ok = close(g, o, rtol)
    if mask is not None:
        ok = ok | ~mask
    if not np.all(ok):
        bad = np.flatnonzero(~ok)
        i = bad[0]
        raise AssertionError(f"{what}: {len(bad)} of {ok.size} outside tolerance; first at {i}: "
                             f"gpu={np.ravel(g)[i]!r} oracle={np.ravel(o)[i]!r}")


class Spec:
    def __init__(self, kind, N, D, W, eta=1.0, gamma=0.95, seed=1, pi_mode=WL.PI_UNIFORM,
                 pi_temp=2.0, branch_mode=WL.BRANCH_SAMPLE, layout_seed=1, root_seed=1,
                 weights="uniform", pi_fixed=None, pi_bar=None, h_zero=False, root=None):
        self.kind, self.N, self.D, self.W = kind, N, D, W
        self.eta, self.gamma, self.seed = eta, gamma, seed
        self.pi_mode, self.pi_temp, self.branch_mode = pi_mode, pi_temp, branch_mode
        self.layout_seed, self.root_seed, self.weights = layout_seed, root_seed, weights
        self.pi_fixed, self.pi_bar, self.h_zero = pi_fixed, pi_bar, h_zero
        self.A = KIND_A[kind]
        self.rock_x, self.rock_y = WL.grid_layout(layout_seed) if kind == WL.GRID else (None, None)
        if root is not None:
            self.root = root
        elif kind == WL.NAV2D:
            x, y, w = WL.nav_root(N, root_seed, weights)
            self.root = dict(x=x, y=y, w=w)
        elif kind == WL.GRID:
            s, w = WL.grid_root(N, root_seed, weights)
            self.root = dict(s=s, w=w)
        elif kind == WL.CROWD:
            self.root = WL.crowd_root(N, root_seed, weights=weights)
        else:
            s, w = WL.toy2_root_sampled(N, root_seed)
            self.root = dict(s=s, w=None if weights == "uniform" else w)

    @staticmethod
    def from_plan(ps: WL.PlanSpec, **kw):
        return Spec(ps.kind, ps.N, ps.D, ps.W, eta=ps.eta, gamma=ps.gamma, seed=ps.seed,
                    pi_mode=ps.pi_mode, pi_temp=ps.pi_temp, branch_mode=ps.branch_mode,
                    layout_seed=ps.layout_seed, root_seed=ps.root_seed, **kw)

    def states(self):
        if self.kind == WL.CROWD:
            return WL.pack_crowd_states(self.root)
        if self.kind == WL.NAV2D:
            return np.concatenate([self.root["x"], self.root["y"]]).astype(np.float32)
        return np.asarray(self.root["s"], dtype=np.int32)

    # -- oracle --------------------------------------------------------------------------
    def oracle_model(self):
        return O.make_model(self.kind, branch_mode=self.branch_mode, pi_mode=self.pi_mode,
                            pi_temp=self.pi_temp, pi_fixed=self.pi_bar or self.pi_fixed,
                            rock_x=self.rock_x, rock_y=self.rock_y, h_zero=self.h_zero)

    def run_oracle(self, path=(), dump_levels=-1, outputs=True):
        m = self.oracle_model()
        if self.pi_bar is not None and self.pi_mode == WL.PI_NAV_SOFTMAX_DIST:
            m.pi_mode = O.PI_FIXED
        elif self.pi_bar is not None:
            m.pi_mode = O.PI_FIXED
        w = self.root.get("w")
        w = None if w is None else np.asarray(w, dtype=np.float64)
        if self.kind == WL.NAV2D:
            return O.plan(m, self.N, self.D, self.W, self.eta, self.gamma, self.seed,
                          root_x=self.root["x"], root_y=self.root["y"], root_w=w, path=path,
                          dump_levels=dump_levels, outputs=outputs)
        if self.kind == WL.CROWD:
            return O.plan(m, self.N, self.D, self.W, self.eta, self.gamma, self.seed,
                          root_x=self.root["x"], root_y=self.root["y"], root_s=self.root["s"],
                          root_pf=self.root["pf"], root_w=w, path=path,
                          dump_levels=dump_levels, outputs=outputs)
        return O.plan(m, self.N, self.D, self.W, self.eta, self.gamma, self.seed,
                      root_s=self.root["s"], root_w=w, path=path, dump_levels=dump_levels,
                      outputs=outputs)


class Gpu:
    """One context + model per spec (device 0, default stream)."""

    def __init__(self, spec: Spec, detail=None, leaf_gen=True, leaf_threads=None, ctx=None):
        from paper_2510_27191_b300 import vopp as V
        self.V = V
        self.spec = spec
        self.own_ctx = ctx is None
        self.ctx = ctx if ctx is not None else V.vopp_ctx_create(0, 0, 0)
        V.vopp_ctx_set_tree_detail(self.ctx, V.VOPP_TREE_FULL if detail is None else detail)
        V.vopp_ctx_set_option(self.ctx, V.VOPP_OPT_LEAF_GEN, int(leaf_gen))
        if leaf_threads:
            V.vopp_ctx_set_option(self.ctx, V.VOPP_OPT_LEAF_THREADS, leaf_threads)
        d = V.make_desc(spec.kind, spec.branch_mode, spec.pi_mode, spec.pi_temp, spec.pi_fixed,
                        spec.rock_x, spec.rock_y, spec.h_zero)
        self.model = V.vopp_create_model(self.ctx, d)

    def plan(self, device_inputs=False, seed=None):
        V, s = self.V, self.spec
        st = s.states()
        w = s.root.get("w")
        w = None if w is None else np.asarray(w, dtype=np.float32)
        if device_inputs:
            import torch
            st = torch.from_numpy(st).cuda()
            w = None if w is None else torch.from_numpy(w).cuda()
        return V.vopp_plan(self.model, st, w, s.N, s.D, s.W, s.eta, s.gamma, s.pi_bar,
                           s.seed if seed is None else seed)

    def read(self, field, level, count, offset=0, plan=0):
        return self.V.vopp_tree_read(self.ctx, field, level, count, offset, plan)

    def close(self):
        self.V.vopp_model_destroy(self.model)
        if self.own_ctx:
            self.V.vopp_ctx_destroy(self.ctx)


def exempt_masks(orc, A, W, D):
    """Per level, True where a node lies at or below an oracle near-threshold event."""
    AW = A * W
    masks = [np.zeros(AW ** l, dtype=bool) for l in range(D + 1)]
    for l in range(1, D + 1):
        flagged = orc["near"][l].astype(bool)
        masks[l] |= flagged
        if l < D:
            for m in range(l + 1, D + 1):
                masks[m] |= np.repeat(masks[l], AW ** (m - l))
    return masks


def compare_full_tree(spec: Spec, gpu: Gpu, res: dict, orc: dict, materialised_top: int,
                      check_particles=True):
    """Node-by-node comparison of a whole (small) tree; returns the number of exempt nodes."""
    V = gpu.V
    A, W, D, N = spec.A, spec.W, spec.D, spec.N
    AW = A * W
    ex = exempt_masks(orc, A, W, D)
    keep = [~m for m in ex]
    for l in range(D + 1):
        n = AW ** l
        if l < D:
            assert_close(gpu.read(V.VOPP_FIELD_V, l, n), orc["V"][l], f"V[{l}]", keep[l])
            q = gpu.read(V.VOPP_FIELD_Q, l, n * A).reshape(n, A)
            assert_close(q, orc["Q"][l], f"Q[{l}]", np.repeat(keep[l], A).reshape(n, A))
        else:
            assert_close(gpu.read(V.VOPP_FIELD_V, l, n), orc["V"][l], f"V_leaf[{l}]", keep[l])
        if l >= 1:
            assert_close(gpu.read(V.VOPP_FIELD_RBAR, l, n), orc["rbar"][l], f"rbar[{l}]", keep[l])
            assert_close(gpu.read(V.VOPP_FIELD_LOMEGA, l, n), orc["lomega"][l], f"lomega[{l}]", keep[l])
            rep = gpu.read(V.VOPP_FIELD_REP, l, n)
            np.testing.assert_array_equal(rep, orc["rep"][l], err_msg=f"rep[{l}]")
            obs = gpu.read(V.VOPP_FIELD_OBS, l, 2 * n).reshape(n, 2)
            if spec.kind == WL.NAV2D:
                assert_close(obs, orc["obs"][l], f"obs[{l}]", np.repeat(keep[l], 2).reshape(n, 2))
            else:
                np.testing.assert_array_equal(obs[keep[l]], orc["obs"][l][keep[l]], err_msg=f"obs[{l}]")
    if check_particles:
        for l in range(0, materialised_top + 1):
            n = AW ** l
            kp = np.repeat(keep[l], N).reshape(n, N)
            lw = gpu.read(V.VOPP_FIELD_PLW, l, n * N).reshape(n, N)
            assert_close(lw, orc["plw"][l], f"plw[{l}]", kp)
            if spec.kind in (WL.NAV2D, WL.CROWD):
                px = gpu.read(V.VOPP_FIELD_PX, l, n * N).reshape(n, N)
                py = gpu.read(V.VOPP_FIELD_PY, l, n * N).reshape(n, N)
                assert_close(px, orc["px"][l], f"px[{l}]", kp)
                assert_close(py, orc["py"][l], f"py[{l}]", kp)
            if spec.kind != WL.NAV2D:
                ps = gpu.read(V.VOPP_FIELD_PS, l, n * N).reshape(n, N)
                np.testing.assert_array_equal(ps[kp], orc["ps"][l][kp], err_msg=f"ps[{l}]")
            if spec.kind == WL.CROWD:
                pf = gpu.read(V.VOPP_FIELD_PF, l, n * 12 * N).reshape(n, 12, N)
                assert_close(pf, orc["ppf"][l], f"people[{l}]",
                             np.repeat(kp[:, None, :], 12, axis=1))
    # root
    assert_close(res["q"], orc["q_root"], "root Q")
    assert_close([res["v_root"]], [orc["v_root"]], "root V")
    return int(sum(m.sum() for m in ex))


def action_agrees(res, orc, spec):
    """The chosen action matches whenever the oracle's top-two score gap exceeds the
    tolerance (score = Q + eta log pibar, Alg. 1)."""
    lpi = np.log(np.maximum(orc["policy"], 1e-300)) - (orc["q_root"] - orc["v_root"]) / spec.eta
    score = orc["q_root"] + spec.eta * lpi
    top = np.sort(score)[::-1]
    if len(top) < 2 or top[0] - top[1] > RTOL * max(abs(top[0]), 1.0):
        return res["action"] == orc["action"]
    return res["action"] in np.flatnonzero(score >= top[0] - RTOL * max(abs(top[0]), 1.0))
