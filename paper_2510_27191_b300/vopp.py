"""Thin ctypes binding of libvopp (include/vopp.h): the same entry points, argument
marshalling only.  Every step of a plan runs in the library's CUDA kernels; this module
never computes any part of the method.  Importing it fails loudly when libvopp.so is
missing; there is no CPU fallback.

PyTorch supplies device memory and streams: pass ``torch.cuda`` tensors (their data_ptr()
becomes a device pointer, VOPP_PTR_DEVICE) and ``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvopp.so")

VOPP_OK, VOPP_E_INVALID, VOPP_E_NOMEM, VOPP_E_BUDGET = 0, -1, -2, -3
VOPP_E_CUDA, VOPP_E_TIMEOUT, VOPP_E_DEGENERATE, VOPP_E_BUSY = -4, -5, -6, -7
VOPP_NAV2D, VOPP_GRID, VOPP_TOY2, VOPP_CROWD = 0, 1, 2, 3
VOPP_BRANCH_SAMPLE, VOPP_BRANCH_ENUMERATE = 0, 1
VOPP_PI_UNIFORM, VOPP_PI_FIXED, VOPP_PI_NAV_DIST = 0, 1, 2
VOPP_PTR_DEVICE = 1
VOPP_FLAG_DEGENERATE_BRANCH, VOPP_FLAG_FP64_ROOT, VOPP_FLAG_REUSED = 1, 2, 4
VOPP_TREE_MINIMAL, VOPP_TREE_FULL = 0, 1
(VOPP_FIELD_V, VOPP_FIELD_Q, VOPP_FIELD_RBAR, VOPP_FIELD_LOMEGA, VOPP_FIELD_REP, VOPP_FIELD_OBS,
 VOPP_FIELD_PX, VOPP_FIELD_PY, VOPP_FIELD_PS, VOPP_FIELD_PLW, VOPP_FIELD_MU,
 VOPP_FIELD_PSI, VOPP_FIELD_PF) = range(13)
VOPP_OPT_LEAF_GEN, VOPP_OPT_LEAF_THREADS, VOPP_OPT_GRID_CAP = 1, 2, 3
VOPP_OPT_PERSISTENT = 5
VOPP_OPT_FP64_ROOT = 6
VOPP_OPT_GRAPHS = 7
VOPP_OPT_REUSE_COPY = 8
VOPP_OPT_SERVER_DIRECT = 9
VOPP_MAX_ACTIONS = 16
NUM_ACTIONS = {VOPP_NAV2D: 4, VOPP_GRID: 13, VOPP_TOY2: 2}

ERRORS = {VOPP_E_INVALID: "VOPP_E_INVALID", VOPP_E_NOMEM: "VOPP_E_NOMEM",
          VOPP_E_BUDGET: "VOPP_E_BUDGET", VOPP_E_CUDA: "VOPP_E_CUDA",
          VOPP_E_TIMEOUT: "VOPP_E_TIMEOUT", VOPP_E_DEGENERATE: "VOPP_E_DEGENERATE",
          VOPP_E_BUSY: "VOPP_E_BUSY"}


class VoppError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class vopp_model_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("branch_mode", ctypes.c_int32),
                ("pi_mode", ctypes.c_int32), ("h_zero", ctypes.c_int32),
                ("pi_temp", ctypes.c_float), ("pi_fixed", ctypes.c_float * VOPP_MAX_ACTIONS),
                ("rock_x", ctypes.c_int32 * 8), ("rock_y", ctypes.c_int32 * 8)]


class vopp_plan_result(ctypes.Structure):
    _fields_ = [("action", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("v_root", ctypes.c_double), ("q", ctypes.c_double * VOPP_MAX_ACTIONS),
                ("policy", ctypes.c_double * VOPP_MAX_ACTIONS),
                ("particle_steps", ctypes.c_uint64), ("nodes", ctypes.c_uint64),
                ("degenerate_actions", ctypes.c_uint32), ("reused_levels", ctypes.c_uint32)]


class vopp_plan_params(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("width", ctypes.c_int32), ("eta", ctypes.c_float),
                ("gamma", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("pi_bar", ctypes.POINTER(ctypes.c_float))]


class vopp_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "completed", "rejected", "batches", "batched_plans", "max_batch_seen",
        "particle_steps", "pending", "in_flight_bytes", "peak_in_flight_bytes")]


class vopp_tune_result(ctypes.Structure):
    _fields_ = [("leaf_threads", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("n_tried", ctypes.c_int32),
                ("tried_threads", ctypes.c_int32 * 8), ("tried_persistent", ctypes.c_int32 * 8),
                ("tried_ms", ctypes.c_double * 8)]


class vopp_pipe_rate(ctypes.Structure):
    _fields_ = [("op", ctypes.c_char * 32), ("thread_ops_per_clock_per_sm", ctypes.c_double),
                ("ops_per_second", ctypes.c_double), ("sms", ctypes.c_int32)]


class vopp_episode_result(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("terminated", ctypes.c_int32),
                ("status", ctypes.c_int32), ("min_depth", ctypes.c_int32),
                ("total_reward", ctypes.c_double), ("discounted_return", ctypes.c_double),
                ("particle_steps", ctypes.c_uint64), ("plan_seconds", ctypes.c_double)]


class vopp_episode_params(ctypes.Structure):
    _fields_ = [("episodes", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("eta", ctypes.c_float), ("gamma", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("max_nodes", ctypes.c_int32)]


(VOPP_EP_PARENT, VOPP_EP_DEPTH, VOPP_EP_PSI, VOPP_EP_V, VOPP_EP_REWARD, VOPP_EP_VISITS) = range(6)


class vopp_plan_request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_void_p), ("root_states", ctypes.c_void_p),
                ("root_weights", ctypes.c_void_p), ("n_particles", ctypes.c_int32),
                ("ptr_flags", ctypes.c_uint32), ("params", vopp_plan_params)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvopp.so not built ({LIB_PATH}); run "
                          "`python -m paper_2510_27191_b300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, u64, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
    sz, fp, dp = ctypes.c_size_t, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
    sig = {
        "vopp_ctx_create": ([ctypes.c_int, sz, ctypes.c_size_t, ctypes.POINTER(vp)], ctypes.c_int),
        "vopp_ctx_destroy": ([vp], None),
        "vopp_ctx_set_tree_detail": ([vp, ctypes.c_int], ctypes.c_int),
        "vopp_ctx_set_option": ([vp, i32, i64], ctypes.c_int),
        "vopp_ctx_set_timing": ([vp, ctypes.c_int], ctypes.c_int),
        "vopp_ctx_kernel_times": ([vp, ctypes.POINTER(ctypes.c_char_p), dp,
                                   ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "vopp_ctx_reset_kernel_times": ([vp], ctypes.c_int),
        "vopp_ctx_counters": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                               ctypes.POINTER(u64)], ctypes.c_int),
        "vopp_plan_footprint": ([vp, i32, i32, i32, ctypes.POINTER(sz)], ctypes.c_int),
        "vopp_create_model": ([vp, ctypes.POINTER(vopp_model_desc), ctypes.POINTER(vp)], ctypes.c_int),
        "vopp_model_destroy": ([vp], None),
        "vopp_model_num_actions": ([vp], ctypes.c_int),
        "vopp_grid_thresholds": ([ctypes.POINTER(u64), i32], ctypes.c_int),
        "vopp_plan": ([vp, vp, vp, i32, i32, i32, ctypes.c_float, ctypes.c_float, fp, u64, u32,
                       ctypes.POINTER(vopp_plan_result)], ctypes.c_int),
        "vopp_plan_submit": ([vp, vp, vp, i32, i32, i32, ctypes.c_float, ctypes.c_float, fp, u64,
                              u32], ctypes.c_int),
        "vopp_plan_finish": ([vp, ctypes.POINTER(vopp_plan_result)], ctypes.c_int),
        "vopp_model_ctx": ([vp], vp),
        "vopp_tree_read": ([vp, i32, i32, u64, u64, vp, u32], ctypes.c_int),
        "vopp_tree_read_plan": ([vp, i32, i32, i32, u64, u64, vp, u32], ctypes.c_int),
        "vopp_agent_create": ([vp, vp, vp, i32, u64, u32, ctypes.POINTER(vp)], ctypes.c_int),
        "vopp_agent_plan": ([vp, ctypes.POINTER(vopp_plan_params),
                             ctypes.POINTER(vopp_plan_result)], ctypes.c_int),
        "vopp_belief_update": ([vp, i32, vp, dp, ctypes.POINTER(i32)], ctypes.c_int),
        "vopp_agent_get_particles": ([vp, vp, vp, vp, u32], ctypes.c_int),
        "vopp_agent_num_particles": ([vp], ctypes.c_int),
        "vopp_agent_destroy": ([vp], None),
        "vopp_belief_update_noalloc": ([vp, vp, vp, i32, i32, vp, u64, u64, ctypes.c_size_t, vp,
                                        dp, ctypes.POINTER(i32)], ctypes.c_int),
        "vopp_plan_batch": ([vp, i32, ctypes.POINTER(vopp_plan_request),
                             ctypes.POINTER(vopp_plan_result)], ctypes.c_int),
        "vopp_server_create": ([vp, i32, i32, ctypes.c_size_t, ctypes.POINTER(vp)], ctypes.c_int),
        "vopp_server_destroy": ([vp], None),
        "vopp_submit": ([vp, ctypes.POINTER(vopp_plan_request), ctypes.POINTER(u64)], ctypes.c_int),
        "vopp_submit_agent": ([vp, vp, ctypes.POINTER(vopp_plan_params), ctypes.POINTER(u64)],
                              ctypes.c_int),
        "vopp_poll": ([vp, u64, ctypes.POINTER(vopp_plan_result), dp], ctypes.c_int),
        "vopp_wait": ([vp, u64, ctypes.c_double, ctypes.POINTER(vopp_plan_result), dp], ctypes.c_int),
        "vopp_server_get_stats": ([vp, ctypes.POINTER(vopp_server_stats)], ctypes.c_int),
        "vopp_server_set_paused": ([vp, ctypes.c_int], ctypes.c_int),
        "vopp_wait_any": ([vp, ctypes.c_double, ctypes.POINTER(u64), ctypes.POINTER(vopp_plan_result),
                           dp], ctypes.c_int),
        "vopp_autotune": ([vp, i32, ctypes.POINTER(vopp_plan_request), i32,
                           ctypes.POINTER(vopp_tune_result)], ctypes.c_int),
        "vopp_last_error": ([], ctypes.c_char_p),
        "vopp_version": ([], ctypes.c_char_p),
        "vopp_pipe_rates": ([ctypes.c_int, vp, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "vopp_plan_anytime": ([vp, vp, vp, i32, ctypes.POINTER(vopp_plan_params), ctypes.c_double,
                               u32, ctypes.POINTER(vopp_plan_result), ctypes.POINTER(i32)],
                              ctypes.c_int),
        "vopp_plan_episodes": ([vp, vp, vp, i32, ctypes.POINTER(vopp_episode_params), ctypes.c_double,
                                u32, ctypes.POINTER(vopp_plan_result), ctypes.POINTER(i32),
                                ctypes.POINTER(i32)], ctypes.c_int),
        "vopp_agent_plan_episodes": ([vp, ctypes.POINTER(vopp_episode_params), ctypes.c_double,
                                      ctypes.POINTER(vopp_plan_result), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32)], ctypes.c_int),
        "vopp_episode_tree_read": ([vp, i32, u64, u64, vp], ctypes.c_int),
        "vopp_env_create": ([vp, vp, u64, ctypes.POINTER(vp)], ctypes.c_int),
        "vopp_env_step": ([vp, i32, vp, fp, ctypes.POINTER(i32)], ctypes.c_int),
        "vopp_env_get_state": ([vp, vp], ctypes.c_int),
        "vopp_env_destroy": ([vp], None),
        "vopp_run_episode": ([vp, vp, ctypes.POINTER(vopp_plan_params), i32, i32, ctypes.c_double,
                              ctypes.POINTER(vopp_episode_result), vp, vp], ctypes.c_int),
        "vopp_agent_plan_anytime": ([vp, ctypes.POINTER(vopp_plan_params), ctypes.c_double,
                                     ctypes.POINTER(vopp_plan_result), ctypes.POINTER(i32)],
                                    ctypes.c_int),
        "vopp_agent_set_reuse": ([vp, i32], ctypes.c_int),
        "vopp_belief_update_batch": ([vp, i32, ctypes.POINTER(vp), ctypes.POINTER(i32),
                                      ctypes.POINTER(vp), dp, ctypes.POINTER(i32),
                                      ctypes.POINTER(i32)], ctypes.c_int),
        "vopp_agent_reuse_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(i32)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def check(rc: int) -> int:
    if rc < 0:
        raise VoppError(rc, lib.vopp_last_error().decode())
    return rc


# ---- the C entry points under their own names (ctypes handles as ints) ------------------
def vopp_ctx_create(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int = 0) -> int:
    h = ctypes.c_void_p()
    check(lib.vopp_ctx_create(device, hbm_budget_bytes, cuda_stream, ctypes.byref(h)))
    return h.value


def vopp_ctx_destroy(ctx: int) -> None:
    lib.vopp_ctx_destroy(ctx)


def vopp_ctx_set_tree_detail(ctx: int, detail: int) -> None:
    check(lib.vopp_ctx_set_tree_detail(ctx, detail))


def vopp_ctx_set_option(ctx: int, option: int, value: int) -> None:
    check(lib.vopp_ctx_set_option(ctx, option, value))


def vopp_ctx_set_timing(ctx: int, enable: bool) -> None:
    check(lib.vopp_ctx_set_timing(ctx, int(enable)))


def vopp_ctx_kernel_times(ctx: int) -> dict:
    n = ctypes.c_int(16)
    names = (ctypes.c_char_p * 16)()
    ms = (ctypes.c_double * 16)()
    cnt = (ctypes.c_uint64 * 16)()
    check(lib.vopp_ctx_kernel_times(ctx, names, ms, cnt, ctypes.byref(n)))
    return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(n.value)}


def vopp_ctx_reset_kernel_times(ctx: int) -> None:
    check(lib.vopp_ctx_reset_kernel_times(ctx))


def vopp_ctx_counters(ctx: int) -> dict:
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    check(lib.vopp_ctx_counters(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return dict(h2d_bytes=a.value, d2h_bytes=b.value, launches=c.value)


def make_desc(kind: int, branch_mode: int = VOPP_BRANCH_SAMPLE, pi_mode: int = VOPP_PI_UNIFORM,
              pi_temp: float = 2.0, pi_fixed=None, rock_x=None, rock_y=None,
              h_zero: bool = False) -> vopp_model_desc:
    d = vopp_model_desc()
    d.kind, d.branch_mode, d.pi_mode, d.h_zero, d.pi_temp = kind, branch_mode, pi_mode, int(h_zero), pi_temp
    if pi_fixed is not None:
        for a, v in enumerate(pi_fixed):
            d.pi_fixed[a] = float(v)
    if rock_x is not None:
        for r in range(8):
            d.rock_x[r], d.rock_y[r] = int(rock_x[r]), int(rock_y[r])
    return d


def vopp_create_model(ctx: int, desc: vopp_model_desc) -> int:
    h = ctypes.c_void_p()
    check(lib.vopp_create_model(ctx, ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def vopp_model_destroy(model: int) -> None:
    lib.vopp_model_destroy(model)


def vopp_model_num_actions(model: int) -> int:
    return check(lib.vopp_model_num_actions(model))


def vopp_grid_thresholds(n: int = 222) -> np.ndarray:
    out = (ctypes.c_uint64 * n)()
    check(lib.vopp_grid_thresholds(out, n))
    return np.array(out[:], dtype=np.uint64)


def vopp_plan_footprint(model: int, n: int, depth: int, width: int) -> int:
    b = ctypes.c_size_t()
    check(lib.vopp_plan_footprint(model, n, depth, width, ctypes.byref(b)))
    return b.value


def _addr(a):
    """(pointer, is_device, keepalive) for a numpy array, torch tensor or None."""
    if a is None:
        return None, False, None
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), bool(a.is_cuda), a
    arr = np.ascontiguousarray(a)
    return arr.ctypes.data, False, arr


def _result_dict(r: vopp_plan_result, A: int) -> dict:
    return dict(action=r.action, flags=r.flags, v_root=r.v_root, q=np.array(r.q[:A]),
                policy=np.array(r.policy[:A]), particle_steps=r.particle_steps, nodes=r.nodes,
                degenerate_actions=r.degenerate_actions, reused_levels=r.reused_levels)


def vopp_plan(model: int, root_states, root_weights, n_particles: int, depth: int, width: int,
              eta: float, gamma: float, pi_bar=None, seed: int = 0, ptr_flags: int | None = None) -> dict:
    """root_states: NAV2D float32[2N] (x then y), GRID/TOY2 int32[N], CROWD the 15-row layout
    (workloads.pack_crowd_states); numpy (host) or torch
    CUDA tensors (device).  Returns the vopp_plan_result as a dict."""
    sp, sdev, keep1 = _addr(root_states)
    wp, wdev, keep2 = _addr(root_weights)
    if ptr_flags is None:
        ptr_flags = VOPP_PTR_DEVICE if sdev else 0
    pib = None
    if pi_bar is not None:
        pib = (ctypes.c_float * len(pi_bar))(*[float(v) for v in pi_bar])
    r = vopp_plan_result()
    check(lib.vopp_plan(model, sp, wp, n_particles, depth, width, eta, gamma,
                        ctypes.cast(pib, ctypes.POINTER(ctypes.c_float)) if pib is not None else None,
                        seed & 0xFFFFFFFFFFFFFFFF, ptr_flags, ctypes.byref(r)))
    del keep1, keep2
    return _result_dict(r, vopp_model_num_actions(model))


_PENDING = {}   # ctx -> (number of actions, buffers kept alive until vopp_plan_finish)


def vopp_plan_submit(model: int, root_states, root_weights, n_particles: int, depth: int,
                     width: int, eta: float, gamma: float, pi_bar=None, seed: int = 0,
                     ptr_flags: int | None = None) -> None:
    """Enqueue a plan on its context's stream (vopp_plan's arguments); collect it with
    vopp_plan_finish(ctx)."""
    sp, sdev, keep1 = _addr(root_states)
    wp, wdev, keep2 = _addr(root_weights)
    if ptr_flags is None:
        ptr_flags = VOPP_PTR_DEVICE if sdev else 0
    pib = None
    if pi_bar is not None:
        pib = (ctypes.c_float * len(pi_bar))(*[float(v) for v in pi_bar])
    check(lib.vopp_plan_submit(model, sp, wp, n_particles, depth, width, eta, gamma,
                               ctypes.cast(pib, ctypes.POINTER(ctypes.c_float)) if pib is not None else None,
                               seed & 0xFFFFFFFFFFFFFFFF, ptr_flags))
    ctx = lib.vopp_model_ctx(model)
    _PENDING[ctx] = (vopp_model_num_actions(model), (root_states, root_weights, keep1, keep2))


def vopp_plan_finish(ctx: int) -> dict:
    """Wait for the context's submitted plan; its vopp_plan_result as a dict."""
    r = vopp_plan_result()
    A, _ = _PENDING.get(ctx, (0, None))
    try:
        check(lib.vopp_plan_finish(ctx, ctypes.byref(r)))
    finally:
        _PENDING.pop(ctx, None)
    return _result_dict(r, A)


def vopp_plan_anytime(model: int, root_states, root_weights, n_particles: int, max_depth: int,
                      width: int, eta: float, gamma: float, seed: int, budget_s: float = 0.0,
                      pi_bar=None) -> dict:
    """Anytime plan (iterative deepening with persistent preferences); the result dict
    carries ``depth_reached``."""
    sp, sdev, k1 = _addr(root_states)
    wp, _, k2 = _addr(root_weights)
    p, k3 = make_params(max_depth, width, eta, gamma, seed, pi_bar)
    r = vopp_plan_result()
    d = ctypes.c_int32()
    check(lib.vopp_plan_anytime(model, sp, wp, n_particles, ctypes.byref(p), float(budget_s),
                                VOPP_PTR_DEVICE if sdev else 0, ctypes.byref(r), ctypes.byref(d)))
    del k1, k2, k3
    out = _result_dict(r, vopp_model_num_actions(model))
    out["depth_reached"] = d.value
    return out


def vopp_agent_plan_anytime(agent: int, model: int, max_depth: int, width: int, eta: float,
                            gamma: float, seed: int, budget_s: float = 0.0, pi_bar=None) -> dict:
    p, keep = make_params(max_depth, width, eta, gamma, seed, pi_bar)
    r = vopp_plan_result()
    d = ctypes.c_int32()
    check(lib.vopp_agent_plan_anytime(agent, ctypes.byref(p), float(budget_s), ctypes.byref(r),
                                      ctypes.byref(d)))
    del keep
    out = _result_dict(r, vopp_model_num_actions(model))
    out["depth_reached"] = d.value
    return out


def vopp_tree_read(ctx: int, field: int, level: int, count: int, offset: int = 0, plan: int = 0,
                   out=None) -> np.ndarray:
    dtype = np.int32 if field in (VOPP_FIELD_REP, VOPP_FIELD_PS) else np.float32
    if out is None:
        out = np.empty(count, dtype=dtype)
    check(lib.vopp_tree_read_plan(ctx, plan, field, level, offset, count, out.ctypes.data, 0))
    return out


def vopp_agent_create(model: int, states, weights, n: int, seed: int) -> int:
    sp, sdev, k1 = _addr(states)
    wp, _, k2 = _addr(weights)
    h = ctypes.c_void_p()
    check(lib.vopp_agent_create(model, sp, wp, n, seed & 0xFFFFFFFFFFFFFFFF,
                                VOPP_PTR_DEVICE if sdev else 0, ctypes.byref(h)))
    del k1, k2
    return h.value


def make_params(depth: int, width: int, eta: float, gamma: float, seed: int, pi_bar=None):
    p = vopp_plan_params()
    p.depth, p.width, p.eta, p.gamma = int(depth), int(width), float(eta), float(gamma)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    keep = None
    if pi_bar is not None:
        keep = (ctypes.c_float * len(pi_bar))(*[float(v) for v in pi_bar])
        p.pi_bar = ctypes.cast(keep, ctypes.POINTER(ctypes.c_float))
    return p, keep


def vopp_agent_plan(agent: int, model: int, depth: int, width: int, eta: float, gamma: float,
                    seed: int, pi_bar=None) -> dict:
    p, keep = make_params(depth, width, eta, gamma, seed, pi_bar)
    r = vopp_plan_result()
    check(lib.vopp_agent_plan(agent, ctypes.byref(p), ctypes.byref(r)))
    del keep
    return _result_dict(r, vopp_model_num_actions(model))


def vopp_belief_update(agent: int, action: int, obs, kind: int):
    if kind == VOPP_NAV2D:
        o = (ctypes.c_float * 2)(float(obs[0]), float(obs[1]))
    else:
        o = (ctypes.c_int32 * 1)(int(np.atleast_1d(obs)[0]))
    ess = ctypes.c_double()
    res = ctypes.c_int32()
    check(lib.vopp_belief_update(agent, action, o, ctypes.byref(ess), ctypes.byref(res)))
    return ess.value, bool(res.value)


def _state_words(kind: int) -> int:
    return {VOPP_NAV2D: 2, VOPP_CROWD: 15}.get(kind, 1)


def vopp_belief_update_batch(ctx: int, agents, actions, obs, kinds):
    """Update agents[i] with (actions[i], obs[i]) for every i in one call (kinds[i]: the
    agent's model kind, which fixes the observation's type).  Returns (status, ess,
    resampled) arrays; a failing update shows in its status, not as an exception."""
    n = len(agents)
    keep = []
    ptrs = (ctypes.c_void_p * n)()
    for i, (o, k) in enumerate(zip(obs, kinds)):
        if k == VOPP_NAV2D:
            b = (ctypes.c_float * 2)(float(o[0]), float(o[1]))
        else:
            b = (ctypes.c_int32 * 1)(int(np.atleast_1d(o)[0]))
        keep.append(b)
        ptrs[i] = ctypes.cast(b, ctypes.c_void_p)
    ags = (ctypes.c_void_p * n)(*agents)
    acts = (ctypes.c_int32 * n)(*[int(a) for a in actions])
    ess = np.zeros(n, dtype=np.float64)
    res = np.zeros(n, dtype=np.int32)
    st = np.zeros(n, dtype=np.int32)
    rc = lib.vopp_belief_update_batch(ctx, n, ags, acts, ptrs,
                                      ess.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      res.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc not in (VOPP_OK, VOPP_E_DEGENERATE):
        check(rc)
    del keep
    return st, ess, res.astype(bool)


def vopp_agent_set_reuse(agent: int, enable: int = 1) -> None:
    """enable: 0 off, 1 (or True) on for discrete-observation models (NAV2D keeps nothing),
    2 on for every model."""
    check(lib.vopp_agent_set_reuse(agent, int(enable)))


def vopp_agent_reuse_info(agent: int) -> dict:
    """adopted_slot (a*W + k, or -1 after an SIR update), kept_levels, key_level."""
    a, k, lv = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(lib.vopp_agent_reuse_info(agent, ctypes.byref(a), ctypes.byref(k), ctypes.byref(lv)))
    return dict(adopted_slot=a.value, kept_levels=k.value, key_level=lv.value)


def vopp_agent_get_particles(agent: int, kind: int):
    """(states, log weights, ancestors of the last update); states in the root layout
    (NAV2D float32 [2N]; GRID / TOY2 int32 [N]; CROWD float32 [15N], the last row int32
    flags)."""
    n = check(lib.vopp_agent_num_particles(agent))
    st = (np.empty(_state_words(kind) * n, dtype=np.float32) if kind in (VOPP_NAV2D, VOPP_CROWD)
          else np.empty(n, dtype=np.int32))
    lw = np.empty(n, dtype=np.float32)
    anc = np.empty(n, dtype=np.int32)
    check(lib.vopp_agent_get_particles(agent, st.ctypes.data, lw.ctypes.data, anc.ctypes.data, 0))
    return st, lw, anc


def vopp_belief_update_noalloc(model: int, states, log_weights, action: int, obs, seed: int,
                               t: int, kind: int, cuda_stream: int = 0, ancestors=None):
    """In-place SIR update of caller-owned CUDA tensors (states, log_weights) using the
    library's static scratch; returns (ess, resampled).

    The kernel writes every one of n = log_weights.numel() particles, so the tensors are
    checked here first (the C entry point sees only pointers): contiguous CUDA tensors on
    one device, log_weights float32, states of 4-byte elements holding exactly the model's
    words per particle times n, ancestors int32 with at least n entries."""
    import torch
    words = {VOPP_NAV2D: 2, VOPP_CROWD: 15}.get(kind, 1)
    n = log_weights.numel()
    tensors = [("states", states), ("log_weights", log_weights)]
    if ancestors is not None:
        tensors.append(("ancestors", ancestors))
    for name, ten in tensors:
        if not isinstance(ten, torch.Tensor) or not ten.is_cuda or not ten.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if ten.device != log_weights.device:
            raise ValueError(f"{name} is on {ten.device}, log_weights on {log_weights.device}")
    if log_weights.dtype != torch.float32:
        raise ValueError("log_weights must be float32")
    if states.element_size() != 4 or states.numel() != words * n:
        raise ValueError(f"states must hold {words} 4-byte words per particle ({words * n}), "
                         f"got {states.numel()} of {states.element_size()} bytes")
    if ancestors is not None and (ancestors.dtype != torch.int32 or ancestors.numel() < n):
        raise ValueError(f"ancestors must be int32 with at least {n} entries")
    if kind == VOPP_NAV2D:
        o = (ctypes.c_float * 2)(float(obs[0]), float(obs[1]))
    else:
        o = (ctypes.c_int32 * 1)(int(np.atleast_1d(obs)[0]))
    ess = ctypes.c_double()
    res = ctypes.c_int32()
    check(lib.vopp_belief_update_noalloc(model, states.data_ptr(), log_weights.data_ptr(), n,
                                         action, o, seed & 0xFFFFFFFFFFFFFFFF, t, cuda_stream,
                                         None if ancestors is None else ancestors.data_ptr(),
                                         ctypes.byref(ess), ctypes.byref(res)))
    return ess.value, bool(res.value)


# ---- episode mode ------------------------------------------------------------------------
def _episode_params(episodes, max_depth, eta, gamma, seed, max_nodes=0):
    p = vopp_episode_params()
    p.episodes, p.max_depth, p.eta, p.gamma = int(episodes), int(max_depth), float(eta), float(gamma)
    p.seed, p.max_nodes = int(seed) & 0xFFFFFFFFFFFFFFFF, int(max_nodes)
    return p


def vopp_plan_episodes(model: int, root_states, root_weights, n_particles: int, episodes: int,
                       max_depth: int, eta: float, gamma: float, seed: int,
                       budget_s: float = 0.0, max_nodes: int = 0) -> dict:
    """Episode mode; the result dict carries ``depth_reached`` and ``n_nodes``."""
    sp, sdev, k1 = _addr(root_states)
    wp, _, k2 = _addr(root_weights)
    p = _episode_params(episodes, max_depth, eta, gamma, seed, max_nodes)
    r = vopp_plan_result()
    d, n = ctypes.c_int32(), ctypes.c_int32()
    check(lib.vopp_plan_episodes(model, sp, wp, n_particles, ctypes.byref(p), float(budget_s),
                                 VOPP_PTR_DEVICE if sdev else 0, ctypes.byref(r), ctypes.byref(d),
                                 ctypes.byref(n)))
    del k1, k2
    out = _result_dict(r, vopp_model_num_actions(model))
    out["depth_reached"], out["n_nodes"] = d.value, n.value
    return out


def vopp_agent_plan_episodes(agent: int, model: int, episodes: int, max_depth: int, eta: float,
                             gamma: float, seed: int, budget_s: float = 0.0) -> dict:
    p = _episode_params(episodes, max_depth, eta, gamma, seed)
    r = vopp_plan_result()
    d, n = ctypes.c_int32(), ctypes.c_int32()
    check(lib.vopp_agent_plan_episodes(agent, ctypes.byref(p), float(budget_s), ctypes.byref(r),
                                       ctypes.byref(d), ctypes.byref(n)))
    out = _result_dict(r, vopp_model_num_actions(model))
    out["depth_reached"], out["n_nodes"] = d.value, n.value
    return out


def vopp_episode_tree_read(ctx: int, field: int, count: int, offset: int = 0) -> np.ndarray:
    dtype = {VOPP_EP_PARENT: np.int32, VOPP_EP_DEPTH: np.int32,
             VOPP_EP_VISITS: np.uint64}.get(field, np.float64)
    out = np.empty(count, dtype=dtype)
    check(lib.vopp_episode_tree_read(ctx, field, offset, count, out.ctypes.data))
    return out


# ---- closed loop -------------------------------------------------------------------------
def _env_state(state, kind):
    if kind == VOPP_NAV2D:
        return np.asarray(state, dtype=np.float32).reshape(2)
    if kind == VOPP_CROWD:   # (x, y, flags, people[12])
        st = np.empty(15, dtype=np.float32)
        st[0], st[1] = state[0], state[1]
        st[2:14] = np.asarray(state[3], dtype=np.float32).reshape(12)
        st[14:15] = np.asarray([int(state[2])], dtype=np.int32).view(np.float32)
        return st
    return np.asarray([int(state)], dtype=np.int32)


def vopp_env_create(model: int, state, seed: int, kind: int) -> int:
    """state: (x, y) for NAV2D, an int for GRID / TOY2, (x, y, flags, people[12]) for CROWD
    (kind: the model's kind)."""
    st = _env_state(state, kind)
    h = ctypes.c_void_p()
    check(lib.vopp_env_create(model, st.ctypes.data, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(h)))
    return h.value


def vopp_env_step(env: int, action: int, kind: int):
    """(observation, reward, terminal) of one step; observation (x, y) or an int."""
    o = np.zeros(2, dtype=np.float32) if kind == VOPP_NAV2D else np.zeros(1, dtype=np.int32)
    r = ctypes.c_float()
    t = ctypes.c_int32()
    check(lib.vopp_env_step(env, int(action), o.ctypes.data, ctypes.byref(r), ctypes.byref(t)))
    obs = (float(o[0]), float(o[1])) if kind == VOPP_NAV2D else int(o[0])
    return obs, r.value, bool(t.value)


def vopp_env_get_state(env: int, kind: int):
    o = np.zeros(_state_words(kind), dtype=np.float32 if kind != VOPP_GRID and kind != VOPP_TOY2
                 else np.int32)
    check(lib.vopp_env_get_state(env, o.ctypes.data))
    if kind == VOPP_NAV2D:
        return (float(o[0]), float(o[1]))
    if kind == VOPP_CROWD:
        return (float(o[0]), float(o[1]), int(o[14:15].view(np.int32)[0]), o[2:14].copy())
    return int(o[0])


def vopp_env_destroy(env: int) -> None:
    lib.vopp_env_destroy(env)


def vopp_run_episode(agent: int, env: int, depth: int, width: int, eta: float, gamma: float,
                     seed: int, max_steps: int, anytime: bool = False, budget_s: float = 0.0):
    """Closed loop: (result dict, actions, rewards); the dict carries the status instead of
    raising when an error ends the episode early."""
    p, keep = make_params(depth, width, eta, gamma, seed)
    r = vopp_episode_result()
    acts = np.full(max_steps, -1, dtype=np.int32)
    rews = np.zeros(max_steps, dtype=np.float32)
    rc = lib.vopp_run_episode(agent, env, ctypes.byref(p), int(max_steps), int(bool(anytime)),
                              float(budget_s), ctypes.byref(r), acts.ctypes.data, rews.ctypes.data)
    del keep
    res = {n: getattr(r, n) for n, _ in vopp_episode_result._fields_}
    res["rc"] = rc
    return res, acts[:r.steps], rews[:r.steps]


def vopp_agent_destroy(agent: int) -> None:
    lib.vopp_agent_destroy(agent)


def vopp_plan_batch(ctx: int, requests: list) -> tuple[list, list]:
    """requests: dicts with model, states, weights, n, depth, width, eta, gamma, seed, pi_bar,
    A.  Returns (results, keepalive)."""
    n = len(requests)
    reqs = (vopp_plan_request * n)()
    keep = []
    for i, q in enumerate(requests):
        sp, sdev, k1 = _addr(q["states"])
        wp, _, k2 = _addr(q.get("weights"))
        keep += [k1, k2]
        p, k3 = make_params(q["depth"], q["width"], q["eta"], q["gamma"], q["seed"], q.get("pi_bar"))
        keep.append(k3)
        reqs[i].model = q["model"]
        reqs[i].root_states = sp
        reqs[i].root_weights = wp
        reqs[i].n_particles = q["n"]
        reqs[i].ptr_flags = VOPP_PTR_DEVICE if sdev else 0
        reqs[i].params = p
    outs = (vopp_plan_result * n)()
    check(lib.vopp_plan_batch(ctx, n, reqs, outs))
    return [_result_dict(outs[i], requests[i]["A"]) for i in range(n)], keep


def vopp_version() -> str:
    return lib.vopp_version().decode()


def vopp_pipe_rates(device: int = 0) -> dict:
    """Issue-rate microbenchmark: {op: (thread ops per SM cycle, ops per second)}."""
    out = (vopp_pipe_rate * 16)()
    n = ctypes.c_int32()
    check(lib.vopp_pipe_rates(device, out, 16, ctypes.byref(n)))
    return {out[i].op.decode(): (out[i].thread_ops_per_clock_per_sm, out[i].ops_per_second)
            for i in range(n.value)}


# ---- serving ---------------------------------------------------------------------------
def vopp_server_create(ctx: int, max_batch: int = 64, n_slots: int = 2, hbm_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    check(lib.vopp_server_create(ctx, max_batch, n_slots, hbm_budget_bytes, ctypes.byref(h)))
    return h.value


def vopp_server_destroy(srv: int) -> None:
    lib.vopp_server_destroy(srv)


def vopp_submit_agent(srv: int, agent: int, depth: int, width: int, eta: float, gamma: float,
                      seed: int, pi_bar=None) -> int:
    p, keep = make_params(depth, width, eta, gamma, seed, pi_bar)
    t = ctypes.c_uint64()
    check(lib.vopp_submit_agent(srv, agent, ctypes.byref(p), ctypes.byref(t)))
    del keep
    return t.value


def vopp_submit(srv: int, model: int, states, weights, n: int, depth: int, width: int, eta: float,
                gamma: float, seed: int, pi_bar=None) -> int:
    """Queue one plan; host (numpy) inputs are copied at submission, CUDA tensors must stay
    alive until the ticket completes."""
    sp, sdev, k1 = _addr(states)
    wp, _, k2 = _addr(weights)
    p, k3 = make_params(depth, width, eta, gamma, seed, pi_bar)
    r = vopp_plan_request()
    r.model, r.root_states, r.root_weights, r.n_particles = model, sp, wp, n
    r.ptr_flags = VOPP_PTR_DEVICE if sdev else 0
    r.params = p
    t = ctypes.c_uint64()
    check(lib.vopp_submit(srv, ctypes.byref(r), ctypes.byref(t)))
    del k1, k2, k3
    return t.value


def vopp_poll(srv: int, ticket: int, A: int):
    """None while busy; else (result dict, latency seconds)."""
    r = vopp_plan_result()
    lat = ctypes.c_double()
    rc = lib.vopp_poll(srv, ticket, ctypes.byref(r), ctypes.byref(lat))
    if rc == VOPP_E_BUSY:
        return None
    check(rc)
    return _result_dict(r, A), lat.value


def vopp_wait(srv: int, ticket: int, A: int, timeout_s: float = 10.0):
    r = vopp_plan_result()
    lat = ctypes.c_double()
    check(lib.vopp_wait(srv, ticket, timeout_s, ctypes.byref(r), ctypes.byref(lat)))
    return _result_dict(r, A), lat.value


def vopp_server_get_stats(srv: int) -> dict:
    st = vopp_server_stats()
    check(lib.vopp_server_get_stats(srv, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in vopp_server_stats._fields_}


def vopp_wait_any(srv: int, timeout_s: float = 0.0):
    """(ticket, status, result-or-None, latency) of the next finished plan, or None when none
    finished within timeout_s."""
    t = ctypes.c_uint64()
    r = vopp_plan_result()
    lat = ctypes.c_double()
    rc = lib.vopp_wait_any(srv, timeout_s, ctypes.byref(t), ctypes.byref(r), ctypes.byref(lat))
    if rc == VOPP_E_TIMEOUT:
        return None
    return t.value, rc, (_result_dict(r, VOPP_MAX_ACTIONS) if rc == VOPP_OK else None), lat.value


def vopp_server_set_paused(srv: int, paused: bool) -> None:
    check(lib.vopp_server_set_paused(srv, int(paused)))


def _requests(requests):
    n = len(requests)
    reqs = (vopp_plan_request * n)()
    keep = []
    for i, q in enumerate(requests):
        sp, sdev, k1 = _addr(q["states"])
        wp, _, k2 = _addr(q.get("weights"))
        p, k3 = make_params(q["depth"], q["width"], q["eta"], q["gamma"], q["seed"], q.get("pi_bar"))
        keep += [k1, k2, k3]
        reqs[i].model, reqs[i].root_states, reqs[i].root_weights = q["model"], sp, wp
        reqs[i].n_particles = q["n"]
        reqs[i].ptr_flags = VOPP_PTR_DEVICE if sdev else 0
        reqs[i].params = p
    return reqs, keep


def vopp_autotune(ctx: int, requests: list, reps: int = 2) -> dict:
    reqs, keep = _requests(requests)
    out = vopp_tune_result()
    check(lib.vopp_autotune(ctx, len(requests), reqs, reps, ctypes.byref(out)))
    del keep
    return dict(leaf_threads=out.leaf_threads, persistent=out.persistent, best_ms=out.best_ms,
                tried=[(out.tried_threads[i], out.tried_persistent[i], out.tried_ms[i])
                       for i in range(out.n_tried)])

