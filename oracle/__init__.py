"""FP64 CPU oracle of the VOPP planning hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference
leg may import this package.  The product path (the CUDA library and its Python binding)
never imports, links or runs anything here, and this package imports nothing from it.

The arithmetic lives in ``vopp_oracle.c`` (plain double-precision loops following the
paper's Eq. 1-3 and Algorithms 1-3, plus the SIR belief update of Sec. III-B).  This module
compiles it with gcc on first use and marshals numpy arrays through ctypes.

Parity pins: every function is checked by ``tests/test_oracle_pins.py`` against things
other than itself -- cuRAND's and Triton's Philox4x32-10, a brute-force exact soft
expectimax over exact Bayesian beliefs, the eta -> 0 / eta -> infinity limits of the
log-sum-exp value, the V = Q invariant, hand-checked grid transitions and the
distribution moments of the model noise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vopp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

MAXA = 16
MAXD = 8
NAV2D, GRID, TOY2, CROWD = 0, 1, 2, 3
SAMPLE, ENUMERATE = 0, 1
PI_UNIFORM, PI_FIXED, PI_NAV_DIST = 0, 1, 2
OK, E_INVALID, E_NOMEM, E_DEGENERATE = 0, -1, -2, -6
NUM_ACTIONS = {NAV2D: 4, GRID: 13, TOY2: 2, CROWD: 5}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile vopp_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-Wall",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("branch_mode", ctypes.c_int),
                ("pi_mode", ctypes.c_int), ("h_zero", ctypes.c_int),
                ("pi_temp", ctypes.c_double), ("pi_fixed", ctypes.c_double * MAXA),
                ("rock_x", ctypes.c_int * 8), ("rock_y", ctypes.c_int * 8)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_up = ctypes.POINTER(ctypes.c_uint8)


class PlanArgs(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("D", ctypes.c_int), ("W", ctypes.c_int),
                ("eta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("P", ctypes.c_int),
                ("path", ctypes.c_int * MAXD), ("dump_levels", ctypes.c_int),
                ("V", _dp), ("Q", _dp), ("rbar", _dp), ("lomega", _dp), ("obs", _dp),
                ("rep", _ip), ("near", _up), ("px", _dp), ("py", _dp), ("plw", _dp),
                ("ps", _ip),
                ("action", ctypes.c_int), ("v_root", ctypes.c_double),
                ("q_root", ctypes.c_double * MAXA), ("policy", ctypes.c_double * MAXA),
                ("near_threshold", ctypes.c_longlong), ("degenerate", ctypes.c_longlong),
                ("particle_steps", ctypes.c_longlong),
                ("psi", _dp), ("psi_new_level", ctypes.c_int),
                ("root_pf", _dp), ("ppf", _dp)]


class BuResult(ctypes.Structure):
    _fields_ = [("ess", ctypes.c_double), ("resampled", ctypes.c_int), ("ess_tie", ctypes.c_int),
                ("near_ties", ctypes.c_longlong), ("ties", _up), ("prop_x", _dp), ("prop_y", _dp),
                ("prop_s", _ip), ("pf", _dp)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.orc_philox4x32_10.restype = None
            L.orc_uniform.argtypes = [ctypes.c_uint32]
            L.orc_uniform.restype = ctypes.c_double
            L.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _dp, _dp]
            L.orc_crowd_loglik.argtypes = [ctypes.c_int32, ctypes.c_int]
            L.orc_crowd_loglik.restype = ctypes.c_double
            L.orc_crowd_heuristic.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_double]
            L.orc_crowd_heuristic.restype = ctypes.c_double
            L.orc_grid_acc.argtypes = [ctypes.c_int]
            L.orc_grid_acc.restype = ctypes.c_double
            L.orc_grid_threshold.argtypes = [ctypes.c_int]
            L.orc_grid_threshold.restype = ctypes.c_uint64
            L.orc_level_offsets.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_longlong)]
            L.orc_plan.argtypes = [ctypes.POINTER(Model), _dp, _dp, _ip, _dp,
                                   ctypes.POINTER(PlanArgs)]
            L.orc_plan.restype = ctypes.c_int
            L.orc_belief_update.argtypes = [ctypes.POINTER(Model), ctypes.c_int, _dp, _dp, _ip,
                                            _dp, ctypes.c_int, _dp, ctypes.c_uint64,
                                            ctypes.c_uint64, _ip, ctypes.POINTER(BuResult)]
            L.orc_belief_update.restype = ctypes.c_int
            L.orc_nav_heuristic.argtypes = [ctypes.c_double] * 3
            L.orc_nav_heuristic.restype = ctypes.c_double
            L.orc_grid_step.argtypes = [ctypes.POINTER(Model), ctypes.c_int32, ctypes.c_int, _ip, _dp]
            L.orc_grid_loglik.argtypes = [ctypes.POINTER(Model), ctypes.c_int32, ctypes.c_int,
                                          ctypes.c_int]
            L.orc_grid_loglik.restype = ctypes.c_double
            L.orc_grid_draw_obs.argtypes = [ctypes.POINTER(Model), ctypes.c_int32, ctypes.c_int,
                                            ctypes.c_uint32]
            L.orc_grid_draw_obs.restype = ctypes.c_int
            L.orc_nav_step.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_uint32, ctypes.c_uint32, _dp, _dp, _dp]
            L.orc_nav_loglik.argtypes = [ctypes.c_double] * 4
            L.orc_nav_loglik.restype = ctypes.c_double
            L.orc_belief_value.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double]
            L.orc_belief_value.restype = ctypes.c_double
            _lib = L
    return _lib


def _ptr(a, typ):
    return None if a is None else a.ctypes.data_as(typ)


def make_model(kind: int, branch_mode: int = SAMPLE, pi_mode: int = PI_UNIFORM,
               pi_temp: float = 2.0, pi_fixed=None, rock_x=None, rock_y=None,
               h_zero: bool = False) -> Model:
    m = Model()
    m.kind, m.branch_mode, m.pi_mode, m.h_zero = kind, branch_mode, pi_mode, int(h_zero)
    m.pi_temp = pi_temp
    if pi_fixed is not None:
        for a, v in enumerate(pi_fixed):
            m.pi_fixed[a] = float(v)
    rx = rock_x if rock_x is not None else [-100] * 8
    ry = rock_y if rock_y is not None else [-100] * 8
    for r in range(8):
        m.rock_x[r], m.rock_y[r] = int(rx[r]), int(ry[r])
    return m


def philox(ctr, key):
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(x: int) -> float:
    return lib().orc_uniform(int(x) & 0xFFFFFFFF)


def box_muller(a: int, b: int):
    g1, g2 = ctypes.c_double(), ctypes.c_double()
    lib().orc_box_muller(a, b, ctypes.byref(g1), ctypes.byref(g2))
    return g1.value, g2.value


def grid_threshold(d2: int) -> int:
    return int(lib().orc_grid_threshold(d2))


def grid_acc(d2: int) -> float:
    return lib().orc_grid_acc(d2)


def level_offsets(A: int, W: int, D: int, P: int = 0) -> np.ndarray:
    off = (ctypes.c_longlong * (MAXD + 2))()
    lib().orc_level_offsets(A, W, D, P, off)
    return np.array(off[:D + 2], dtype=np.int64)


def plan(model: Model, N: int, D: int, W: int, eta: float, gamma: float, seed: int,
         root_x=None, root_y=None, root_s=None, root_w=None, path=(), dump_levels: int = -1,
         outputs: bool = True, psi=None, psi_new_level: int = 0, root_pf=None):
    """Run one full-width plan (or the subtree below ``path``) and return a result dict.

    Per-level arrays are returned as lists indexed by level: ``V[l]`` (levels 0..D),
    ``Q[l]`` (levels 0..D-1, shape [n_l, A]), ``rbar/lomega/rep/obs/near[l]`` (levels 1..D,
    indexed by the branch's child node), and the particle dumps ``px/py/plw/ps[l]``.

    CROWD: root_x / root_y are the robot, root_s the flags and ``root_pf`` [12, N] the people
    (rows 2q, 2q+1 = person q's x, y); the dumps add ``ppf`` [nodes, 12, N].

    ``psi`` (float64, updated in place, one row of A preferences per internal node,
    concatenated by level) switches the backup to the persistent preference update of
    Eq. 3; nodes at levels >= ``psi_new_level`` start from eta log pibar.
    """
    A = NUM_ACTIONS[model.kind]
    P = len(path)
    off = level_offsets(A, W, D, P)
    tot = int(off[-1])
    io = PlanArgs()
    io.N, io.D, io.W, io.eta, io.gamma, io.seed, io.P = N, D, W, eta, gamma, seed, P
    for l, s in enumerate(path):
        io.path[l] = int(s)
    io.dump_levels = dump_levels
    if psi is not None:
        assert psi.dtype == np.float64 and psi.flags.c_contiguous and psi.size >= off[D] * A
        io.psi = _ptr(psi, _dp)
        io.psi_new_level = int(psi_new_level)
    arrs = {}
    if outputs:
        arrs = dict(V=np.full(tot, np.nan), Q=np.full(tot * A, np.nan), rbar=np.full(tot, np.nan),
                    lomega=np.full(tot, np.nan), obs=np.full(2 * tot, np.nan),
                    rep=np.full(tot, -2, dtype=np.int32), near=np.zeros(tot, dtype=np.uint8))
        io.V, io.Q = _ptr(arrs["V"], _dp), _ptr(arrs["Q"], _dp)
        io.rbar, io.lomega = _ptr(arrs["rbar"], _dp), _ptr(arrs["lomega"], _dp)
        io.obs, io.rep, io.near = _ptr(arrs["obs"], _dp), _ptr(arrs["rep"], _ip), _ptr(arrs["near"], _up)
    if dump_levels >= 0:
        dtot = int(off[min(dump_levels, D) + 1]) * N
        if model.kind in (NAV2D, CROWD):
            arrs["px"], arrs["py"] = np.zeros(dtot), np.zeros(dtot)
            io.px, io.py = _ptr(arrs["px"], _dp), _ptr(arrs["py"], _dp)
        if model.kind != NAV2D:
            arrs["ps"] = np.zeros(dtot, dtype=np.int32)
            io.ps = _ptr(arrs["ps"], _ip)
        if model.kind == CROWD:
            arrs["ppf"] = np.zeros(dtot * 12)
            io.ppf = _ptr(arrs["ppf"], _dp)
        arrs["plw"] = np.zeros(dtot)
        io.plw = _ptr(arrs["plw"], _dp)
    rx = None if root_x is None else np.ascontiguousarray(root_x, dtype=np.float64)
    ry = None if root_y is None else np.ascontiguousarray(root_y, dtype=np.float64)
    rs = None if root_s is None else np.ascontiguousarray(root_s, dtype=np.int32)
    rw = None if root_w is None else np.ascontiguousarray(root_w, dtype=np.float64)
    rpf = None if root_pf is None else np.ascontiguousarray(root_pf, dtype=np.float64).ravel()
    io.root_pf = _ptr(rpf, _dp)
    rc = lib().orc_plan(ctypes.byref(model), _ptr(rx, _dp), _ptr(ry, _dp), _ptr(rs, _ip),
                        _ptr(rw, _dp), ctypes.byref(io))
    res = dict(status=rc, action=io.action, v_root=io.v_root,
               q_root=np.array(io.q_root[:A]), policy=np.array(io.policy[:A]),
               near_threshold=io.near_threshold, degenerate=io.degenerate,
               particle_steps=io.particle_steps, offsets=off)
    if outputs:
        def split(a, width=1, levels=range(D + 1)):
            return [a[off[l] * width:off[l + 1] * width] for l in levels]
        res["V"] = split(arrs["V"])
        res["Q"] = [q.reshape(-1, A) for q in split(arrs["Q"], A, range(D))]
        for k in ("rbar", "lomega", "rep", "near"):
            res[k] = split(arrs[k])
        res["obs"] = [o.reshape(-1, 2) for o in split(arrs["obs"], 2)]
    if dump_levels >= 0:
        nl = min(dump_levels, D) + 1
        for k in ("px", "py", "ps", "plw"):
            if k in arrs:
                res[k] = [arrs[k][off[l] * N:off[l + 1] * N].reshape(-1, N) for l in range(nl)]
        if "ppf" in arrs:
            res["ppf"] = [arrs["ppf"][off[l] * N * 12:off[l + 1] * N * 12].reshape(-1, 12, N)
                          for l in range(nl)]
    return res


def plan_anytime(model: Model, N: int, K: int, W: int, eta: float, gamma: float, seed: int,
                 root_x=None, root_y=None, root_s=None, root_w=None, outputs: bool = False,
                 root_pf=None):
    """Anytime iterative deepening (Alg. 1 planning loop): iterations k = 1..K each search
    the full-width tree of depth k with the same random numbers and back it up with the
    preference update of Eq. 3 on preferences that persist across iterations (the nodes of
    level k-1 are new in iteration k).  Returns the last iteration's result dict (with the
    per-level arrays of ``plan`` when ``outputs``), the root preferences ``psi_root``, the
    per-iteration root Q values ``q_iters`` and the preferences of every internal node,
    ``psi_levels[l]`` of shape [n_l, A]."""
    A = NUM_ACTIONS[model.kind]
    off = level_offsets(A, W, K, 0)
    psi = np.zeros(int(off[K]) * A)
    q_iters, res = [], None
    for k in range(1, K + 1):
        res = plan(model, N, k, W, eta, gamma, seed, root_x=root_x, root_y=root_y,
                   root_s=root_s, root_w=root_w, outputs=outputs and k == K, psi=psi,
                   psi_new_level=k - 1, root_pf=root_pf)
        if res["status"] != OK:
            return res
        q_iters.append(res["q_root"].copy())
    res["psi_root"] = psi[:A].copy()
    res["q_iters"] = q_iters
    res["psi_levels"] = [psi[off[l] * A:off[l + 1] * A].reshape(-1, A) for l in range(K)]
    return res


class EpisodeArgs(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("K", ctypes.c_int), ("O", ctypes.c_int),
                ("eta", ctypes.c_double), ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("cap", ctypes.c_int), ("root_pf", _dp),
                ("parent_an", _ip), ("depth", _ip),
                ("psi", _dp), ("V", _dp), ("C", _dp), ("Ws", _dp), ("Hs", _dp),
                ("N", ctypes.POINTER(ctypes.c_int64)), ("Nl", ctypes.POINTER(ctypes.c_int64)),
                ("child", _ip),
                ("n_nodes", ctypes.c_int), ("action", ctypes.c_int), ("v_root", ctypes.c_double),
                ("q_root", ctypes.c_double * MAXA), ("policy", ctypes.c_double * MAXA),
                ("particle_steps", ctypes.c_longlong), ("near_decisions", ctypes.c_longlong),
                ("near_threshold", ctypes.c_longlong)]


NUM_OBS = {NAV2D: 0, GRID: 3, TOY2: 2, CROWD: 64}


def plan_episodes(model: Model, M: int, K: int, eta: float, gamma: float, seed: int,
                  root_x=None, root_y=None, root_s=None, root_w=None, cap: int = 0,
                  root_pf=None):
    """Episode mode (Alg. 1-3 as printed): K planning iterations of M sampled episodes, the
    tree grown by first visits, visit-weighted backups of the persistent preferences.
    Returns the root result and the tree arrays (``parent_an``, ``depth``, ``psi``, ``V``,
    ``C``, ``N``, ``Nl``, ``Hs`` trimmed to the node count)."""
    A = NUM_ACTIONS[model.kind]
    O = NUM_OBS[model.kind]
    Np = len(root_x) if root_x is not None else len(root_s)
    cap = cap or M * K * (K + 1) // 2 + 1
    arr = dict(parent_an=np.zeros(cap, np.int32), depth=np.zeros(cap, np.int32),
               psi=np.zeros(cap * A), V=np.zeros(cap), C=np.zeros(cap * A), Ws=np.zeros(cap * A),
               Hs=np.zeros(cap), N=np.zeros(cap * A, np.int64), Nl=np.zeros(cap, np.int64),
               child=np.zeros(max(cap * A * O, 1), np.int32))
    io = EpisodeArgs()
    io.M, io.K, io.O, io.eta, io.gamma, io.seed, io.cap = M, K, O, eta, gamma, seed & (2**64 - 1), cap
    i64 = ctypes.POINTER(ctypes.c_int64)
    io.parent_an, io.depth = _ptr(arr["parent_an"], _ip), _ptr(arr["depth"], _ip)
    io.psi, io.V, io.C = _ptr(arr["psi"], _dp), _ptr(arr["V"], _dp), _ptr(arr["C"], _dp)
    io.Ws, io.Hs = _ptr(arr["Ws"], _dp), _ptr(arr["Hs"], _dp)
    io.N, io.Nl = _ptr(arr["N"], i64), _ptr(arr["Nl"], i64)
    io.child = _ptr(arr["child"], _ip)
    rx = None if root_x is None else np.ascontiguousarray(root_x, dtype=np.float64)
    ry = None if root_y is None else np.ascontiguousarray(root_y, dtype=np.float64)
    rs = None if root_s is None else np.ascontiguousarray(root_s, dtype=np.int32)
    rw = None if root_w is None else np.ascontiguousarray(root_w, dtype=np.float64)
    rpf = None if root_pf is None else np.ascontiguousarray(root_pf, dtype=np.float64).ravel()
    io.root_pf = _ptr(rpf, _dp)
    rc = lib().orc_plan_episodes(ctypes.byref(model), _ptr(rx, _dp), _ptr(ry, _dp),
                                 _ptr(rs, _ip), _ptr(rw, _dp), Np, ctypes.byref(io))
    n = io.n_nodes
    res = dict(status=rc, action=io.action, v_root=io.v_root, q_root=np.array(io.q_root[:A]),
               policy=np.array(io.policy[:A]), n_nodes=n, particle_steps=io.particle_steps,
               near_decisions=io.near_decisions, near_threshold=io.near_threshold)
    for k in ("parent_an", "depth", "V", "Hs", "Nl"):
        res[k] = arr[k][:n].copy()
    for k in ("psi", "C", "N"):
        res[k] = arr[k][:n * A].reshape(n, A).copy()
    res["psi_root"] = res["psi"][0].copy() if n else None
    return res


def env_step(model: Model, state, action: int, seed: int, t: int):
    """One step of the true state (closed loop, Alg. 1): returns (status, next state,
    observation, reward, terminal); state is (x, y) for NAV2D, an int for GRID / TOY2 and
    (x, y, flags, people[12]) for CROWD."""
    pf = None
    if model.kind == NAV2D:
        x, y, s = ctypes.c_double(state[0]), ctypes.c_double(state[1]), ctypes.c_int32(0)
    elif model.kind == CROWD:
        x, y, s = ctypes.c_double(state[0]), ctypes.c_double(state[1]), ctypes.c_int32(int(state[2]))
        pf = np.ascontiguousarray(state[3], dtype=np.float64).copy()
    else:
        x, y, s = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int32(int(state))
    o = (ctypes.c_double * 2)()
    r = ctypes.c_double()
    term = ctypes.c_int()
    rc = lib().orc_env_step(ctypes.byref(model), ctypes.byref(x), ctypes.byref(y),
                            ctypes.byref(s), _ptr(pf, _dp), int(action),
                            ctypes.c_uint64(seed & (2**64 - 1)), ctypes.c_uint64(t), o,
                            ctypes.byref(r), ctypes.byref(term))
    if model.kind == NAV2D:
        nxt = (x.value, y.value)
    elif model.kind == CROWD:
        nxt = (x.value, y.value, s.value, pf)
    else:
        nxt = s.value
    obs = (o[0], o[1]) if model.kind == NAV2D else int(o[0])
    return rc, nxt, obs, r.value, bool(term.value)


def belief_update(model: Model, lw, action: int, obs, seed: int, t: int, x=None, y=None, s=None,
                  pf=None):
    """SIR update in place on float64 copies; returns (status, dict of new arrays).  CROWD:
    x, y the robot, s the flags, pf [12, N] the people."""
    pf = None if pf is None else np.array(pf, dtype=np.float64).reshape(12, -1).copy()
    N = len(lw)
    lw = np.array(lw, dtype=np.float64)
    x = None if x is None else np.array(x, dtype=np.float64)
    y = None if y is None else np.array(y, dtype=np.float64)
    s = None if s is None else np.array(s, dtype=np.int32)
    o = np.zeros(2)
    o[:len(np.atleast_1d(obs))] = np.atleast_1d(obs)
    anc = np.zeros(N, dtype=np.int32)
    ties = np.zeros(N, dtype=np.uint8)
    px = np.zeros(N) if x is not None else None
    py = np.zeros(N) if y is not None else None
    ps = np.zeros(N, dtype=np.int32) if s is not None else None
    r = BuResult()
    r.ties, r.prop_x, r.prop_y, r.prop_s = _ptr(ties, _up), _ptr(px, _dp), _ptr(py, _dp), _ptr(ps, _ip)
    r.pf = _ptr(pf, _dp)
    rc = lib().orc_belief_update(ctypes.byref(model), N, _ptr(x, _dp), _ptr(y, _dp), _ptr(s, _ip),
                                 _ptr(lw, _dp), action, _ptr(o, _dp), seed, t, _ptr(anc, _ip),
                                 ctypes.byref(r))
    return rc, dict(x=x, y=y, s=s, lw=lw, ancestors=anc, ess=r.ess, resampled=bool(r.resampled),
                    ess_tie=bool(r.ess_tie), near_ties=r.near_ties, ties=ties.astype(bool),
                    prop_x=px, prop_y=py, prop_s=ps, pf=pf)


def crowd_loglik(flags: int, obs: int) -> float:
    return lib().orc_crowd_loglik(int(flags), int(obs))


def crowd_heuristic(y: float, flags: int, gamma: float) -> float:
    return lib().orc_crowd_heuristic(float(y), int(flags), float(gamma))


def nav_heuristic(x: float, y: float, gamma: float) -> float:
    return lib().orc_nav_heuristic(x, y, gamma)


def nav_step(x, y, a, wa, wb):
    ox, oy, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_nav_step(x, y, a, wa, wb, ctypes.byref(ox), ctypes.byref(oy), ctypes.byref(r))
    return ox.value, oy.value, r.value


def nav_loglik(sx, sy, ox, oy) -> float:
    return lib().orc_nav_loglik(sx, sy, ox, oy)


def grid_step(model: Model, s: int, a: int):
    out, r = ctypes.c_int32(), ctypes.c_double()
    lib().orc_grid_step(ctypes.byref(model), s, a, ctypes.byref(out), ctypes.byref(r))
    return int(out.value), r.value


def grid_loglik(model: Model, s: int, a: int, obs: int) -> float:
    return lib().orc_grid_loglik(ctypes.byref(model), s, a, obs)


def grid_draw_obs(model: Model, s: int, a: int, w0: int) -> int:
    return lib().orc_grid_draw_obs(ctypes.byref(model), s, a, w0)


def belief_value(q, lpi, eta: float) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    lpi = np.ascontiguousarray(lpi, dtype=np.float64)
    return lib().orc_belief_value(_ptr(q, _dp), _ptr(lpi, _dp), len(q), eta)
