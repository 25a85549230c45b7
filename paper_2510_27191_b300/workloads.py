"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This module holds input generation only: root particle sets, grid layouts, per-plan size
draws.  It contains none of the planner's arithmetic (no transition, likelihood, reward,
heuristic or backup), so the oracle and the CUDA path can both consume its output without
sharing any of the method.

The workloads stand in for the paper's benchmark problems (Sec. IV: MARS, Navigation,
CrowdNav), whose maps and code are not available: a continuous 2-D navigation problem
(NAV2D), a RockSample-like discrete grid-sensing problem (GRID), a two-state test
problem (TOY2) and a crowd-navigation problem shaped like the paper's CrowdNav (CROWD).  All numbers come from numpy's PCG64 generator seeded explicitly.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NAV2D, GRID, TOY2, CROWD = 0, 1, 2, 3
KIND_NAMES = {NAV2D: "nav2d", GRID: "grid", TOY2: "toy2", CROWD: "crowd"}
NUM_ACTIONS = {NAV2D: 4, GRID: 13, TOY2: 2, CROWD: 5}
CROWD_PEOPLE = 6

BRANCH_SAMPLE, BRANCH_ENUMERATE = 0, 1
PI_UNIFORM, PI_FIXED, PI_NAV_SOFTMAX_DIST = 0, 1, 2

GRID_SIZE = 11
GRID_ROCKS = 8
GRID_START = (0, 5)


def pack_grid_state(rock_bits: np.ndarray, x: int, y: int, terminal: bool = False) -> np.ndarray:
    """Packed int32 grid state: bits 0-7 rock bits, 8-11 x (11 = exited), 12-15 y, 16 terminal."""
    rb = np.asarray(rock_bits, dtype=np.int64) & 0xFF
    s = rb | (int(x) << 8) | (int(y) << 12) | ((1 << 16) if terminal else 0)
    return s.astype(np.int32)


def grid_layout(layout_seed: int) -> tuple[list[int], list[int]]:
    """Eight distinct rock cells on the 11x11 grid, excluding the start cell (0, 5)."""
    rng = np.random.default_rng(np.random.SeedSequence([layout_seed, 0x6C61796F]))
    cells = [c for c in range(GRID_SIZE * GRID_SIZE)
             if (c % GRID_SIZE, c // GRID_SIZE) != GRID_START]
    pick = rng.choice(len(cells), size=GRID_ROCKS, replace=False)
    xs = [cells[i] % GRID_SIZE for i in pick]
    ys = [cells[i] // GRID_SIZE for i in pick]
    return xs, ys


def nav_root(n: int, seed: int, weights: str = "uniform"):
    """Root belief for NAV2D: n particles uniform in [0,10]^2 (float32 SoA x, y) + weights."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x6E6176]))
    x = rng.uniform(0.0, 10.0, size=n).astype(np.float32)
    y = rng.uniform(0.0, 10.0, size=n).astype(np.float32)
    return x, y, _weights(rng, n, weights)


def grid_root(n: int, seed: int, weights: str = "uniform"):
    """Root belief for GRID: agent at (0,5), rock bits i.i.d. Bernoulli(1/2) per particle."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x67726964]))
    bits = rng.integers(0, 256, size=n)
    s = pack_grid_state(bits, GRID_START[0], GRID_START[1])
    return s, _weights(rng, n, weights)


def toy2_root(b0=(0.6, 0.4)):
    """Root belief for TOY2: the two states, weighted by the prior b0."""
    s = np.array([0, 1], dtype=np.int32)
    w = np.array(b0, dtype=np.float32)
    return s, w


def toy2_root_sampled(n: int, seed: int, b0=(0.6, 0.4)):
    """TOY2 root with n equally weighted particles drawn from b0."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x746F79]))
    s = (rng.uniform(size=n) >= b0[0]).astype(np.int32)
    return s, np.full(n, 1.0 / n, dtype=np.float32)


def crowd_root(n: int, seed: int, p_curious: float = 0.5, weights: str = "uniform",
               robot=(25.0, 0.5)):
    """Root belief for CROWD: the robot on the southern border, the six nearest people at
    positions known to every particle (drawn within 8 m ahead of the robot), and per particle
    each person's hidden trait, curious with probability p_curious.  Returns dict(x, y, s,
    pf, w): robot x, y [N], flags s [N] (bits 0-5 traits), people pf [12, N] (rows 2q, 2q+1
    = person q's x, y), weights."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x63726F77]))
    px = np.clip(robot[0] + rng.uniform(-6.0, 6.0, size=CROWD_PEOPLE), 0.0, 50.0)
    py = np.clip(robot[1] + rng.uniform(0.5, 8.0, size=CROWD_PEOPLE), 0.0, 40.0)
    traits = (rng.uniform(size=(n, CROWD_PEOPLE)) < p_curious).astype(np.int64)
    s = (traits << np.arange(CROWD_PEOPLE)).sum(axis=1).astype(np.int32)
    pf = np.empty((2 * CROWD_PEOPLE, n), dtype=np.float32)
    pf[0::2] = px.astype(np.float32)[:, None]
    pf[1::2] = py.astype(np.float32)[:, None]
    x = np.full(n, robot[0], dtype=np.float32)
    y = np.full(n, robot[1], dtype=np.float32)
    return dict(x=x, y=y, s=s, pf=pf, w=_weights(rng, n, weights))


def pack_crowd_states(root: dict) -> np.ndarray:
    """The C ABI's CROWD root layout: 15 rows of N 32-bit words -- robot x, robot y, the 12
    people coordinates (float32), then the int32 flags."""
    n = len(root["x"])
    out = np.empty((15, n), dtype=np.float32)
    out[0], out[1], out[2:14] = root["x"], root["y"], root["pf"]
    out[14] = np.asarray(root["s"], dtype=np.int32).view(np.float32)
    return out.ravel()


def _weights(rng, n, kind):
    if kind == "uniform":
        return None
    if kind == "random":
        return rng.uniform(0.05, 1.0, size=n).astype(np.float32)
    if kind == "sparse":
        w = rng.uniform(0.05, 1.0, size=n).astype(np.float32)
        w[rng.uniform(size=n) < 0.5] = 0.0
        if not np.any(w > 0):
            w[0] = 1.0
        return w
    raise ValueError(kind)


def particle_steps(A: int, W: int, N: int, D: int) -> int:
    """Counting rule: one generative-model evaluation per particle per child node."""
    return sum((A * W) ** l for l in range(1, D + 1)) * N


@dataclasses.dataclass
class PlanSpec:
    kind: int
    N: int
    D: int
    W: int
    eta: float
    gamma: float
    seed: int
    pi_mode: int = PI_UNIFORM
    pi_temp: float = 2.0
    branch_mode: int = BRANCH_SAMPLE
    layout_seed: int = 0
    root_seed: int = 0

    @property
    def A(self) -> int:
        return NUM_ACTIONS[self.kind]

    @property
    def steps(self) -> int:
        return particle_steps(self.A, self.W, self.N, self.D)


# The five workloads: small plain plan, single large plan, bit-exact grid plan,
# a batch of mixed plans and a served request stream.
CONFIG1 = PlanSpec(kind=NAV2D, N=256, D=3, W=4, eta=1.0, gamma=0.95, seed=1, root_seed=1)
CONFIG2 = PlanSpec(kind=NAV2D, N=1024, D=4, W=4, eta=0.5, gamma=0.95, seed=1,
                   pi_mode=PI_NAV_SOFTMAX_DIST, pi_temp=2.0, root_seed=1)
CONFIG3 = PlanSpec(kind=GRID, N=2048, D=5, W=3, eta=1.0, gamma=0.95, seed=1, layout_seed=1,
                   root_seed=1)

BATCH_CAP_STEPS = 1 << 30     # per-plan work cap for the batched workload
SERVE_CAP_STEPS = 1 << 26     # per-plan work cap for the served workload (50 ms deadline)


def draw_mixed_plans(n_plans: int, seed: int, cap_steps: int = BATCH_CAP_STEPS) -> list[PlanSpec]:
    """Mixed batch: model 1/2 NAV2D 1/2 GRID, N ~ logU[128,4096], D ~ U{3..6}, W ~ {2,4}.

    After drawing, D is lowered until the plan's particle-step count is within cap_steps.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x6D6978]))
    out = []
    for i in range(n_plans):
        kind = NAV2D if rng.uniform() < 0.5 else GRID
        N = int(round(math.exp(rng.uniform(math.log(128), math.log(4096)))))
        D = int(rng.integers(3, 7))
        W = 2 if rng.uniform() < 0.5 else 4
        A = NUM_ACTIONS[kind]
        while D > 1 and particle_steps(A, W, N, D) > cap_steps:
            D -= 1
        out.append(PlanSpec(kind=kind, N=N, D=D, W=W, eta=1.0, gamma=0.95,
                            seed=int(rng.integers(1, 2**62)), layout_seed=int(seed),
                            root_seed=int(rng.integers(1, 2**31))))
    return out
