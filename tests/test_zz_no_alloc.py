"""The allocation-free belief update against the regular one (needs a GPU).

vopp_belief_update_noalloc serves callers that cannot allocate device memory when they
update a belief; it keeps its working memory in a static device array instead.  It must
give the same particles, weights and ancestors as vopp_belief_update (the agent path, which
allocates its scratch at agent creation) on two updates in a row, within the value
tolerance of the parity tests (|a - b| <= 1e-4 max(|b|, 1); integers exact).  This file is
collected last so that a failure here cannot hide any other test's result.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2510_27191_b300 import workloads as WL

pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _close(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both = np.isneginf(a) & np.isneginf(b)
    with np.errstate(invalid="ignore"):
        ok = both | (np.abs(a - b) <= RTOL * np.maximum(np.abs(b), 1.0))
    return bool(np.all(ok))


@pytest.mark.parametrize("kind", [WL.NAV2D, WL.GRID])
def test_noalloc_update_matches_agent_update_twice(kind):
    import torch
    from paper_2510_27191_b300 import vopp as V
    N, seed = 3000, 77
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        if kind == WL.NAV2D:
            desc = V.make_desc(V.VOPP_NAV2D)
            x, y, _ = WL.nav_root(N, 5)
            x = (9.0 + 0.5 * (x / 10.0)).astype(np.float32)   # near x = 9: informative sensor
            host_states = np.concatenate([x, y]).astype(np.float32)
            steps = [(1, (8.9, 4.0)), (2, (8.2, 5.1))]
        else:
            rx, ry = WL.grid_layout(3)
            desc = V.make_desc(V.VOPP_GRID, rock_x=rx, rock_y=ry)
            s, _ = WL.grid_root(N, 5)
            host_states = np.asarray(s, dtype=np.int32)
            steps = [(5, 1), (6, 2)]
        model = V.vopp_create_model(ctx, desc)
        agent = V.vopp_agent_create(model, host_states, None, N, seed)
        states = torch.from_numpy(host_states.copy()).cuda()
        lw = torch.full((N,), float(np.float32(math.log(1.0 / N))), dtype=torch.float32,
                        device="cuda")
        anc = torch.empty(N, dtype=torch.int32, device="cuda")
        for t, (action, obs) in enumerate(steps):
            ess_a, res_a = V.vopp_belief_update(agent, action, obs, kind)
            ess_b, res_b = V.vopp_belief_update_noalloc(model, states, lw, action, obs, seed, t,
                                                        kind, 0, anc)
            st_a, lw_a, anc_a = V.vopp_agent_get_particles(agent, kind)
            assert res_a == res_b
            assert _close([ess_b], [ess_a])
            np.testing.assert_array_equal(anc.cpu().numpy(), anc_a)
            if kind == WL.NAV2D:
                assert _close(states.cpu().numpy(), st_a)
            else:
                np.testing.assert_array_equal(states.cpu().numpy(), st_a)
            assert _close(lw.cpu().numpy(), lw_a)
        # host arrays are refused by the entry point itself (cudaPointerGetAttributes),
        # before any device work, and the caller's current device is left as it was
        host = np.zeros(2 * N, dtype=np.float32)
        hlw = np.zeros(N, dtype=np.float32)
        o = (ctypes.c_float * 2)(1.0, 1.0)
        rc = V.lib.vopp_belief_update_noalloc(model, host.ctypes.data, hlw.ctypes.data, N, 0, o,
                                              1, 0, 0, None, None, None)
        assert rc == V.VOPP_E_INVALID
        assert torch.cuda.current_device() == 0
        # sizes beyond the static scratch are refused before any device work
        big = torch.zeros(65537, dtype=torch.float32, device="cuda")
        big_states = torch.zeros(2 * 65537, dtype=torch.float32, device="cuda")
        with pytest.raises(V.VoppError) as e:
            V.vopp_belief_update_noalloc(model, big_states, big, 0, (1.0, 1.0), 1, 0, V.VOPP_NAV2D)
        assert e.value.code == V.VOPP_E_INVALID
        V.vopp_agent_destroy(agent)
        V.vopp_model_destroy(model)
    finally:
        V.vopp_ctx_destroy(ctx)


def test_no_alloc_crowd_update_equals_agent_update():
    """CROWD particles (15 words each) through the allocation-free update equal the agent's
    update from the same particles, seed and step; beyond the scratch's CROWD capacity the
    call is refused."""
    import torch
    from paper_2510_27191_b300 import vopp as V
    from paper_2510_27191_b300 import workloads as WL
    ctx = V.vopp_ctx_create(0, 0, 0)
    try:
        m = V.vopp_create_model(ctx, V.make_desc(V.VOPP_CROWD))
        N = 700
        st = WL.pack_crowd_states(WL.crowd_root(N, 3, robot=(25.0, 3.0)))
        g = V.vopp_agent_create(m, st, None, N, 21)
        V.vopp_belief_update(g, 4, 0b000101, V.VOPP_CROWD)
        ga, glw, _ = V.vopp_agent_get_particles(g, V.VOPP_CROWD)
        dst = torch.from_numpy(st.copy()).cuda()
        dlw = torch.full((N,), -float(np.log(N)), dtype=torch.float32, device="cuda")
        V.vopp_belief_update_noalloc(m, dst, dlw, 4, 0b000101, 21, 0, V.VOPP_CROWD)
        assert dst.cpu().numpy().tolist() == ga.tolist()
        assert dlw.cpu().numpy().tolist() == glw.tolist()
        big = torch.zeros(15 * 30000, dtype=torch.float32, device="cuda")
        bw = torch.zeros(30000, dtype=torch.float32, device="cuda")
        with pytest.raises(V.VoppError) as e:
            V.vopp_belief_update_noalloc(m, big, bw, 0, 0, 1, 0, V.VOPP_CROWD)
        assert e.value.code == V.VOPP_E_INVALID
        V.vopp_agent_destroy(g)
        V.vopp_model_destroy(m)
    finally:
        V.vopp_ctx_destroy(ctx)
