"""The C ABI without a GPU: the library builds, loads and exports every declared symbol;
host-side tables agree with the oracle's; calls fail cleanly without a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2510_27191_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vopp.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^VOPP_API\s+[\w\s\*]*?\b(vopp_\w+)\s*\(", src, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_loads_the_in_tree_library():
    build.build()
    from paper_2510_27191_b300 import vopp as V
    assert os.path.samefile(V.LIB_PATH, build.LIB)
    assert "sm_103a" in V.vopp_version()


def test_grid_threshold_table_matches_oracle():
    build.build()
    from paper_2510_27191_b300 import vopp as V
    t = V.vopp_grid_thresholds(222)
    assert [int(v) for v in t] == [O.grid_threshold(d) for d in range(222)]


def test_calls_fail_cleanly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    build.build()
    from paper_2510_27191_b300 import vopp as V
    with pytest.raises(V.VoppError) as e:
        V.vopp_ctx_create(0, 0, 0)
    assert e.value.code in (V.VOPP_E_CUDA, V.VOPP_E_INVALID)
    assert V.lib.vopp_model_num_actions(None) == V.VOPP_E_INVALID
    assert V.lib.vopp_plan(None, None, None, 1, 1, 1, 1.0, 0.5, None, 0, 0, None) == V.VOPP_E_INVALID


def test_noalloc_binding_refuses_tensors_the_kernel_would_overrun():
    """The allocation-free update writes n = log_weights.numel() particles into caller
    tensors the C entry point sees only as pointers, so the binding checks them first:
    host tensors, a short states tensor, wrong dtypes and short ancestors are refused
    before the library is called."""
    import torch
    build.build()
    from paper_2510_27191_b300 import vopp as V
    lw = torch.zeros(8, dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        V.vopp_belief_update_noalloc(0, torch.zeros(16), lw, 0, (1.0, 1.0), 1, 0, V.VOPP_NAV2D)
    if not torch.cuda.is_available():
        return
    lw = lw.cuda()
    for states in (torch.zeros(15, device="cuda"),                      # one word short
                   torch.zeros(16, dtype=torch.float64, device="cuda")):  # 8-byte elements
        with pytest.raises(ValueError, match="states"):
            V.vopp_belief_update_noalloc(0, states, lw, 0, (1.0, 1.0), 1, 0, V.VOPP_NAV2D)
    with pytest.raises(ValueError, match="ancestors"):
        V.vopp_belief_update_noalloc(0, torch.zeros(16, device="cuda"), lw, 0, (1.0, 1.0), 1, 0,
                                     V.VOPP_NAV2D, 0, torch.zeros(7, dtype=torch.int32, device="cuda"))
