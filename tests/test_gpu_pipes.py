"""Issue-rate microbenchmark of the leaf kernel's arithmetic (needs a GPU).  The rates are
counted in SM cycles, so they must sit near the per-SM issue widths of the part whatever
its clock: 128 FP32 lanes per cycle (4 schedulers x 32 lanes) is the ceiling of any
single-instruction operation."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_within_the_issue_width():
    from paper_2510_27191_b300 import vopp as V
    r = V.vopp_pipe_rates(0)
    assert len(r) == 12
    for op, (per_clk, per_s) in r.items():
        assert per_clk > 0 and per_s > 0, op
        if op != "philox4x32-10 call":
            assert per_clk <= 128 * 1.05, (op, per_clk)
    # an FP32 FMA issues at least at half the issue width on any recent NVIDIA SM
    assert r["fma.rn.f32"][0] >= 64, r["fma.rn.f32"]
    # one Philox call is tens of instructions
    assert r["philox4x32-10 call"][0] < r["fma.rn.f32"][0] / 10
