"""The FP32 FMA-peak measurement behind the pair kernel's arithmetic
cross-check: positive, repeatable to a few percent, and the paired f32x2 form
at least as fast per flop as the scalar one (it issues half the
instructions)."""
import pytest

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_positive_and_repeatable():
    a1, b1 = le.le_fp32_peak()
    a2, b2 = le.le_fp32_peak()
    assert a1 > 1.0 and b1 > 1.0
    assert abs(a1 - a2) <= 0.1 * max(a1, a2)
    assert abs(b1 - b2) <= 0.1 * max(b1, b2)
    assert b1 >= 0.9 * a1
