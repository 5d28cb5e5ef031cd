"""The cost kernel's reciprocal: exhaustive comparison with the IEEE round-to-nearest reciprocal.

The arithmetic contract defines r = 1/Wz as the IEEE round-to-nearest reciprocal. On devices where a
one-step Newton-Raphson refinement of the hardware estimate agrees with it for every float in
[2^-126, 2^126), the kernel uses that refinement (and the IEEE routine outside the range); this test
runs the same exhaustive comparison the library runs at start-up and checks the fast path is in use on
this GPU, so the parity tests above exercise it.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu

ftv = pytest.importorskip("paper_1909_02294_gb300")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_newton_reciprocal_equals_ieee_on_the_whole_range():
    mismatches, used = ftv.ftv_reciprocal_check()
    assert mismatches == 0
    assert used
