"""The integer-pipe FP64 multiply that the 2D double kernels use for their weights' products, checked
on the GPU against the FP64 pipe's own DMUL, bit for bit, through the C ABI."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 7])
def test_integer_multiply_matches_dmul_on_device(seed):
    import paper_2208_01260_gb300 as hw
    accepted, mismatches, rejected = hw.hw_selftest_mul_int(1 << 26, seed)
    assert mismatches == 0 and rejected == 0
    assert accepted > (1 << 25)
