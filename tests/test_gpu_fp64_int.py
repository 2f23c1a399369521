"""The integer-pipe FP64 multiply and add that the 2D double kernels use, checked on the GPU against
the FP64 pipe's own DMUL and DADD, bit for bit, through the C ABI."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op", [0, 1], ids=["mul", "add"])
@pytest.mark.parametrize("seed", [1, 7])
def test_integer_arithmetic_matches_fp64_pipe(op, seed):
    import paper_2208_01260_gb300 as hw
    accepted, mismatches, rejected = hw.hw_selftest_fp64_int(op, 1 << 26, seed)
    assert mismatches == 0 and rejected == 0
    assert accepted > (1 << 25)
