"""The integer-pipe FP64 multiply and reciprocal that the 2D double kernels use, checked on the GPU
through the C ABI: products (general and by the kernels' literal constants) bit for bit against the
FP64 pipe's DMUL, reciprocals within one ulp of the correctly rounded one."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op", [0, 1, 2], ids=["mul", "rcp", "const"])
@pytest.mark.parametrize("seed", [1, 7])
def test_integer_arithmetic_against_fp64_pipe(op, seed):
    import paper_2208_01260_gb300 as hw
    accepted, mismatches, rejected = hw.hw_selftest_fp64_int(op, 1 << 26, seed)
    assert mismatches == 0 and rejected == 0
    assert accepted > (1 << 25)
