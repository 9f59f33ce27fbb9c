"""The float32 <-> float64 conversions that the operand packers and the GEMM
epilogues do with integer operations (IEEE 754 binary32 / binary64 formats,
round to nearest with ties to even) give the same bits as the GPU's own
conversion instructions, on generated bit patterns that cover the whole
float32 range, its edges, exact ties and both directions of overflow."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_14822_gb300 import build, tnh
    build.build()
    c = tnh.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("seed", [1, 2024])
def test_integer_path_conversions_match_the_hardware(ctx, seed):
    assert ctx.debug_convert_check(1 << 24, seed=seed) == 0


def test_convert_check_of_nothing(ctx):
    assert ctx.debug_convert_check(0) == 0
