"""The bench's byte and operation models (the numerators of its roofline
fractions), checked on the CPU against their closed forms."""
import pytest

import bench


@pytest.mark.parametrize("n", [32, 64, 128, 256])
@pytest.mark.parametrize("s", [4, 8])
def test_pass_bytes_sum_to_the_27v_model_on_cubes(n, s):
    """Per-pass algorithmic bytes (R2C on axis 0) add up to the reference
    five-pass model 2V + 24 n^2 (n+1) + octant on a cube."""
    pb = bench.pass_bytes((n, n, n), s)
    assert sum(pb.values()) == bench.reference_model_bytes((n, n, n), s)
    V, X = n ** 3, (n + 1) * n * n * 2
    assert pb["r2c_ax0"] == pb["c2r_ax0"] == (V + X) * s
    assert pb["row_fwd"] == pb["row_inv"] == 3 * X * s


def test_fused_pairs_step_is_19v_plus_octant():
    """With both outer pairs fused (rho -> Y, Y -> phi) X never moves: the step
    is (V + Y) + (2 Y + oct) + (Y + V) reals, 19.07 V at 256^3."""
    n, s = 256, 4
    V = n ** 3
    Yr = (n + 1) * n * 2 * n * 2
    pb = bench.pass_bytes((n, n, n), s)
    step = 2 * (V + Yr) * s + pb["col_mid"]
    assert step == (2 * V + 4 * Yr + (n + 1) ** 3) * s
    assert step / (V * s) == pytest.approx(19.07, abs=0.01)
    assert step == pytest.approx(1.28e9, rel=1e-3)


def test_double_word_middle_pass_operation_count():
    """223,232 FP32 operations per length-512 column line, 257 x 512 lines at
    256^3 (the count ncu's FADD + FMUL + FFMA total matched)."""
    assert bench.dw_mid_ops((256, 256, 256)) == 29_373_759_488
    assert bench.dw_mid_ops((256, 256, 256)) == 223_232 * 257 * 512
