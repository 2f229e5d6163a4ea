"""A3: the E4M3 digit layout (and the INT8 two-limb split) proved exhaustively
for every residue of every Rev-34 modulus; pinned by exact integer algebra."""
import pytest

from oracle import constants as C
from oracle import layouts as LY


@pytest.mark.parametrize("m", C.MODULI)
def test_fp8_layout_exact(m):
    info = LY.check_fp8_layout(m)
    assert info["max_combined"] < 2 ** 24


@pytest.mark.parametrize("m", C.MODULI)
def test_fp8_layout_exact_for_real_form_complex_product(m):
    """Re = a_R b_R + (-a_I) b_I accumulates 2 x 32 digit products per class."""
    info = LY.check_fp8_layout(m, K=64)
    assert info["max_combined"] < 2 ** 24


@pytest.mark.parametrize("m", C.MODULI)
def test_fp16_carrier_layout(m):
    info = LY.check_fp16_carrier(m)
    assert info["max_c0"] <= 16 and info["max_c1"] <= 32


@pytest.mark.parametrize("m", C.MODULI)
def test_int8_two_limb(m):
    LY.check_int8_two_limb(m)


def test_alpha_count():
    a = LY.alpha_fp8()
    # squares 3, 9-bit 4, 11-bit 9 MMAs per real product
    assert a["per_modulus"][1089] == 3 and a["per_modulus"][511] == 4 and a["per_modulus"][2039] == 9
    assert a["alpha_real"] == 6 * 3 + 3 * 4 + 3 * 9 == 57
    assert a["alpha_complex"] == 171


def test_e4m3_predicate():
    import numpy as np
    ok = LY.e4m3_exact(np.array([0, 1, 15, 16, 17, 18, 240, 448, 449, 480, -16, -17]))
    assert list(ok) == [True, True, True, True, False, True, True, True, False, False, True, False]
