"""Pins of the oracle's output stage (Algorithm 4, I <- reshape(I~)).

The slice layout is checked element by element against index loops on a small
volume; the 16-bit roundings against values whose nearest-even result is fixed
by the formats (bfloat16: 8 significant bits, float16: 11)."""
import numpy as np
import pytest

import oracle


def test_slices_match_index_loops():
    rng = np.random.default_rng(5)
    vol = rng.standard_normal((5, 4, 7)).astype(np.float32)
    for kb, kc in ((0, 7), (2, 3), (6, 1), (3, 0)):
        out = oracle.volume_slices(vol, kb, kc)
        assert out.shape == (kc, 4, 5)
        for k in range(kb, kb + kc):
            for j in range(4):
                for i in range(5):
                    assert out[k - kb, j, i] == vol[i, j, k]


def test_slice_range_errors():
    vol = np.zeros((2, 2, 4), np.float32)
    for kb, kc in ((-1, 1), (0, 5), (3, 2), (1, -1)):
        with pytest.raises(ValueError):
            oracle.volume_slices(vol, kb, kc)


def test_bf16_round_to_nearest_even():
    one = 0x3F80                       # bfloat16 1.0; the unit in the last place is 2^-7
    cases = {
        1.0: one,
        1.0 + 2.0 ** -7: one + 1,      # representable
        1.0 + 2.0 ** -8: one,          # tie between 1 and 1 + 2^-7: even (1.0)
        1.0 + 3 * 2.0 ** -8: one + 2,  # tie between odd 1 + 2^-7 and even 1 + 2^-6
        1.0 + 2.0 ** -8 + 2.0 ** -20: one + 1,   # above the tie
        1.0 + 2.0 ** -8 - 2.0 ** -20: one,       # below the tie
        -(1.0 + 2.0 ** -8): 0x8000 | one,
        0.0: 0,
        2.0 ** -135: 0,                # below half a bf16 subnormal unit (2^-133)
        3 * 2.0 ** -134: 2,            # subnormal tie between odd 1 and even 2 units
        3.0 * 2.0 ** 100: 0x7240,      # 1.5 * 2^101: exponent 228, mantissa 0x40
    }
    x = np.array(list(cases), dtype=np.float32)
    got = oracle.round_bf16_bits(x)
    assert got.tolist() == list(cases.values())
    # widening back is exact and the error is at most half a unit
    y = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    w = (oracle.round_bf16_bits(y).astype(np.uint32) << 16).view(np.float32)
    ulp = 2.0 ** (np.floor(np.log2(np.abs(y))) - 7)
    assert np.all(np.abs(w - y) <= ulp / 2)


def test_f16_round_to_nearest_even():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -11 + 2.0 ** -20], np.float32)
    out = oracle.volume_slices(x.reshape(3, 1, 1), dtype="f16").ravel()
    assert out.tolist() == [1.0, 1.0 + 2.0 ** -9, 1.0 + 2.0 ** -10]
