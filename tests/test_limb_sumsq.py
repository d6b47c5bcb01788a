"""Exactness of the integer arithmetic in the limb kernel's epilogue (host restatement).

For each SNP and row tile the epilogue reads, for every row i, the S limb sums C_il of
L^{-1} x: exact integers in FP32 accumulators, |C_il| <= n 2^B < 2^24 (limbs in
[-2^(B-1), 2^(B-1)], dosages <= 2). It forms T_i = sum_l C_il 2^(B(S-1-l)) in 64-bit
integers and adds T_i^2 over the tile's R = floor(256/S) rows in 128 bits. For cohorts with
n 2^B < 2^22 it converts the accumulators with an add of 1.5 2^23 instead of a
float-to-int conversion.

These tests check, with Python integers and numpy float32, that neither integer can
overflow at the extremes the kernel allows (every limb count and radix, every row of a
tile at the bound), that the recombination is the exact value, and that the fast
conversion is exact on its whole range and no further.
"""
import random

import numpy as np
import pytest

ROWS = {2: 128, 3: 85, 4: 64, 5: 51}   # rows per tile: floor(256 / S)


def combine(C, B):
    T = 0
    for c in C:               # T = T base + C_l, as the kernel does in int64
        T = T * (1 << B) + c
        assert -(1 << 63) <= T < (1 << 63)
    return T


@pytest.mark.parametrize("S", [2, 3, 4, 5])
@pytest.mark.parametrize("B", [7, 8, 9])
def test_tile_sum_of_squares_fits_128_bits(S, B):
    rng = random.Random(100 * S + B)
    R = ROWS[S]
    lim = (1 << 24) - 1
    cases = [[[lim] * S] * R, [[-lim] * S] * R,
             [[lim if (i + l) % 2 else -lim for l in range(S)] for i in range(R)]]
    for _ in range(20):
        cases.append([[rng.randint(-lim, lim) for _ in range(S)] for _ in range(R)])
    for rows in cases:
        total = 0
        for C in rows:
            T = combine(C, B)
            assert T == sum(C[l] * 2 ** (B * (S - 1 - l)) for l in range(S))
            total += T * T
        assert total < (1 << 128)


def test_magic_add_converts_every_integer_below_2_22():
    v = np.arange(-(1 << 22) + 1, 1 << 22, dtype=np.int64)
    f = v.astype(np.float32)
    back = (f + np.float32(12582912.0)).view(np.int32).astype(np.int64) - 0x4B400000
    assert np.array_equal(back, v)
    # and the bound is tight: from 2^22 + 1 on the sum passes 2^24, where the spacing is 2
    g = np.float32((1 << 22) + 1) + np.float32(12582912.0)
    assert int(g.view(np.int32)) - 0x4B400000 != (1 << 22) + 1


def test_small_sums_bound_matches_the_radix_rule():
    """The fast conversion is taken when n 2^B < 2^22: with 9-bit limbs (n < 32768) that is
    n < 8192, and the largest |C| = n 2^B then stays below 2^22."""
    for n in (1, 1000, 8191):
        assert n * 2 ** 9 < 2 ** 22
    assert not 8192 * 2 ** 9 < 2 ** 22
