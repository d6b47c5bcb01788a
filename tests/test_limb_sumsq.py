"""Exactness of the integer arithmetic in the limb kernel's epilogue (host restatement).

For each SNP and row tile the epilogue reads, for every row i, the S limb sums C_il of
L^{-1} x: exact integers in FP32 accumulators, |C_il| <= n 2^B < 2^24 (limbs in
[-2^(B-1), 2^(B-1)], dosages <= 2). It needs sum_i T_i^2 with
T_i = sum_l C_il 2^(B(S-1-l)) exactly, over the tile's R = floor(256/S) rows. It groups
T_i^2 by powers of 2^B (P_ip = sum_{l+m=p} C_il C_im), sums 32 x 32 -> 64-bit products per
power over the rows and combines the powers once, modulo 2^128. For cohorts with
n 2^B < 2^22 it converts the accumulators with an add of 1.5 2^23 instead of a
float-to-int conversion.

These tests check both facts with Python integers and numpy float32 at the extremes of the
ranges the kernel allows (the largest |C| for every limb count and radix, every row of a
tile at the bound), so a wrong shift, a dropped cross term or a per-power sum that could
overflow 64 bits fails here.
"""
import random

import numpy as np
import pytest

M128 = (1 << 128) - 1
ROWS = {2: 128, 3: 85, 4: 64, 5: 51}   # rows per tile: floor(256 / S)


def direct(rows, S, B):
    total = 0
    for C in rows:
        T = sum(C[l] << (B * (S - 1 - l)) for l in range(S))
        total += T * T
    return total


def by_powers(rows, S, B):
    dg = [0] * S
    cr = [0] * (2 * S - 3)
    for C in rows:
        for l in range(S):
            dg[l] += C[l] * C[l]
            for m in range(l + 1, S):
                cr[l + m - 1] += C[l] * C[m]
    for x in dg + cr:   # each per-power sum fits a signed 64-bit accumulator
        assert -(1 << 63) <= x < (1 << 63)
    acc = 0
    for l in range(S):
        acc = (acc + ((dg[l] & M128) << (B * (2 * S - 2 - 2 * l)))) & M128
    for p in range(1, 2 * S - 2):
        acc = (acc + ((cr[p - 1] & M128) << (B * (2 * S - 2 - p) + 1))) & M128
    return acc


@pytest.mark.parametrize("S", [2, 3, 4, 5])
@pytest.mark.parametrize("B", [7, 8, 9])
def test_sum_of_squares_by_powers_is_exact(S, B):
    rng = random.Random(100 * S + B)
    R = ROWS[S]
    lim = (1 << 24) - 1
    cases = [[[lim] * S] * R, [[-lim] * S] * R,
             [[lim if (i + l) % 2 else -lim for l in range(S)] for i in range(R)]]
    for _ in range(40):
        cases.append([[rng.choice([rng.randint(-lim, lim), lim, -lim, 0]) for _ in range(S)]
                      for _ in range(R)])
    for rows in cases:
        d = direct(rows, S, B)
        assert d < (1 << 127)
        assert by_powers(rows, S, B) == d


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
