"""The integer form of the VEGAS bin that the mixed-precision kinematics use (vegas_map_df): with
u = (2k + 1) 2^-53 (the 52-bit Philox integer k), the product u nb is the integer (2k + 1) nb in
units of 2^-53; rounding that integer to 53 significant bits, nearest-even, reproduces the FP64
product fl(u nb) exactly, so the bin floor(fl(u nb)) and the fraction fl(u nb) - b equal the FP64
map's.  The rounding is written here in Python integers, as the device code writes it in 64-bit
integers, and held against numpy's IEEE double multiplication (no GPU needed)."""
import numpy as np


def _round53(N: int) -> int:
    nbits = N.bit_length()
    sh = max(nbits - 53, 0)
    q = N >> sh
    if sh:
        rem, half = N & ((1 << sh) - 1), 1 << (sh - 1)
        if rem > half or (rem == half and (q & 1)):
            q += 1
    return q << sh


def _integer_bin(k: int, nb: int):
    Y = _round53((2 * k + 1) * nb)
    b = min(Y >> 53, nb - 1)
    return b, (Y - (b << 53))


def _fp64_bin(k: int, nb: int):
    u = (np.float64(k) + 0.5) * np.float64(2.0 ** -52)
    y = u * np.float64(nb)
    b = min(int(y), nb - 1)
    return b, y - np.float64(b)


def test_integer_bin_equals_fp64_product():
    rng = np.random.default_rng(20)
    ks = [int(v) for v in rng.integers(0, 2 ** 52, 200_000, dtype=np.int64)]
    ks += [0, 1, 2 ** 52 - 1, 2 ** 52 - 2, 2 ** 51, 2 ** 51 - 1]
    ties = 0
    for nb in (1, 7, 50, 63, 64):
        for k in ks:
            b_int, f_int = _integer_bin(k, nb)
            b_fp, f_fp = _fp64_bin(k, nb)
            assert b_int == b_fp, (k, nb)
            assert np.float64(f_int) * np.float64(2.0 ** -53) == f_fp, (k, nb)
            N = (2 * k + 1) * nb
            sh = max(N.bit_length() - 53, 0)
            ties += sh > 0 and (N & ((1 << sh) - 1)) == 1 << (sh - 1)
    # the nearest-even branch is exercised, not only the plain rounding
    assert ties > 100
