"""Pins for Strategy 2 of Sec. 6.1 (truncation), the approximate product with
the high-order bits of the residue operand, for one modulus q.

Checked against things other than the oracle's own formulas: rounding to a
multiple of 2^s written as an argmin over the candidates, Python-integer
products, the exact Mod-PP-MM where the truncation drops nothing, and the
error bounds the truncation implies (Sec. 6.1: about 2^-50 * k * ||U|| *
||B|| for the binary64 form; k * max|U| * 2^(s-1) for the rounding to a
multiple of 2^s)."""
import numpy as np
import pytest

from paper_2503_16080_gb300 import synth


def _centered_int(v, q):
    v = int(v) % q
    return v - q if 2 * v > q else v


def _nearest_multiple(x, s):
    """Nearest multiple of 2^s to x, ties to the larger: argmin over two candidates."""
    if s == 0:
        return x
    m = 1 << s
    lo = (x // m) * m
    hi = lo + m
    return hi if abs(hi - x) <= abs(x - lo) else lo


@pytest.mark.parametrize("q,s", [(97, 0), (97, 1), (97, 3), (101, 5), (2**31 - 1, 12)])
def test_round_high_matches_argmin(oracle_mod, q, s):
    B = np.arange(0, min(q, 4000), dtype=np.uint64).reshape(1, -1)
    got = oracle_mod.strategy2_round_high(B, q, s)
    want = [_nearest_multiple(_centered_int(v, q), s) for v in B[0]]
    assert [int(v) for v in got[0]] == want


def test_trunc_brute_force_small(oracle_mod):
    q, s = 1000003, 7
    U = synth.uniform_int8(1, 1, (5, 9)).astype(np.int64)
    B = synth.uniform_mod(1, 2, (9, 4), q)
    got = oracle_mod.strategy2_trunc(U, B, q, s)
    for r in range(5):
        for c in range(4):
            acc = sum(int(U[r, t]) * _nearest_multiple(_centered_int(B[t, c], q), s)
                      for t in range(9))
            assert int(got[r, c]) == acc % q


def test_trunc_without_dropped_bits_is_exact(oracle_mod):
    q = synth.ntt_primes(54, 1)[0]
    U = synth.uniform_int8(2, 1, (17, 33))
    B = synth.uniform_mod(2, 2, (33, 11), q)
    exact = oracle_mod.mod_pp_mm(U, B[None], [q])[0]
    assert np.array_equal(oracle_mod.strategy2_trunc(U, B, q, 0), exact)
    # Entries whose centred value is a multiple of 2^s lose nothing either.
    s = 9
    x = (synth.uniform_mod(2, 3, (33, 11), q >> (s + 1)).astype(object) - (q >> (s + 2))) * (1 << s)
    Bm = np.asarray(x % q, dtype=np.uint64)
    assert np.array_equal(oracle_mod.strategy2_trunc(U, Bm, q, s),
                          oracle_mod.mod_pp_mm(U, Bm[None], [q])[0])


@pytest.mark.parametrize("s", [1, 9, 20, 40])
def test_trunc_error_bound(oracle_mod, s):
    q = synth.ntt_primes(54, 1)[0]
    k = 200
    U = synth.uniform_int8(3, 1, (24, k))
    B = synth.uniform_mod(3, 2, (k, 16), q)
    diff = (oracle_mod.strategy2_trunc(U, B, q, s).astype(object)
            - oracle_mod.mod_pp_mm(U, B[None], [q])[0].astype(object)) % q
    diff = np.where(2 * diff > q, diff - q, diff)
    bound = k * int(np.max(np.abs(U.astype(np.int64)))) * (1 << (s - 1))
    assert int(np.max(np.abs(diff))) <= bound
    assert int(np.max(np.abs(diff))) > 0          # something was dropped


def test_fp64_exact_when_everything_fits(oracle_mod):
    # |B| < 2^20 and k * 128 * 2^20 < 2^53: every double is exact.
    q = synth.ntt_primes(21, 1, two_adicity=1)[0]
    U = synth.uniform_int8(4, 1, (12, 64))
    B = synth.uniform_mod(4, 2, (64, 10), q)
    assert np.array_equal(oracle_mod.strategy2_fp64(U, B, q), oracle_mod.mod_pp_mm(U, B[None], [q])[0])


def test_fp64_rounds_to_nearest_double(oracle_mod):
    # 2^53 + 1 is not a double: it rounds to 2^53 (nearest, ties to even), so
    # the product with U = 1 is off by one; 2^53 + 2 is exact.
    q = synth.ntt_primes(56, 1)[0]
    U = np.ones((1, 1), dtype=np.int8)
    for x, want in ((2 ** 53 + 1, 2 ** 53), (2 ** 53 + 2, 2 ** 53 + 2), (-(2 ** 53) - 1, -(2 ** 53))):
        B = np.array([[x % q]], dtype=np.uint64)
        assert int(oracle_mod.strategy2_fp64(U, B, q)[0, 0]) == want % q


def test_fp64_within_papers_bound(oracle_mod):
    # The paper's setting: one modulus q ~ 2^54, k = 4096.
    q = synth.ntt_primes(54, 1)[0]
    k = 4096
    U = synth.uniform_int8(5, 1, (8, k))
    B = synth.uniform_mod(5, 2, (k, 6), q)
    diff = (oracle_mod.strategy2_fp64(U, B, q).astype(object)
            - oracle_mod.mod_pp_mm(U, B[None], [q])[0].astype(object)) % q
    diff = np.where(2 * diff > q, diff - q, diff)
    normU = int(np.max(np.abs(U.astype(np.int64))))
    normB = int(np.max(np.abs(oracle_mod.centered(B, q))))
    assert int(np.max(np.abs(diff))) <= 2.0 ** -50 * k * normU * normB
