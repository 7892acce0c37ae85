"""Pins for Strategy 1 of Sec. 6.1 (Lemma le:strategy1), the FP64-limb form."""
import math
import os

import numpy as np
import pytest

from paper_2503_16080_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_base_closed_form(oracle_mod):
    # K = floor(sqrt(2^53/d2)): at d2 = 2^12 that is floor(2^20.5) = 1482910.
    assert oracle_mod.strategy1_base(4096) == 1482910
    assert oracle_mod.strategy1_base(4096) ** 2 * 4096 <= 2 ** 53
    assert (oracle_mod.strategy1_base(4096) + 1) ** 2 * 4096 > 2 ** 53
    assert oracle_mod.strategy1_base(1) == math.isqrt(2 ** 53)


def test_digit_counts_golden(oracle_mod):
    with open(os.path.join(GOLDEN, "strategy1_counts.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for d2, t1, t2, k1, k2 in rows:
        K = oracle_mod.strategy1_base(int(d2))
        assert oracle_mod.strategy1_digit_count(2 ** int(t1), K) == int(k1)
        assert oracle_mod.strategy1_digit_count(2 ** int(t2), K) == int(k2)


def test_digit_count_at_exact_power(oracle_mod):
    # |r| < K^k is needed; theta = K^2 exactly takes three digits.
    assert oracle_mod.strategy1_digit_count(1000 ** 2, 1000) == 3
    assert oracle_mod.strategy1_digit_count(1000 ** 2 - 1, 1000) == 2


def test_signed_digits_recompose(oracle_mod):
    K = 1482910
    X = np.array([0, 1, -1, K - 1, -(K - 1), K, -K, 2 ** 53 - 1, -(2 ** 53 - 1), 123456789012345],
                 dtype=object)
    digits = oracle_mod.strategy1_signed_digits(X, K, 3)
    back = sum(d.astype(object) * K ** i for i, d in enumerate(digits))
    assert np.array_equal(back, X)
    for d in digits:
        assert np.all(np.abs(d) < K)
        assert np.all((d == 0) | (np.sign(d) == np.sign(X.astype(np.int64))))


@pytest.mark.parametrize("d,k,n,bits", [(7, 64, 9, 50), (16, 4096, 4, 54), (5, 300, 6, 62)])
def test_strategy1_equals_definition(oracle_mod, d, k, n, bits):
    q = synth.ntt_primes(bits, 1)[0]
    U = synth.uniform_int8(d + k, 1, (d, k)).astype(np.int32)
    A = synth.uniform_mod(d + k, 2, (k, n), q)
    C, info = oracle_mod.strategy1_mod_pp_mm(U, A, q)
    assert np.array_equal(C, oracle_mod.mod_pp_mm(U, A, [q]))
    assert info["k2"] == 1
    # All three shapes need three A digits: K^2 <= max|A| < K^3.
    K = oracle_mod.strategy1_base(k)
    theta1 = int(np.max(np.abs(oracle_mod.centered(A, q))))
    assert info["k1"] == 3 and K ** 2 <= theta1 < K ** 3
