"""Pins for the oracle's textbook CKKS harness (Sec. 2.2) and the exact PC-MM
identity behind the row-wise reduction (Thm th:pcmm, row format of Eq. mat_row_format)."""
import os

import numpy as np
import pytest

from paper_2503_16080_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_rounding_golden(oracle_mod):
    rows = load_golden("rounding.txt")
    x = np.array([float(r[0]) for r in rows])
    want = np.array([int(r[1]) for r in rows])
    assert np.array_equal(oracle_mod.ckks_encode(x, 1.0), want)


def test_encode_scale(oracle_mod):
    z = synth.uniform_unit(1, 1, (1000,))
    m = oracle_mod.ckks_encode(z, 2.0 ** 40)
    # |Delta z - m| <= 1/2 and the values are integers of magnitude <= 2^40.
    assert np.max(np.abs(z * 2.0 ** 40 - m)) <= 0.5
    assert np.max(np.abs(m)) <= 2 ** 40
    assert np.allclose(oracle_mod.ckks_decode(m, 2.0 ** 40), z, atol=2.0 ** -41)


def _encrypt(oracle_mod, rows, N, primes, seed=1):
    P = len(primes)
    a = np.stack([synth.uniform_mod(seed, 10 + j, (rows, N), q) for j, q in enumerate(primes)])
    s = synth.ternary(seed, 2, N)
    z = synth.uniform_unit(seed, 3, (rows, N))
    m = oracle_mod.ckks_encode(z, 2.0 ** 40)
    e = synth.rounded_gaussian(seed, 4, (rows, N))
    b = oracle_mod.rlwe_encrypt_rows(a, s, m, e, primes)
    return a, b, s, z, m, e


def test_decrypt_of_encrypt_is_exact(oracle_mod):
    primes = synth.ntt_primes(50, 3)
    a, b, s, z, m, e = _encrypt(oracle_mod, 6, 64, primes)
    dec = oracle_mod.rlwe_decrypt_rows(a, b, s, primes)
    for j, q in enumerate(primes):
        assert np.array_equal(dec[j], ((m + e).astype(object) % q).astype(np.uint64))
    assert np.array_equal(oracle_mod.crt2(dec[0], dec[1], primes[0], primes[1]), m + e)


def test_trivial_encryption(oracle_mod):
    # a = 0 gives b = m + e (nothing hidden): a check of the sign convention b = -a*s + m + e.
    primes = synth.ntt_primes(50, 2)
    N = 32
    a = np.zeros((2, 3, N), np.uint64)
    s = synth.ternary(2, 1, N)
    m = np.arange(3 * N, dtype=np.int64).reshape(3, N) - 40
    e = np.zeros_like(m)
    b = oracle_mod.rlwe_encrypt_rows(a, s, m, e, primes)
    for j, q in enumerate(primes):
        assert np.array_equal(b[j], (m.astype(object) % q).astype(np.uint64))


def test_encryption_matches_toeplitz_form(oracle_mod):
    # Row format (Eq. mat_row_format with S = Toep(s)): a_i . Toep(s)^t + b_i = m_i + e_i.
    primes = synth.ntt_primes(50, 1)
    q = primes[0]
    N = 16
    a, b, s, z, m, e = _encrypt(oracle_mod, 4, N, primes, seed=5)
    T = oracle_mod.toeplitz([int(x) for x in s])
    for i in range(4):
        lhs = (np.array([int(x) for x in a[0, i]], dtype=object).dot(T.T)
               + np.array([int(x) for x in b[0, i]], dtype=object))
        assert [int(v) % q for v in lhs] == [int(v) % q for v in (m[i] + e[i])]


@pytest.mark.parametrize("rows,N,d", [(16, 32, 8), (64, 64, 40)])
def test_pc_mm_rowwise_identity_exact(oracle_mod, rows, N, d):
    # Thm th:pcmm, transposed to the row format: Dec(U*A, U*B) = U * (m + e) exactly.
    primes = synth.ntt_primes(50, 3)
    a, b, s, z, m, e = _encrypt(oracle_mod, rows, N, primes, seed=7)
    U = synth.quantised_normal_int8(7, 9, (d, rows)).astype(np.int32)
    UA = oracle_mod.mod_pp_mm(U, a, primes)
    UB = oracle_mod.mod_pp_mm(U, b, primes)
    dec = oracle_mod.rlwe_decrypt_rows(UA, UB, s, primes)
    exact = U.astype(np.int64) @ (m + e)  # |.| <= 128 * 2^40 * rows < 2^63
    got = oracle_mod.crt2(dec[0], dec[1], primes[0], primes[1])
    assert np.array_equal(got, exact)
    assert np.array_equal(oracle_mod.crt2(dec[1], dec[2], primes[1], primes[2]), exact)
    # Decoded result vs the binary64 product (U/32) * M (quantisation scale 2^5).
    ref = (U.astype(np.float64) / 32.0) @ z
    dec_real = oracle_mod.ckks_decode(got, 2.0 ** 40 * 32.0)
    assert np.max(np.abs(dec_real - ref)) <= 2.0 ** -20
