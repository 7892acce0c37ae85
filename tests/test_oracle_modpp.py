"""Pins for the oracle's Mod-PP-MM (C = U*A mod q_j; Sec. 5 notation ModPPMM).

Each check compares the oracle with something other than itself: pure-Python
big-integer loops, closed forms, exact int64 numpy products, or algebraic
identities (linearity, identity matrix, negation)."""
import numpy as np
import pytest

from paper_2503_16080_gb300 import synth

Q62 = synth.ntt_primes(62, 1)[0]
Q50 = synth.ntt_primes(50, 3)
SMALL_PRIMES = [97, 65537, 2305843009213693951]  # 2^61-1 is a Mersenne prime


def brute(U, A, q):
    d, k = U.shape
    n = A.shape[1]
    out = np.empty((d, n), dtype=np.uint64)
    for r in range(d):
        for c in range(n):
            s = 0
            for t in range(k):
                s += int(U[r, t]) * int(A[t, c])
            out[r, c] = s % q
    return out


@pytest.mark.parametrize("q", SMALL_PRIMES + [Q62] + Q50[:1])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 2), (8, 7, 8), (5, 1, 6), (2, 9, 3)])
def test_brute_force_tiny(oracle_mod, q, shape):
    d, k, n = shape
    seed = hash((q, shape)) & 0xFFFF
    U = synth.uniform_int8(seed, 1, (d, k)).astype(np.int32)
    A = synth.uniform_mod(seed, 2, (k, n), q)
    assert np.array_equal(oracle_mod.mod_pp_mm(U, A, [q]), brute(U, A, q))


def test_brute_force_int32_entries(oracle_mod):
    q = Q62
    U = (synth.u64(5, 1, 6 * 4).astype(np.int64) >> 33).astype(np.int32).reshape(6, 4)
    A = synth.uniform_mod(5, 2, (4, 3), q)
    assert np.array_equal(oracle_mod.mod_pp_mm(U, A, [q]), brute(U, A, q))


@pytest.mark.parametrize("k", [1, 255, 256, 4096, 16384])
def test_worst_case_closed_form(oracle_mod, k):
    # U = -128 everywhere and A = q-1 (= -1 mod q): each entry is 128*k mod q.
    q = Q50[0]
    U = np.full((2, k), -128, dtype=np.int32)
    A = np.full((k, 3), q - 1, dtype=np.uint64)
    C = oracle_mod.mod_pp_mm(U, A, [q])
    assert np.all(C == (128 * k) % q)
    U2 = np.full((2, k), 127, dtype=np.int32)
    C2 = oracle_mod.mod_pp_mm(U2, A, [q])
    assert np.all(C2 == (-127 * k) % q)


def test_identity_and_negation(oracle_mod):
    q = Q50[1]
    A = synth.uniform_mod(9, 1, (16, 5), q)
    eye = np.eye(16, dtype=np.int32)
    assert np.array_equal(oracle_mod.mod_pp_mm(eye, A, [q]), A)
    neg = oracle_mod.mod_pp_mm(-eye, A, [q])
    assert np.array_equal(neg, np.where(A == 0, 0, np.uint64(q) - A))


def test_linearity(oracle_mod):
    q = Q50[2]
    U1 = synth.uniform_int8(3, 1, (12, 20)).astype(np.int32)
    U2 = synth.uniform_int8(3, 2, (12, 20)).astype(np.int32)
    A1 = synth.uniform_mod(3, 3, (20, 9), q)
    A2 = synth.uniform_mod(3, 4, (20, 9), q)
    f = lambda U, A: oracle_mod.mod_pp_mm(U, A, [q]).astype(object)
    A12 = ((A1.astype(object) + A2.astype(object)) % q).astype(np.uint64)
    assert np.array_equal((f(U1, A1) + f(U1, A2)) % q, f(U1, A12))
    assert np.array_equal((f(U1, A1) + f(U2, A1)) % q, f(U1 + U2, A1))


def test_cross_prime_consistency(oracle_mod):
    # Small A shared by all primes: C_j must be the integer product reduced mod q_j.
    primes = Q50 + [Q62, 65537]
    U = synth.uniform_int8(4, 1, (10, 300)).astype(np.int32)
    A_small = (synth.u64(4, 2, 300 * 7) >> np.uint64(44)).reshape(300, 7)
    exact = U.astype(np.int64) @ A_small.astype(np.int64)  # |.| < 2^7 * 2^20 * 300 < 2^36
    A = np.stack([A_small] * len(primes))
    C = oracle_mod.mod_pp_mm(U, A, primes)
    for j, q in enumerate(primes):
        assert np.array_equal(C[j], (exact.astype(object) % q).astype(np.uint64))


def test_row_subset(oracle_mod):
    q = Q50[0]
    U = synth.uniform_int8(6, 1, (33, 40)).astype(np.int32)
    A = synth.uniform_mod(6, 2, (2, 40, 17), q)
    full = oracle_mod.mod_pp_mm(U, A, [q, q])
    rows = np.array([0, 5, 32])
    assert np.array_equal(oracle_mod.mod_pp_mm_rows(U, A, [q, q], rows), full[:, rows])


def test_residue_operands(oracle_mod):
    q = Q50[0]
    U = synth.uniform_mod(7, 1, (5, 6), q)
    A = synth.uniform_mod(7, 2, (6, 4), q)
    assert np.array_equal(oracle_mod.mod_pp_mm_residues(U, A, q), brute(U.astype(object), A, q))


def test_outputs_canonical(oracle_mod):
    q = Q50[0]
    U = synth.uniform_int8(8, 1, (20, 50)).astype(np.int32)
    A = synth.uniform_mod(8, 2, (50, 30), q)
    C = oracle_mod.mod_pp_mm(U, A, [q])
    assert C.dtype == np.uint64 and int(C.max()) < q
