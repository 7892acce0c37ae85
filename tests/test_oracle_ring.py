"""Pins for the oracle's ring arithmetic in R_q = Z_q[X]/(X^N+1) (Sec. 2)."""
import numpy as np
import pytest

from paper_2503_16080_gb300 import synth


def negacyclic_bigint(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            p = int(a[i]) * int(b[j])
            if i + j < N:
                out[i + j] += p
            else:
                out[i + j - N] -= p
    return np.array([v % q for v in out], dtype=np.uint64)


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("q", [97, 12289, None])
def test_schoolbook_vs_bigint(oracle_mod, N, q):
    q = q or synth.ntt_primes(50, 1)[0]
    a = synth.uniform_mod(N, 1, (N,), q)
    b = synth.uniform_mod(N, 2, (N,), q)
    assert np.array_equal(oracle_mod.negacyclic_mul(a, b, q, schoolbook=True),
                          negacyclic_bigint(a, b, q))


@pytest.mark.parametrize("N", [2, 8, 64, 256, 1024])
def test_ntt_vs_schoolbook(oracle_mod, N):
    for q in synth.ntt_primes(50, 2) + synth.ntt_primes(60, 1):
        a = synth.uniform_mod(N, 3, (N,), q)
        b = synth.uniform_mod(N, 4, (N,), q)
        assert oracle_mod.find_psi(q, N) != 0
        assert np.array_equal(oracle_mod.negacyclic_mul(a, b, q),
                              oracle_mod.negacyclic_mul(a, b, q, schoolbook=True))


def test_psi_order(oracle_mod):
    q = synth.ntt_primes(50, 1)[0]
    for N in (4, 4096, 65536):
        psi = oracle_mod.find_psi(q, N)
        assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1


@pytest.mark.parametrize("i,j", [(0, 0), (3, 4), (5, 7), (7, 7), (1, 6)])
def test_monomial_products(oracle_mod, i, j):
    # X^i * X^j = (-1)^floor((i+j)/N) X^((i+j) mod N): the sign rule of X^N = -1.
    N, q = 8, synth.ntt_primes(50, 1)[0]
    a = np.zeros(N, np.uint64); a[i] = 1
    b = np.zeros(N, np.uint64); b[j] = 1
    c = oracle_mod.negacyclic_mul(a, b, q)
    expect = np.zeros(N, np.uint64)
    expect[(i + j) % N] = 1 if i + j < N else q - 1
    assert np.array_equal(c, expect)


def test_toeplitz_is_multiplication_matrix(oracle_mod):
    # Sec. 2: Toep(m) is the matrix of u -> u*m, so Toep(m) @ Vec(u) = Vec(u*m).
    N, q = 16, synth.ntt_primes(50, 1)[0]
    m = synth.uniform_mod(11, 1, (N,), q)
    u = synth.uniform_mod(11, 2, (N,), q)
    T = oracle_mod.toeplitz([int(x) for x in m])
    lhs = np.array([int(v) % q for v in T.dot(np.array([int(x) for x in u], dtype=object))],
                   dtype=np.uint64)
    assert np.array_equal(lhs, oracle_mod.negacyclic_mul(u, m, q))


def test_toeplitz_shape_matches_definition(oracle_mod):
    # The printed matrix of Sec. 2: first row (m0, -m_{N-1}, ..., -m1), first column (m0..m_{N-1}).
    T = oracle_mod.toeplitz([1, 2, 3, 4])
    assert [int(x) for x in T[0]] == [1, -4, -3, -2]
    assert [int(x) for x in T[:, 0]] == [1, 2, 3, 4]
    assert [int(x) for x in T[3]] == [4, 3, 2, 1]
