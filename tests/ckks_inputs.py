"""Seeded CKKS inputs for the ring / CC-MM tests: random ciphertext batches,
switching keys (generated by the oracle's key generator from seeded secrets,
masks and errors), and column-wise encryptions of real matrices.

Oracle layout throughout: a ciphertext batch is [n, 2, L, N] (ciphertext,
part a/b, prime, coefficient); a switching key is [dnum, 2, L+K, N] (dnum
digits; L chain primes and K special primes).  The default gadget is one
digit per chain prime and one special prime; PR4/SP2 give the paper's
experimental gadget of two digits (two chain primes each) and two special
primes."""
import numpy as np

from paper_2503_16080_gb300 import synth

PR = synth.ntt_primes(50, 3)
SP = synth.ntt_primes(60, 1)[0]
PRP = PR + [SP]
PR4 = synth.ntt_primes(50, 4)
SP2 = synth.ntt_primes(60, 2)


def rand_cts(seed, n, N, primes):
    L = len(primes)
    cts = np.empty((n, 2, L, N), dtype=np.uint64)
    for pl, q in enumerate(primes):
        cts[:, :, pl, :] = synth.uniform_mod(seed, 10 + pl, (n, 2, N), q)
    return cts


def switching_key(oracle_mod, s_old, s_new, N, seed, primes_with_P=PRP, L=None, dnum=None):
    """Key s_old -> s_new; primes_with_P = L chain primes then the special ones
    (L defaults to one special prime), dnum digits (default L)."""
    L = len(primes_with_P) - 1 if L is None else L
    dnum = L if dnum is None else dnum
    a = np.stack([np.stack([synth.uniform_mod(seed, 100 + 10 * i + k, (N,), q)
                            for k, q in enumerate(primes_with_P)]) for i in range(dnum)])
    e = synth.rounded_gaussian(seed, 200, (dnum, N))
    return oracle_mod.ks_keygen(s_old, s_new, primes_with_P, a, e, L=L, dnum=dnum)


def aut_keys(oracle_mod, s, N, seed, primes_with_P=PRP, L=None, dnum=None):
    """Key j switches s(X^(2j+1)) -> s, 1 <= j < N; entry 0 is None."""
    keys = [None]
    for j in range(1, N):
        keys.append(switching_key(oracle_mod, oracle_mod.aut_key_secret(s, 2 * j + 1), s, N,
                                  seed + j, primes_with_P, L, dnum))
    return keys


def relin_key(oracle_mod, s, N, seed, primes_with_P=PRP, L=None, dnum=None):
    """Switches s^2 -> s."""
    return switching_key(oracle_mod, oracle_mod.negacyclic_int(s, s), s, N, seed, primes_with_P,
                         L, dnum)


def encrypt_columns(oracle_mod, M, s, delta, seed, primes=PR):
    """Column-wise RLWE: ciphertext j encrypts column j of M."""
    N = M.shape[0]
    L = len(primes)
    m = oracle_mod.ckks_encode(np.ascontiguousarray(M.T), delta)  # row j = column j of M
    a = np.stack([synth.uniform_mod(seed, 30 + pl, (N, N), q) for pl, q in enumerate(primes)])
    e = synth.rounded_gaussian(seed, 40, (N, N))
    b = oracle_mod.rlwe_encrypt_rows(a, s, m, e, primes)
    cts = np.empty((N, 2, L, N), dtype=np.uint64)
    cts[:, 0] = np.transpose(a, (1, 0, 2))
    cts[:, 1] = np.transpose(b, (1, 0, 2))
    return cts, m, e


def encrypt_rows(oracle_mod, X, s, delta, seed, primes=PR):
    """Ciphertext t encrypts row t of X (rows x N): the row-wise encryption of
    X, or the column-wise encryption of X^T."""
    rows, N = X.shape
    L = len(primes)
    m = oracle_mod.ckks_encode(np.ascontiguousarray(X), delta)
    a = np.stack([synth.uniform_mod(seed, 30 + pl, (rows, N), q) for pl, q in enumerate(primes)])
    e = synth.rounded_gaussian(seed, 40, (rows, N))
    b = oracle_mod.rlwe_encrypt_rows(a, s, m, e, primes)
    cts = np.empty((rows, 2, L, N), dtype=np.uint64)
    cts[:, 0] = np.transpose(a, (1, 0, 2))
    cts[:, 1] = np.transpose(b, (1, 0, 2))
    return cts, m, e


def encrypt_shared_a(oracle_mod, M, secrets, delta, seed, primes=PR):
    """Shared-a encryption of M (N x d2): column j as (a, b_j) under its own
    secret secrets[j], one uniform a for every column.  Returns the ciphertexts
    [d2, 2, L, N], the encoded message (d2 x N) and the errors (d2 x N)."""
    N, d2 = M.shape
    L = len(primes)
    m = oracle_mod.ckks_encode(np.ascontiguousarray(M.T), delta)       # row j = column j
    a = np.stack([synth.uniform_mod(seed, 30 + pl, (1, N), q) for pl, q in enumerate(primes)])
    e = synth.rounded_gaussian(seed, 40, (d2, N))
    cts = np.empty((d2, 2, L, N), dtype=np.uint64)
    for j in range(d2):
        b = oracle_mod.rlwe_encrypt_rows(a, secrets[j], m[j:j + 1], e[j:j + 1], primes)
        cts[j, 0] = a[:, 0, :]
        cts[j, 1] = b[:, 0, :]
    return cts, m, e


def precomp_keys(oracle_mod, secrets, U, s_new, N, seed, primes_with_P=PRP, L=None, dnum=None):
    """Key k switches s'_k = sum_j U[j, k] s_j (column k of S * U) to s_new."""
    S = np.stack([np.asarray(x, dtype=np.int64) for x in secrets])      # d2 x N
    SU = (U.astype(np.int64).T @ S)                                      # d3 x N: row k = s'_k
    return [switching_key(oracle_mod, SU[k], s_new, N, seed + k, primes_with_P, L, dnum)
            for k in range(U.shape[1])], SU


def to_batch(cts):
    """[n, 2, L, N] -> the library's part-major batch [2, L, n, N]."""
    return np.ascontiguousarray(np.transpose(cts, (1, 2, 0, 3)))


def from_batch(b):
    return np.ascontiguousarray(np.transpose(b, (2, 0, 1, 3)))


def stack_keys(keys, N, L):
    """List of keys (None for unused slots) -> [count, dnum, 2, L+K, N] (the
    shape of the first key present; N and L are checked against it)."""
    shape = next(k.shape for k in keys if k is not None)
    assert shape[3] == N and shape[2] > L
    out = np.zeros((len(keys),) + shape, dtype=np.uint64)
    for i, k in enumerate(keys):
        if k is not None:
            out[i] = k
    return out
