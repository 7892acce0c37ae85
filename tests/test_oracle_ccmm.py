"""Pins for the oracle's ring operations of the ciphertext-ciphertext product:
Tweak (Alg. 3), Aut, KeySwitch, Rescale, Transpose (Alg. 4), CC-MM (Alg. 8).

Each is checked against something other than itself: the definition of Tweak,
the coefficient formula of Aut (Sec. 2.2), ring-homomorphism laws, exact
results on noise-free (trivial) ciphertexts, and decryption identities within
the error bounds the algebra implies."""
import numpy as np
import pytest

from paper_2503_16080_gb300 import synth

import ckks_inputs
from ckks_inputs import PR, PRP, SP, rand_cts


@pytest.mark.parametrize("n,N", [(1, 8), (2, 8), (4, 8), (8, 8), (16, 8), (16, 32), (8, 64)])
def test_tweak_algorithm_equals_definition(oracle_mod, n, N):
    cts = rand_cts(n + N, n, N, PR[:2])
    assert np.array_equal(oracle_mod.tweak_alg(cts, PR[:2]), oracle_mod.tweak_def(cts, PR[:2]))


@pytest.mark.parametrize("n,N", [(2, 8), (4, 8), (8, 8), (16, 8), (8, 32), (64, 32)])
def test_tweak_twice_is_n_times_index_negation(oracle_mod, n, N):
    # Tweak is the n-point DFT over R_q with omega = X^(2N/n), a primitive
    # n-th root of unity there (X^t - 1 is invertible for 0 < t < 2N when q
    # splits X^N + 1), so applying it twice gives n * ct_(-j mod n): the DFT
    # inversion theorem, independent of how Tweak is computed.
    primes = PR[:2]
    cts = rand_cts(3 * n + N, n, N, primes)
    for f in (oracle_mod.tweak_def, oracle_mod.tweak_alg):
        if f is oracle_mod.tweak_alg and n > 2 * N:
            continue
        twice = f(f(cts, primes), primes)
        for pl, q in enumerate(primes):
            want = (cts[(-np.arange(n)) % n, :, pl, :].astype(object) * n) % q
            assert np.array_equal(twice[:, :, pl, :], want.astype(np.uint64)), (f.__name__, pl)


def test_tweak_n2_by_hand(oracle_mod):
    # n = 2: ct'_0 = ct_0 + ct_1 and ct'_1 = ct_0 + X^N ct_1 = ct_0 - ct_1.
    q = PR[0]
    cts = rand_cts(5, 2, 8, [q])
    out = oracle_mod.tweak_alg(cts, [q])
    a, b = cts[0].astype(object), cts[1].astype(object)
    assert np.array_equal(out[0], ((a + b) % q).astype(np.uint64))
    assert np.array_equal(out[1], ((a - b) % q).astype(np.uint64))


def test_monomial_rules(oracle_mod):
    q, N = PR[0], 16
    m = synth.uniform_mod(1, 1, (N,), q)
    assert np.array_equal(oracle_mod.monomial_mul(m, 2 * N, q), m)
    assert np.array_equal(oracle_mod.monomial_mul(m, N, q), np.where(m == 0, 0, np.uint64(q) - m))
    assert np.array_equal(oracle_mod.monomial_mul(oracle_mod.monomial_mul(m, 3, q), 5, q),
                          oracle_mod.monomial_mul(m, 8, q))


@pytest.mark.parametrize("ell", [1, 3, 5, 31, 33, 63])
def test_automorphism_coefficient_formula(oracle_mod, ell):
    # Sec. 2.2 (Aut): the result holds (-1)^floor(l' i / N) x_{l' i mod N}, l' = l^-1 mod 2N.
    q, N = PR[0], 32
    x = synth.uniform_mod(ell, 2, (N,), q)
    out = oracle_mod.automorphism(x, ell, q)
    li = pow(ell, -1, 2 * N)
    for i in range(N):
        src = (li * i) % N
        sign = -1 if ((li * i) // N) % 2 else 1
        assert int(out[i]) == (sign * int(x[src])) % q


def test_automorphism_is_a_ring_homomorphism(oracle_mod):
    q, N = PR[1], 64
    a = synth.uniform_mod(3, 1, (N,), q)
    b = synth.uniform_mod(3, 2, (N,), q)
    for ell in (3, 5, 127):
        lhs = oracle_mod.automorphism(oracle_mod.negacyclic_mul(a, b, q), ell, q)
        rhs = oracle_mod.negacyclic_mul(oracle_mod.automorphism(a, ell, q),
                                        oracle_mod.automorphism(b, ell, q), q)
        assert np.array_equal(lhs, rhs)
    comp = oracle_mod.automorphism(oracle_mod.automorphism(a, 3, q), 5, q)
    assert np.array_equal(comp, oracle_mod.automorphism(a, 15, q))


def _decrypt_centered(oracle_mod, ct, s, primes):
    """a*s + b per plane, then two-prime CRT to a centred integer."""
    L = ct.shape[1]
    dec = oracle_mod.rlwe_decrypt_rows(ct[0][:, None, :], ct[1][:, None, :], s, primes[:L])[:, 0]
    return oracle_mod.crt2(dec[0], dec[1], primes[0], primes[1])


def test_keyswitch(oracle_mod):
    N = 32
    s_old = synth.ternary(1, 1, N)
    s_new = synth.ternary(1, 2, N)
    L = len(PR)
    a = np.stack([np.stack([synth.uniform_mod(4, 100 + 10 * i + k, (N,), q)
                            for k, q in enumerate(PRP)]) for i in range(L)])
    e = synth.rounded_gaussian(4, 200, (L, N))
    key = oracle_mod.ks_keygen(s_old, s_new, PRP, a, e)
    # Noise-free trivial ciphertext: (0, b) is unchanged.
    triv = np.zeros((2, L, N), dtype=np.uint64)
    triv[1] = rand_cts(2, 1, N, PR)[0, 1]
    assert np.array_equal(oracle_mod.keyswitch(triv, key, PRP), triv)
    # An encryption of a small message under s_old decrypts to (almost) the
    # same message under s_new.
    m = (synth.uniform_unit(3, 1, (1, N)) * 2.0 ** 40).astype(np.int64)
    ea = np.stack([synth.uniform_mod(3, 2 + pl, (1, N), q) for pl, q in enumerate(PR)])
    eb = oracle_mod.rlwe_encrypt_rows(ea, s_old, m, np.zeros_like(m), PR)
    ct = np.stack([ea[:, 0, :], eb[:, 0, :]])
    before = _decrypt_centered(oracle_mod, ct, s_old, PR)
    assert np.array_equal(before, m[0])
    after = _decrypt_centered(oracle_mod, oracle_mod.keyswitch(ct, key, PRP), s_new, PR)
    # |error| <= (L * N * max|d_i| * max|e| / P) + 1/2 + N/2 (rounding times s)
    assert np.max(np.abs(after.astype(object) - before.astype(object))) <= N


def test_rescale(oracle_mod):
    N, L = 16, len(PR)
    ql = PR[-1]
    t = synth.uniform_int8(1, 1, (N,)).astype(np.int64) * 1000
    r = synth.uniform_int8(1, 2, (N,)).astype(np.int64)
    m = t.astype(object) * ql + r.astype(object)  # |r| < ql/2: round(m / ql) = t exactly
    ct = np.zeros((2, L, N), dtype=np.uint64)
    for pl, q in enumerate(PR):
        ct[1, pl] = (m.astype(object) % q).astype(np.uint64)
    out = oracle_mod.rescale(ct, PR)
    assert out.shape == (2, L - 1, N)
    assert np.all(out[0] == 0)
    for pl, q in enumerate(PR[:-1]):
        assert np.array_equal(out[1, pl], (t.astype(object) % q).astype(np.uint64))


def _aut_keys(oracle_mod, s, N, seed):
    return ckks_inputs.aut_keys(oracle_mod, s, N, seed)


def _encrypt_columns(oracle_mod, M, s, delta, seed):
    return ckks_inputs.encrypt_columns(oracle_mod, M, s, delta, seed)


def test_transpose_trivial_is_exact(oracle_mod):
    # Noise-free ciphertexts (0, m_i): Alg. 4 returns exactly (0, columns of M).
    N, L = 16, len(PR)
    s = synth.ternary(7, 1, N)
    keys = _aut_keys(oracle_mod, s, N, 1000)
    M = synth.uniform_mod(7, 2, (N, N), 1 << 20).astype(np.int64) - (1 << 19)
    cts = np.zeros((N, 2, L, N), dtype=np.uint64)
    for pl, q in enumerate(PR):
        cts[:, 1, pl, :] = (M.astype(object) % q).astype(np.uint64)  # ciphertext i holds row i
    out = oracle_mod.transpose(cts, keys, PRP)
    assert np.all(out[:, 0] == 0)
    for pl, q in enumerate(PR):
        assert np.array_equal(out[:, 1, pl, :], (M.T.astype(object) % q).astype(np.uint64))


def test_transpose_encrypted(oracle_mod):
    N = 16
    s = synth.ternary(8, 1, N)
    keys = _aut_keys(oracle_mod, s, N, 2000)
    M = synth.uniform_unit(8, 2, (N, N))
    delta = 2.0 ** 40
    cts, m, e = _encrypt_columns(oracle_mod, M, s, delta, 8)  # ciphertext j = column j
    out = oracle_mod.transpose(cts, keys, PRP)  # ciphertext i = row i
    for i in range(N):
        got = _decrypt_centered(oracle_mod, out[i], s, PR)
        want = m[:, i] + e[:, i]  # row i of (Delta*M + E): entries (j, i) of the column data
        assert np.max(np.abs(got.astype(object) - want.astype(object))) <= 64


def test_cc_mm_decrypts_to_product(oracle_mod):
    N = 16
    s = synth.ternary(9, 1, N)
    keys = _aut_keys(oracle_mod, s, N, 3000)
    L = len(PR)
    a = np.stack([np.stack([synth.uniform_mod(9, 500 + 10 * i + k, (N,), q)
                            for k, q in enumerate(PRP)]) for i in range(L)])
    e = synth.rounded_gaussian(9, 600, (L, N))
    s2 = oracle_mod.negacyclic_int(s, s)
    relin = oracle_mod.ks_keygen(s2, s, PRP, a, e)
    delta = 2.0 ** 40
    M1 = synth.uniform_unit(9, 2, (N, N))
    M2 = synth.uniform_unit(9, 3, (N, N))
    c1, _, _ = _encrypt_columns(oracle_mod, M1, s, delta, 11)
    c2, _, _ = _encrypt_columns(oracle_mod, M2, s, delta, 12)
    out, _ = oracle_mod.cc_mm(c1, c2, keys, relin, PRP)
    scale = delta * delta / PR[-1]
    ref = M1 @ M2
    for j in range(N):
        dec = _decrypt_centered(oracle_mod, out[j], s, PR[:-1]).astype(np.float64) / scale
        assert np.max(np.abs(dec - ref[:, j])) <= 2.0 ** -20


@pytest.mark.parametrize("n", [1, 4, 16])
def test_cc_mm_rowwise_trivial_is_exact(oracle_mod, n):
    # Alg. 8 without Step 1 on noise-free ciphertexts (0, m): every a-part
    # product is 0, so the result is exactly (0, Rescale(M * M')) with the
    # rescale rounding x -> (x - [x]_q)/q, [x]_q centred -- computed here
    # with Python integers from M (N x n) and M' (n x N).
    N, L = 16, len(PR)
    keys = _aut_keys(oracle_mod, synth.ternary(17, 1, N), N, 7000)
    relin = ckks_inputs.relin_key(oracle_mod, synth.ternary(17, 1, N), N, 71)
    M = synth.uniform_mod(17, 2, (N, n), 1 << 36).astype(object) - (1 << 35)
    Mp = synth.uniform_mod(17, 3, (n, N), 1 << 36).astype(object) - (1 << 35)
    c1 = np.zeros((n, 2, L, N), dtype=np.uint64)
    rw = np.zeros((n, 2, L, N), dtype=np.uint64)
    for pl, q in enumerate(PR):
        c1[:, 1, pl, :] = (M.T % q).astype(np.uint64)     # ciphertext j holds column j of M
        rw[:, 1, pl, :] = (Mp % q).astype(np.uint64)      # ciphertext t holds row t of M'
    out, _ = oracle_mod.cc_mm_rowwise(c1, rw, keys, relin, PRP)
    assert out.shape == (N, 2, L - 1, N)
    assert np.all(out[:, 0] == 0)
    X = M.dot(Mp)                                          # exact integers
    ql = PR[-1]
    r = X % ql
    r = np.where(2 * r > ql, r - ql, r)
    t = (X - r) // ql
    for pl, q in enumerate(PR[:-1]):
        assert np.array_equal(out[:, 1, pl, :], (t.T % q).astype(np.uint64))


@pytest.mark.parametrize("n", [4, 16])
def test_cc_mm_rowwise_decrypts_to_product(oracle_mod, n):
    # Column-wise M (N x n) times row-wise M' (n x N): decrypts to M * M'
    # within 2^-20 at scale Delta^2 / q_{L-1}.
    N = 16
    s = synth.ternary(19, 1, N)
    keys = _aut_keys(oracle_mod, s, N, 8000)
    relin = ckks_inputs.relin_key(oracle_mod, s, N, 81)
    delta = 2.0 ** 40
    M = synth.uniform_unit(19, 2, (N, n))
    Mp = synth.uniform_unit(19, 3, (n, N))
    c1, _, _ = ckks_inputs.encrypt_rows(oracle_mod, np.ascontiguousarray(M.T), s, delta, 21)
    rw, _, _ = ckks_inputs.encrypt_rows(oracle_mod, Mp, s, delta, 22)
    out, _ = oracle_mod.cc_mm_rowwise(c1, rw, keys, relin, PRP)
    scale = delta * delta / PR[-1]
    ref = M @ Mp
    for j in range(N):
        dec = _decrypt_centered(oracle_mod, out[j], s, PR[:-1]).astype(np.float64) / scale
        assert np.max(np.abs(dec - ref[:, j])) <= 2.0 ** -20


# ---- KeySwitch with the RNS gadget of dnum digits and K special primes (the
# gadget rank of Sec. 2.2's footnote; the experiments of Sec. 6 use dnum = 2).
# Chain primes, special primes, dnum: one digit per prime; two digits of two
# primes with two special primes (the paper's dnum); uneven digits (2 + 1);
# four one-prime digits with two special primes; one digit of two primes;
# two digits with a single special prime.
GADGETS = [(PR, [SP], 3), (ckks_inputs.PR4, ckks_inputs.SP2, 2), (PR, ckks_inputs.SP2, 2),
           (ckks_inputs.PR4, ckks_inputs.SP2, 4), (ckks_inputs.PR4[:2], ckks_inputs.SP2, 1),
           (ckks_inputs.PR4, [SP], 2)]


def _prod(xs):
    out = 1
    for x in xs:
        out *= int(x)
    return out


def _garner(res, mods):
    """The integer in [0, prod(mods)) with the given residues, by Garner's
    mixed-radix digits (v_0 + m_0 (v_1 + m_1 (v_2 + ...)))."""
    v, x, M = [], 0, 1
    for r, m in zip(res, mods):
        t = (int(r) - x) * pow(M, -1, int(m)) % int(m)
        x += t * M
        M *= int(m)
    return x


def _negacyclic_z(a, b, mod):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                out[i + j] += a[i] * b[j]
            else:
                out[i + j - N] -= a[i] * b[j]
    return [v % mod for v in out]


def _digit_primes(L, dnum):
    alpha = -(-L // dnum)
    return [list(range(d * alpha, min(L, (d + 1) * alpha))) for d in range(dnum)]


@pytest.mark.parametrize("chain,special,dnum", GADGETS)
def test_keyswitch_gadget_integer_route(oracle_mod, chain, special, dnum):
    # The oracle works prime by prime (digit lifts reduced per prime, RNS
    # products, ModDown by residues); here the same KeySwitch runs on whole
    # integers: keys lifted to [0, PQ), digits to [0, Q_d), products in
    # Z[X]/(X^N + 1) mod PQ, then the rounded division by P.
    N, L = 16, len(chain)
    prp = list(chain) + list(special)
    Q, P = _prod(chain), _prod(special)
    key = ckks_inputs.switching_key(oracle_mod, synth.ternary(5, 1, N), synth.ternary(5, 2, N),
                                    N, 31, prp, L, dnum)
    assert key.shape == (dnum, 2, L + len(special), N)
    ct = rand_cts(41, 1, N, chain)[0]
    got = oracle_mod.keyswitch(ct, key, prp)
    U = [[0] * N for _ in range(2)]
    for d, idx in enumerate(_digit_primes(L, dnum)):
        x = [_garner([ct[0, j, c] for j in idx], [chain[j] for j in idx]) for c in range(N)]
        assert all(0 <= v < _prod(chain[j] for j in idx) for v in x)
        for part in range(2):
            kd = [_garner(key[d, part, :, c], prp) for c in range(N)]
            prod = _negacyclic_z(x, kd, P * Q)
            U[part] = [(u + v) % (P * Q) for u, v in zip(U[part], prod)]
    for part in range(2):
        for c in range(N):
            r = U[part][c] % P
            if r > P // 2:
                r -= P
            v = (U[part][c] - r) // P
            for k, q in enumerate(chain):
                want = (v + (int(ct[1, k, c]) if part else 0)) % q
                assert int(got[part, k, c]) == want, (part, c, k)


@pytest.mark.parametrize("chain,special,dnum", GADGETS)
def test_ks_keygen_gadget_identity(oracle_mod, chain, special, dnum):
    # Key d satisfies b_d + a_d * s_new = e_d + P * g_d * s_old mod PQ with
    # g_d = (Q/Q_d) * ((Q/Q_d)^-1 mod Q_d), and sum_d [a]_{Q_d} g_d = a mod Q.
    N, L = 8, len(chain)
    prp = list(chain) + list(special)
    Q, P = _prod(chain), _prod(special)
    s_old, s_new = synth.ternary(6, 1, N), synth.ternary(6, 2, N)
    key = ckks_inputs.switching_key(oracle_mod, s_old, s_new, N, 37, prp, L, dnum)
    e = synth.rounded_gaussian(37, 200, (dnum, N))
    digits = _digit_primes(L, dnum)
    g = []
    for d, idx in enumerate(digits):
        Qd = _prod(chain[j] for j in idx)
        g.append((Q // Qd) * pow(Q // Qd, -1, Qd))
        kb = [_garner(key[d, 1, :, c], prp) for c in range(N)]
        ka = [_garner(key[d, 0, :, c], prp) for c in range(N)]
        lhs = [(u + v) % (P * Q) for u, v in zip(kb, _negacyclic_z(ka, [int(x) for x in s_new], P * Q))]
        rhs = [(int(e[d, c]) + P * g[d] * int(s_old[c])) % (P * Q) for c in range(N)]
        assert lhs == rhs, d
    a = [_garner(rand_cts(43, 1, N, chain)[0, 0, :, c], chain) for c in range(N)]
    for c in range(N):
        total = sum((a[c] % _prod(chain[j] for j in idx)) * g[d] for d, idx in enumerate(digits))
        assert total % Q == a[c]


@pytest.mark.parametrize("chain,special,dnum", GADGETS)
def test_keyswitch_gadget_decrypts(oracle_mod, chain, special, dnum):
    N, L = 32, len(chain)
    prp = list(chain) + list(special)
    s_old, s_new = synth.ternary(1, 1, N), synth.ternary(1, 2, N)
    key = ckks_inputs.switching_key(oracle_mod, s_old, s_new, N, 4, prp, L, dnum)
    triv = np.zeros((2, L, N), dtype=np.uint64)
    triv[1] = rand_cts(2, 1, N, chain)[0, 1]
    assert np.array_equal(oracle_mod.keyswitch(triv, key, prp), triv)
    m = (synth.uniform_unit(3, 1, (1, N)) * 2.0 ** 40).astype(np.int64)
    ea = np.stack([synth.uniform_mod(3, 2 + pl, (1, N), q) for pl, q in enumerate(chain)])
    eb = oracle_mod.rlwe_encrypt_rows(ea, s_old, m, np.zeros_like(m), chain)
    ct = np.stack([ea[:, 0, :], eb[:, 0, :]])
    before = _decrypt_centered(oracle_mod, ct, s_old, chain)
    assert np.array_equal(before, m[0])
    after = _decrypt_centered(oracle_mod, oracle_mod.keyswitch(ct, key, prp), s_new, chain)
    # digit d times e_d, summed and divided by P, plus the rounding (times s)
    e = synth.rounded_gaussian(4, 200, (dnum, N))
    Qd = max(_prod(chain[j] for j in idx) for idx in _digit_primes(L, dnum))
    bound = dnum * N * Qd * int(np.max(np.abs(e))) // _prod(special) + N
    assert np.max(np.abs(after.astype(object) - before.astype(object))) <= bound
