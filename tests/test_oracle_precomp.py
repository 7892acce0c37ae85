"""Pins for Alg. 7 (CP-MM with precomputation) on a shared-a encryption,
with the key switches back to one secret.

Checked against the decryption identities the algebra fixes: before the key
switches, ciphertext k decrypts under s'_k = sum_j U[j,k] s_j to exactly
sum_j U[j,k] (Delta m_j + e_j) (an identity over the integers, so a transposed
U or a wrong secret fails it); after them it decrypts under the target
secret to Delta (M U)_k within the key-switching error; and noise-free
(a = 0) inputs give exactly (0, Delta M U)."""
import numpy as np
import pytest

import ckks_inputs as C
from paper_2503_16080_gb300 import synth


def _setup(oracle_mod, N, d2, d3, seed):
    secrets = [synth.ternary(seed, 100 + j, N) for j in range(d2)]
    s = synth.ternary(seed, 99, N)
    U = synth.uniform_int8(seed, 1, (d2, d3))
    keys, SU = C.precomp_keys(oracle_mod, secrets, U, s, N, 500 * seed)
    return secrets, s, U, keys, SU


@pytest.mark.parametrize("N,d2,d3", [(16, 16, 16), (16, 7, 3), (32, 32, 5)])
def test_product_step_is_an_exact_encryption_under_su(oracle_mod, N, d2, d3):
    secrets, s, U, keys, SU = _setup(oracle_mod, N, d2, d3, 3)
    M = synth.uniform_unit(3, 2, (N, d2))
    cts, m, e = C.encrypt_shared_a(oracle_mod, M, secrets, 2.0 ** 40, 5)
    _, blocks = oracle_mod.pcmm_precomp(cts, U, keys, C.PRP)
    B1 = blocks["B1"]                                  # [d3, L, N]
    want = U.astype(object).T @ (m.astype(object) + e.astype(object))   # d3 x N
    for k in range(d3):
        for pl, q in enumerate(C.PR):
            a_s = oracle_mod.negacyclic_mul(cts[0, 0, pl], SU[k] % q, q).astype(object)
            dec = (a_s + B1[k, pl].astype(object)) % q
            assert np.array_equal(dec, (want[k] % q)), (k, pl)


def test_key_switched_result_decrypts(oracle_mod):
    N, d2, d3 = 32, 32, 6
    secrets, s, U, keys, SU = _setup(oracle_mod, N, d2, d3, 4)
    delta = 2.0 ** 40
    M = synth.uniform_unit(4, 2, (N, d2))
    cts, m, e = C.encrypt_shared_a(oracle_mod, M, secrets, delta, 6)
    out, _ = oracle_mod.pcmm_precomp(cts, U, keys, C.PRP)
    ref = M @ U.astype(np.float64)                     # column k of M U
    for k in range(d3):
        dec = oracle_mod.rlwe_decrypt_rows(out[k, 0][:, None, :], out[k, 1][:, None, :], s,
                                           C.PR)[:, 0]
        val = oracle_mod.crt2(dec[0], dec[1], C.PR[0], C.PR[1]).astype(np.float64) / delta
        # in units of the result's scale Delta * 2^5 (U as int8 at scale 2^5)
        assert np.max(np.abs(val - ref[:, k])) / 32 <= 2.0 ** -20
    # Rescale afterwards drops q_{L-1} and keeps the message exactly scaled.
    out_r, _ = oracle_mod.pcmm_precomp(cts, U, keys, C.PRP, rescale_out=True)
    assert out_r.shape == (d3, 2, len(C.PR) - 1, N)
    for k in range(d3):
        assert np.array_equal(out_r[k], oracle_mod.rescale(out[k], C.PR))


def test_noise_free_is_exact(oracle_mod):
    N, d2, d3 = 16, 9, 4
    secrets, s, U, keys, SU = _setup(oracle_mod, N, d2, d3, 5)
    L = len(C.PR)
    Mi = synth.uniform_mod(5, 7, (d2, N), 1 << 30).astype(object) - (1 << 29)
    cts = np.zeros((d2, 2, L, N), dtype=np.uint64)
    for pl, q in enumerate(C.PR):
        cts[:, 1, pl, :] = (Mi % q).astype(np.uint64)       # a = 0, b_j = m_j
    out, _ = oracle_mod.pcmm_precomp(cts, U, keys, C.PRP)
    want = U.astype(object).T @ Mi                          # row k = sum_j U[j,k] m_j
    assert np.all(out[:, 0] == 0)
    for pl, q in enumerate(C.PR):
        assert np.array_equal(out[:, 1, pl, :], (want % q).astype(np.uint64))


def test_rejects_distinct_a_parts(oracle_mod):
    N = 16
    cts = C.rand_cts(1, 3, N, C.PR)
    with pytest.raises(ValueError):
        oracle_mod.pcmm_precomp(cts, np.ones((3, 2), dtype=np.int8), [None, None], C.PRP)
