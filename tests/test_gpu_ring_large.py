"""GPU parity of the ring path at the degrees where its large-degree kernels
run, bit-exact against the oracle mod every q_j, with real keys (the oracle's
key generator) and ciphertexts whose a-parts are non-zero.

From N = 1024 on, a key switch with one key per ciphertext (the automorphism
keys of Alg. 4, steps 2-5) runs the forward NTT with the digit decomposition
fused into its load, the streaming key multiply-accumulate, the inverse NTT
and ModDown; the Tweaks (Alg. 3) run radix-8 passes.  The tests here drive
exactly that sequence:
- KeySwitch with a distinct key per ciphertext (modpp_keyswitch_indexed) at
  N = 1024 and 8192;
- Transpose (Alg. 4) at N = 1024 and 2048;
- CC-MM (Alg. 8) at N = 1024, whose second transpose also runs the zero-b
  form and whose relinearisation runs the single-key kernel, and its form
  with a row-wise right operand (Step 1 skipped, inner dimension 256)."""
import numpy as np
import pytest
import torch

import ckks_inputs as C
from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ring_mod(cuda_ok):
    import __graft_entry__ as g
    g.build()
    from paper_2503_16080_gb300 import ring
    return ring


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda().view(torch.uint64)


def host(t):
    torch.cuda.synchronize()
    return t.view(torch.int64).cpu().numpy().view(np.uint64)


_cache = {}


def setup(oracle_mod, ring_mod, N, seed=3):
    """Ring, secret, the oracle's N automorphism keys and relinearisation key,
    and their prepared device copies (cached per N)."""
    if N in _cache:
        return _cache[N]
    s = synth.ternary(seed, 1, N)
    keys = C.aut_keys(oracle_mod, s, N, 4000 * seed)
    rk = C.relin_key(oracle_mod, s, N, 97)
    R = ring_mod.Ring(N, C.PRP)
    L = len(C.PR)
    dkeys = R.prepare_keys(dev(C.stack_keys(keys, N, L)))
    drk = R.prepare_keys(dev(rk[None]))
    _cache[N] = (R, s, keys, rk, dkeys, drk)
    return _cache[N]


@pytest.mark.parametrize("N,index", [(1024, [2, 0, -1, 1]), (8192, [1, 0]), (1024, [1])])
def test_keyswitch_indexed_bit_exact(oracle_mod, ring_mod, N, index):
    # Distinct keys (different old secrets) per ciphertext; -1 copies.
    n = len(index)
    s_new = synth.ternary(N, 9, N)
    keys = [C.switching_key(oracle_mod, synth.ternary(N, 20 + i, N), s_new, N, 60 + i)
            for i in range(3)]
    R = ring_mod.Ring(N, C.PRP)
    dk = R.prepare_keys(dev(np.stack(keys)))
    cts = C.rand_cts(N + 7 * n, n, N, C.PR)
    want = np.stack([cts[c] if kid < 0 else oracle_mod.keyswitch(cts[c], keys[kid], C.PRP)
                     for c, kid in enumerate(index)])
    kidx = torch.tensor(index, dtype=torch.int32, device="cuda")
    got = host(R.keyswitch_indexed(dev(C.to_batch(cts)), dk, kidx))
    assert np.array_equal(C.from_batch(got), want)
    # in place
    x = dev(C.to_batch(cts))
    R.keyswitch_indexed(x, dk, kidx, out=x)
    assert np.array_equal(C.from_batch(host(x)), want)


@pytest.mark.parametrize("N", [1024, 2048])
def test_transpose_bit_exact_large(oracle_mod, ring_mod, N):
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, ring_mod, N)
    cts = C.rand_cts(5 * N, N, N, C.PR)
    want = oracle_mod.transpose(cts, keys, C.PRP)
    got = host(R.transpose(dev(C.to_batch(cts)), dkeys))
    assert np.array_equal(C.from_batch(got), want)


def test_cc_mm_bit_exact_n1024(oracle_mod, ring_mod):
    N = 1024
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, ring_mod, N)
    delta = 2.0 ** 40
    M1 = synth.uniform_unit(N, 4, (N, N))
    M2 = synth.uniform_unit(N, 5, (N, N))
    c1, _, _ = C.encrypt_columns(oracle_mod, M1, s, delta, 21)
    c2, _, _ = C.encrypt_columns(oracle_mod, M2, s, delta, 22)
    want, _ = oracle_mod.cc_mm(c1, c2, keys, rk, C.PRP)
    got = C.from_batch(host(R.cc_mm(dev(C.to_batch(c1)), dev(C.to_batch(c2)), dkeys, drk)))
    assert np.array_equal(got, want)
    # The product decrypts to column j of M1 @ M2 at scale Delta^2 / q_{L-1}.
    scale = delta * delta / C.PR[-1]
    ref = M1 @ M2
    for j in range(0, N, 61):
        dec = oracle_mod.rlwe_decrypt_rows(got[j, 0][:, None, :], got[j, 1][:, None, :], s,
                                           C.PR[:-1])[:, 0]
        val = oracle_mod.crt2(dec[0], dec[1], C.PR[0], C.PR[1]).astype(np.float64) / scale
        assert np.max(np.abs(val - ref[:, j])) <= 2.0 ** -20


def test_cc_mm_rowwise_bit_exact_n1024(oracle_mod, ring_mod):
    # Alg. 8 without Step 1 at N = 1024, inner dimension n = 256.
    N, n = 1024, 256
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, ring_mod, N)
    delta = 2.0 ** 40
    M1 = synth.uniform_unit(N, 14, (N, n))
    M2 = synth.uniform_unit(N, 15, (n, N))
    c1, _, _ = C.encrypt_rows(oracle_mod, np.ascontiguousarray(M1.T), s, delta, 41)
    rw, _, _ = C.encrypt_rows(oracle_mod, M2, s, delta, 42)
    want, _ = oracle_mod.cc_mm_rowwise(c1, rw, keys, rk, C.PRP)
    got, mult = R.cc_mm_ex(dev(C.to_batch(c1)), dev(C.to_batch(rw)), dkeys, drk, m2_rowwise=True)
    assert np.array_equal(C.from_batch(host(got)), want)
