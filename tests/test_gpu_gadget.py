"""GPU parity of the ring path with the general key-switching gadget:
dnum digits of up to two chain primes (Garner's lift of a two-prime digit,
fused into the forward NTT's load) and one or two special primes (the CRT
lift of [u]_P in ModDown), bit-exact against the oracle's KeySwitch, which
lifts digits and [u]_P exactly with 128-bit integers.  The paper's
experimental gadget (Sec. 6: dnum = 2) with four 50-bit chain primes and two
60-bit special primes is the main case; uneven digits, one-prime digits with
two special primes, a single digit, and two-prime digits over one special
prime cover the other branches.  Every kernel path runs: N < 1024 (digits,
per-stage NTTs), the fused single-key switch (1024 <= N <= 8192), and the
streaming per-ciphertext-key path of Alg. 4's automorphisms."""
import numpy as np
import pytest
import torch

import ckks_inputs as C
from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu

PAPER = (C.PR4, C.SP2, 2)
GADGETS = [PAPER, (C.PR, C.SP2, 2), (C.PR4, C.SP2, 4), (C.PR4[:2], C.SP2, 1), (C.PR4, [C.SP], 2)]


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


def make_ring(ring_mod, N, chain, special, dnum):
    prp = list(chain) + list(special)
    return ring_mod.Ring(N, prp, special=len(special), dnum=dnum), prp


@pytest.mark.parametrize("gadget", GADGETS, ids=["paper", "uneven", "one-prime", "one-digit",
                                                 "one-special"])
@pytest.mark.parametrize("N,n", [(16, 3), (64, 2), (1024, 2), (8192, 1)])
def test_keyswitch_gadget_bit_exact(oracle_mod, ring_mod, gadget, N, n):
    chain, special, dnum = gadget
    L = len(chain)
    R, prp = make_ring(ring_mod, N, chain, special, dnum)
    key = C.switching_key(oracle_mod, synth.ternary(N, 1, N), synth.ternary(N, 2, N), N, 5, prp,
                          L, dnum)
    dk = R.prepare_keys(dev(key[None]))
    cts = C.rand_cts(N + n, n, N, chain)
    want = np.stack([oracle_mod.keyswitch(c, key, prp) for c in cts])
    got = host(R.keyswitch(dev(C.to_batch(cts)), dk))
    assert np.array_equal(C.from_batch(got), want)


@pytest.mark.parametrize("gadget", [PAPER, (C.PR, C.SP2, 2)], ids=["paper", "uneven"])
@pytest.mark.parametrize("N,index", [(1024, [2, 0, -1, 1]), (8192, [1, 0]), (64, [0, 1, 2])])
def test_keyswitch_indexed_gadget_bit_exact(oracle_mod, ring_mod, gadget, N, index):
    chain, special, dnum = gadget
    L = len(chain)
    R, prp = make_ring(ring_mod, N, chain, special, dnum)
    s_new = synth.ternary(N, 9, N)
    keys = [C.switching_key(oracle_mod, synth.ternary(N, 20 + i, N), s_new, N, 60 + i, prp, L,
                            dnum) for i in range(3)]
    dk = R.prepare_keys(dev(np.stack(keys)))
    cts = C.rand_cts(N + 3 * len(index), len(index), N, chain)
    want = np.stack([cts[c] if kid < 0 else oracle_mod.keyswitch(cts[c], keys[kid], prp)
                     for c, kid in enumerate(index)])
    kidx = torch.tensor(index, dtype=torch.int32, device="cuda")
    got = host(R.keyswitch_indexed(dev(C.to_batch(cts)), dk, kidx))
    assert np.array_equal(C.from_batch(got), want)


_setups = {}


def setup(oracle_mod, ring_mod, N, gadget=PAPER, seed=7):
    key = (N, id(gadget))
    if key in _setups:
        return _setups[key]
    chain, special, dnum = gadget
    L = len(chain)
    R, prp = make_ring(ring_mod, N, chain, special, dnum)
    s = synth.ternary(seed, 1, N)
    keys = C.aut_keys(oracle_mod, s, N, 5000 + N, prp, L, dnum)
    rk = C.relin_key(oracle_mod, s, N, 77, prp, L, dnum)
    dkeys = R.prepare_keys(dev(C.stack_keys(keys, N, L)))
    drk = R.prepare_keys(dev(rk[None]))
    _setups[key] = (R, prp, s, keys, rk, dkeys, drk)
    return _setups[key]


@pytest.mark.parametrize("N", [16, 256, 1024])
def test_transpose_gadget_bit_exact(oracle_mod, ring_mod, N):
    R, prp, s, keys, rk, dkeys, drk = setup(oracle_mod, ring_mod, N)
    cts = C.rand_cts(3 * N + 1, N, N, C.PR4)
    want = oracle_mod.transpose(cts, keys, prp)
    got = host(R.transpose(dev(C.to_batch(cts)), dkeys))
    assert np.array_equal(C.from_batch(got), want)


@pytest.mark.parametrize("N", [16, 64, 1024])
def test_cc_mm_gadget_bit_exact_and_decrypts(oracle_mod, ring_mod, N):
    R, prp, s, keys, rk, dkeys, drk = setup(oracle_mod, ring_mod, N)
    delta = 2.0 ** 40
    M1 = synth.uniform_unit(N, 12, (N, N))
    M2 = synth.uniform_unit(N, 13, (N, N))
    c1, _, _ = C.encrypt_columns(oracle_mod, M1, s, delta, 31, C.PR4)
    c2, _, _ = C.encrypt_columns(oracle_mod, M2, s, delta, 32, C.PR4)
    want, _ = oracle_mod.cc_mm(c1, c2, keys, rk, prp)
    got = C.from_batch(host(R.cc_mm(dev(C.to_batch(c1)), dev(C.to_batch(c2)), dkeys, drk)))
    assert np.array_equal(got, want)
    scale = delta * delta / C.PR4[-1]
    ref = M1 @ M2
    for j in range(0, N, max(1, N // 8)):
        dec = oracle_mod.rlwe_decrypt_rows(got[j, 0][:, None, :], got[j, 1][:, None, :], s,
                                           C.PR4[:-1])[:, 0]
        val = oracle_mod.crt2(dec[0], dec[1], C.PR4[0], C.PR4[1]).astype(np.float64) / scale
        assert np.max(np.abs(val - ref[:, j])) <= 2.0 ** -20


@pytest.mark.parametrize("N,d2,d3,rescale", [(16, 16, 8, True), (1024, 300, 5, False)])
def test_pc_mm_precomp_gadget_bit_exact(oracle_mod, ring_mod, N, d2, d3, rescale):
    chain, special, dnum = PAPER
    L = len(chain)
    R, prp = make_ring(ring_mod, N, chain, special, dnum)
    seed = N + d3
    secrets = [synth.ternary(seed, 100 + j, N) for j in range(d2)]
    s = synth.ternary(seed, 99, N)
    U = synth.uniform_int8(seed, 1, (d2, d3))
    keys, _ = C.precomp_keys(oracle_mod, secrets, U, s, N, 700 + seed, prp, L, dnum)
    M = synth.uniform_unit(seed, 2, (N, d2))
    cts, _, _ = C.encrypt_shared_a(oracle_mod, M, secrets, 2.0 ** 40, seed + 1, chain)
    want, _ = oracle_mod.pcmm_precomp(cts, U, keys, prp, rescale_out=rescale)
    dk = R.prepare_keys(dev(np.stack(keys)))
    a = dev(cts[0, 0])
    B = dev(np.transpose(cts[:, 1], (1, 0, 2)))
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
    got = R.pc_mm_precomp(Ut, a, B, dk, rescale=rescale)
    assert np.array_equal(C.from_batch(host(got)), want)


def test_gadget_rejects_bad_arguments(ring_mod):
    from paper_2503_16080_gb300.api import ModppError
    from paper_2503_16080_gb300.api import lib
    lib()
    prp = list(C.PR4) + list(C.SP2)
    for L, K, dnum in ((4, 3, 2), (4, 2, 0), (4, 2, 5), (6, 2, 2), (5, 2, 2), (4, 0, 2)):
        assert ring_mod._register().modpp_ring_bytes_ks(16, L, K, dnum) == 0, (L, K, dnum)
    with pytest.raises(ModppError):
        ring_mod.Ring(16, prp, special=2, dnum=1)      # two digits of... alpha = 4 > 2
    R = ring_mod.Ring(16, prp, special=2, dnum=2)
    assert R.key_shape() == (2, 2, 6, 16)
    bad = torch.zeros((1, 4, 2, 5, 16), dtype=torch.uint64, device="cuda")
    with pytest.raises(ValueError):
        R.prepare_keys(bad)
