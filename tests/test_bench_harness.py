"""The benchmark's CKKS input harness (plain PyTorch, bench.py) against the
oracle on small rings, on the CPU: the switching keys it generates are the
oracle key generator's keys for the same masks and errors, its encryptions
decrypt, and its decryption of the oracle's CC-MM (Alg. 8) and PC-MM outputs
recovers the FP64 products within 2^-20 of the scale.  A planted wrong secret
must fail the check."""
import numpy as np
import pytest
import torch

import bench
import ckks_inputs as C
from paper_2503_16080_gb300 import synth


def _ccmm_setup(n, K=1, dnum=None):
    L = 4
    primes = synth.ntt_primes(50, L)
    prp = primes + synth.ntt_primes(60, K)
    inp = bench.ccmm_inputs(n, primes, prp, torch.device("cpu"), dnum=dnum)
    return primes, prp, inp


@pytest.mark.parametrize("K,dnum", [(1, None), (2, 2)])
def test_ccmm_harness_keys_are_oracle_keys(oracle_mod, K, dnum):
    n = 16
    primes, prp, inp = _ccmm_setup(n, K, dnum)
    s = inp["s"].numpy()
    L = len(primes)
    D = L if dnum is None else dnum
    for j in (1, 5, n - 1):
        key = inp["keys"][j].numpy()
        a = np.ascontiguousarray(key[:, 0])
        # errors: b + a*s on a special prime's plane (no gadget term there), centred
        q = prp[L]
        e = np.zeros((D, n), dtype=np.int64)
        for i in range(D):
            v = oracle_mod.rlwe_decrypt_rows(a[i][L][None, None, :], key[i, 1, L][None, None, :],
                                             s, [q])[0, 0].astype(object)
            e[i] = np.where(v > q // 2, v - q, v).astype(np.int64)
        assert np.abs(e).max() <= 19
        want = oracle_mod.ks_keygen(oracle_mod.aut_key_secret(s, 2 * j + 1), s, prp, a, e,
                                    L=L, dnum=D)
        assert np.array_equal(key, want)
    rk = inp["rkey"][0].numpy()
    assert rk.shape == (D, 2, L + K, n)


@pytest.mark.parametrize("K,dnum", [(1, None), (2, 2)])
def test_ccmm_harness_decrypts_oracle_product(oracle_mod, K, dnum):
    n = 32
    primes, prp, inp = _ccmm_setup(n, K, dnum)
    ct1 = C.from_batch(inp["ct1"].numpy())
    ct2 = C.from_batch(inp["ct2"].numpy())
    keys = [None] + [inp["keys"][j].numpy() for j in range(1, n)]
    out, _ = oracle_mod.cc_mm(ct1, ct2, keys, inp["rkey"][0].numpy(), prp)
    outb = torch.from_numpy(C.to_batch(out))
    r = bench.ccmm_decrypt_error(inp, outb, primes, cols=16)
    assert r["within_tolerance"] and r["other_primes_agree"], r
    inp["S32"] = -inp["S32"]  # planted mistake: decrypt with -s
    bad = bench.ccmm_decrypt_error(inp, outb, primes, cols=16)
    assert not bad["within_tolerance"]


def test_pcmm_harness_decrypts_oracle_product(oracle_mod, monkeypatch):
    n = 64
    monkeypatch.setattr(bench, "D", n)
    monkeypatch.setattr(bench, "K", n)
    monkeypatch.setattr(bench, "N", n)
    primes, U, A, B, M, sec = bench.make_inputs(with_message=True)
    U32 = U.astype(np.int32)
    Ao = torch.from_numpy(oracle_mod.mod_pp_mm(U32, A, primes))
    Bo = torch.from_numpy(oracle_mod.mod_pp_mm(U32, B, primes))
    r = bench.decrypt_error(U, M, sec, Ao, Bo, primes)
    assert r["within_tolerance"] and r["other_primes_agree"], r
    assert not bench.decrypt_error(U, M, -sec, Ao, Bo, primes)["within_tolerance"]
