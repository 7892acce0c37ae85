"""CC-MM (Alg. 8) at the benchmark's size, N = 8192 with L = 4 primes of 50
bits and a 60-bit special prime, in the launch configuration the benchmark
times, checked on sampled outputs the oracle computes one by one; a
decryption check with real keys at N = 8192 (keys and encryptions from the
benchmark's plain-PyTorch harness, itself pinned to the oracle's key
generator on the CPU); and one at N = 1024 with the oracle's own keys.

Full size uses noise-free ciphertexts (a = 0, b = an arbitrary residue
matrix).  For them every KeySwitch sees a zero a-part and returns its input,
so Transpose is an exact matrix transpose and CC-MM reduces to
Rescale((0, C11)) with C11[m][j] = sum_t B1[t][m] * B2[j][t] mod q_p, where
B1[t] and B2[j] are the b-parts of ciphertexts t of ct1 and j of ct2.  The
oracle computes those dot products for sampled (j, m) and rescales them; the
whole a-part of the output must be 0.  The keys are uniform residues, as in
the benchmark."""
import numpy as np
import pytest
import torch

import ckks_inputs as C
from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 2024


@pytest.fixture(scope="module")
def pkg(cuda_ok):
    import __graft_entry__ as g
    g.build()
    import paper_2503_16080_gb300 as m
    return m


def _samples(n, extra, stream):
    edges = {0, 1, 31, 32, 127, 128, n // 2 - 1, n // 2, n - 2, n - 1}
    rnd = synth.u64(SEED, stream, extra) % np.uint64(n)
    return np.array(sorted(edges | {int(x) for x in rnd}))


def test_cc_mm_n8192_trivial_sampled(oracle_mod, pkg):
    N, L = 8192, 4
    primes = synth.ntt_primes(50, L)
    prp = primes + synth.ntt_primes(60, 1)
    dev = torch.device("cuda")
    ring = pkg.Ring(N, prp)
    keys = torch.empty((N, L, 2, L + 1, N), dtype=torch.uint64, device=dev)
    for k, q in enumerate(prp):
        keys.view(torch.int64)[:, :, :, k, :] = synth.uniform_mod_torch(
            SEED, 300 + k, (N, L, 2, N), q, dev).view(torch.int64)
    rkey = torch.empty((1, L, 2, L + 1, N), dtype=torch.uint64, device=dev)
    for k, q in enumerate(prp):
        rkey.view(torch.int64)[:, :, :, k, :] = synth.uniform_mod_torch(
            SEED, 400 + k, (1, L, 2, N), q, dev).view(torch.int64)
    ct1 = torch.zeros((2, L, N, N), dtype=torch.uint64, device=dev)
    ct2 = torch.zeros_like(ct1)
    for p, q in enumerate(primes):
        ct1.view(torch.int64)[1, p] = synth.uniform_mod_torch(SEED, 800 + p, (N, N), q,
                                                             dev).view(torch.int64)
        ct2.view(torch.int64)[1, p] = synth.uniform_mod_torch(SEED, 900 + p, (N, N), q,
                                                             dev).view(torch.int64)
    out = ring.cc_mm(ct1, ct2, keys, rkey)
    torch.cuda.synchronize()
    del keys, ct1, ct2
    o64 = out.view(torch.int64)
    assert int(torch.count_nonzero(o64[0])) == 0
    js = _samples(N, 14, 1)
    ms = _samples(N, 14, 2)
    got = o64[1][:, torch.from_numpy(js).cuda()][:, :, torch.from_numpy(ms).cuda()]
    got = got.cpu().numpy().view(np.uint64)                         # [L-1][len(js)][len(ms)]
    t = np.arange(N, dtype=np.int64)
    v = np.empty((L, len(js), len(ms)), dtype=np.uint64)
    for p, q in enumerate(primes):
        b2_rows = synth.uniform_mod_at(SEED, 900 + p, (js[:, None] * N + t[None, :]).ravel(),
                                       q).reshape(len(js), N)
        b1_cols = synth.uniform_mod_at(SEED, 800 + p, (t[:, None] * N + ms[None, :]).ravel(),
                                       q).reshape(N, len(ms))
        v[p] = oracle_mod.mod_pp_mm_residues(b2_rows, b1_cols, q)
    cnt = len(js) * len(ms)
    ct = np.zeros((2, L, cnt), dtype=np.uint64)
    ct[1] = v.reshape(L, cnt)
    want = oracle_mod.rescale(ct, primes)
    assert np.all(want[0] == 0)
    assert np.array_equal(got.reshape(L - 1, cnt), want[1])
    ring.close()


def test_cc_mm_n1024_decrypts(oracle_mod, pkg):
    N = 1024
    s = synth.ternary(31, 1, N)
    keys = C.aut_keys(oracle_mod, s, N, 31000)
    rk = C.relin_key(oracle_mod, s, N, 310)
    ring = pkg.Ring(N, C.PRP)
    L = len(C.PR)

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda().view(torch.uint64)

    dkeys = ring.prepare_keys(dev(C.stack_keys(keys, N, L)))
    drk = ring.prepare_keys(dev(rk[None]))
    delta = 2.0 ** 40
    M1 = synth.uniform_unit(31, 2, (N, N))
    M2 = synth.uniform_unit(31, 3, (N, N))
    c1, _, _ = C.encrypt_columns(oracle_mod, M1, s, delta, 41)
    c2, _, _ = C.encrypt_columns(oracle_mod, M2, s, delta, 42)
    out = ring.cc_mm(dev(C.to_batch(c1)), dev(C.to_batch(c2)), dkeys, drk)
    torch.cuda.synchronize()
    got = C.from_batch(out.view(torch.int64).cpu().numpy().view(np.uint64))
    scale = delta * delta / C.PR[-1]
    for j in _samples(N, 6, 3):
        dec = oracle_mod.rlwe_decrypt_rows(got[j, 0][:, None, :], got[j, 1][:, None, :], s,
                                           C.PR[:-1])[:, 0]
        val = oracle_mod.crt2(dec[0], dec[1], C.PR[0], C.PR[1]).astype(np.float64) / scale
        ref = M1 @ M2[:, j]
        assert np.max(np.abs(val - ref)) <= 2.0 ** -20, j
    ring.close()


@pytest.mark.parametrize("K,dnum", [(1, None), (2, 2)], ids=["one-prime-digits", "paper-dnum2"])
def test_cc_mm_n8192_real_keys_decrypts(pkg, K, dnum):
    # The benchmark's configuration (both key-switching gadgets).
    import bench
    N, L = 8192, 4
    primes = synth.ntt_primes(50, L)
    prp = primes + synth.ntt_primes(60, K)
    dev = torch.device("cuda")
    ring = pkg.Ring(N, prp, special=K, dnum=dnum)
    inp = bench.ccmm_inputs(N, primes, prp, dev, seed=77, dnum=dnum)
    keys = ring.prepare_keys(inp.pop("keys"))
    rkey = ring.prepare_keys(inp.pop("rkey"))
    out = ring.cc_mm(inp["ct1"], inp["ct2"], keys, rkey)
    torch.cuda.synchronize()
    del keys, rkey
    r = bench.ccmm_decrypt_error(inp, out, primes, cols=48)
    assert r["other_primes_agree"], r
    assert r["within_tolerance"], r
    ring.close()
