"""GPU parity of the ring / CC-MM path against the oracle, bit-exact mod q_j:
KeySwitch, Tweak (Alg. 3), Transpose (Alg. 4), Rescale and CC-MM (Alg. 8),
through the C ABI of include/modpp_ring.h.  Inputs are seeded; keys come from
the oracle's key generator."""
import numpy as np
import pytest
import torch

import ckks_inputs as C
from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_ready(cuda_ok):
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


def setup(oracle_mod, ring_mod, N, seed=1):
    """Ring, secret, oracle keys and prepared device keys for degree N (cached)."""
    if N in _cache:
        return _cache[N]
    s = synth.ternary(seed, 1, N)
    keys = C.aut_keys(oracle_mod, s, N, 1000 * seed)
    rk = C.relin_key(oracle_mod, s, N, 77)
    R = ring_mod.Ring(N, C.PRP)
    L = len(C.PR)
    dkeys = R.prepare_keys(dev(C.stack_keys(keys, N, L)))
    drk = R.prepare_keys(dev(rk[None]))
    _cache[N] = (R, s, keys, rk, dkeys, drk)
    return _cache[N]


@pytest.mark.parametrize("N,n", [(16, 1), (16, 5), (64, 7), (1024, 3), (2048, 2), (4096, 1), (8192, 2),
                                 (16384, 1)])
def test_keyswitch_bit_exact(oracle_mod, lib_ready, N, n):
    L = len(C.PR)
    s_old, s_new = synth.ternary(N, 1, N), synth.ternary(N, 2, N)
    key = C.switching_key(oracle_mod, s_old, s_new, N, 5)
    R = lib_ready.Ring(N, C.PRP)
    dk = R.prepare_keys(dev(key[None]))
    cts = C.rand_cts(N + n, n, N, C.PR)
    want = np.stack([oracle_mod.keyswitch(c, key, C.PRP) for c in cts])
    got = host(R.keyswitch(dev(C.to_batch(cts)), dk))
    assert np.array_equal(C.from_batch(got), want)
    # in place
    x = dev(C.to_batch(cts))
    R.keyswitch(x, dk, out=x)
    assert np.array_equal(C.from_batch(host(x)), want)


def test_keyswitch_chunked(oracle_mod, lib_ready, monkeypatch):
    # A chunk budget of a few ciphertexts makes the batch run in several chunks.
    N, n = 32, 11
    monkeypatch.setenv("MODPP_KS_CHUNK_BYTES", str(3 * 8 * 32 * (3 * 4 + 2 * 4)))
    key = C.switching_key(oracle_mod, synth.ternary(3, 1, N), synth.ternary(3, 2, N), N, 6)
    R = lib_ready.Ring(N, C.PRP)
    dk = R.prepare_keys(dev(key[None]))
    cts = C.rand_cts(99, n, N, C.PR)
    want = np.stack([oracle_mod.keyswitch(c, key, C.PRP) for c in cts])
    got = host(R.keyswitch(dev(C.to_batch(cts)), dk))
    assert np.array_equal(C.from_batch(got), want)


@pytest.mark.parametrize("N,n", [(16, 1), (16, 2), (16, 16), (16, 32), (64, 8), (256, 256)])
def test_tweak_bit_exact(oracle_mod, lib_ready, N, n):
    R = lib_ready.Ring(N, C.PRP)
    cts = C.rand_cts(7 * n + N, n, N, C.PR)
    want = oracle_mod.tweak_alg(cts, C.PR) if n <= N else oracle_mod.tweak_def(cts, C.PR)
    got = host(R.tweak(dev(C.to_batch(cts))))
    assert np.array_equal(C.from_batch(got), want)


@pytest.mark.parametrize("N,n", [(256, 256), (64, 128)])
def test_tweak_wide_index_form_bit_exact(oracle_mod, lib_ready, monkeypatch, N, n):
    # The radix-8 passes' 64-bit-index form (planes of 2^31 words or more),
    # forced at a small size.
    monkeypatch.setenv("MODPP_TWEAK_WIDE_INDEX", "1")
    R = lib_ready.Ring(N, C.PRP)
    cts = C.rand_cts(9 * n + N, n, N, C.PR)
    want = oracle_mod.tweak_alg(cts, C.PR) if n <= N else oracle_mod.tweak_def(cts, C.PR)
    got = host(R.tweak(dev(C.to_batch(cts))))
    assert np.array_equal(C.from_batch(got), want)


@pytest.mark.parametrize("N", [16, 64])
def test_rescale_bit_exact(oracle_mod, lib_ready, N):
    R = lib_ready.Ring(N, C.PRP)
    cts = C.rand_cts(N, 9, N, C.PR)
    want = np.stack([oracle_mod.rescale(c, C.PR) for c in cts])
    got = host(R.rescale(dev(C.to_batch(cts))))
    assert np.array_equal(C.from_batch(got), want)


@pytest.mark.parametrize("N", [16, 64, 256])
def test_transpose_bit_exact(oracle_mod, lib_ready, N):
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, lib_ready, N)
    cts = C.rand_cts(3 * N, N, N, C.PR)
    want = oracle_mod.transpose(cts, keys, C.PRP)
    got = host(R.transpose(dev(C.to_batch(cts)), dkeys))
    assert np.array_equal(C.from_batch(got), want)


def test_transpose_two_matrices_in_one_batch(oracle_mod, lib_ready):
    N = 16
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, lib_ready, N)
    c1 = C.rand_cts(41, N, N, C.PR)
    c2 = C.rand_cts(42, N, N, C.PR)
    both = np.concatenate([C.to_batch(c1), C.to_batch(c2)], axis=2)
    got = host(R.transpose(dev(both), dkeys))
    assert np.array_equal(C.from_batch(got[:, :, :N]), oracle_mod.transpose(c1, keys, C.PRP))
    assert np.array_equal(C.from_batch(got[:, :, N:]), oracle_mod.transpose(c2, keys, C.PRP))


def test_transpose_trivial_exact(oracle_mod, lib_ready):
    # Noise-free ciphertexts (0, row i): the result is exactly (0, column i).
    N = 64
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, lib_ready, N)
    L = len(C.PR)
    M = synth.uniform_mod(5, 2, (N, N), 1 << 20).astype(np.int64) - (1 << 19)
    b = np.zeros((2, L, N, N), dtype=np.uint64)
    for pl, q in enumerate(C.PR):
        b[1, pl] = (M.astype(object) % q).astype(np.uint64)
    got = host(R.transpose(dev(b), dkeys))
    assert np.all(got[0] == 0)
    for pl, q in enumerate(C.PR):
        assert np.array_equal(got[1, pl], (M.T.astype(object) % q).astype(np.uint64))


@pytest.mark.parametrize("N", [16, 64, 256])
def test_cc_mm_bit_exact_and_decrypts(oracle_mod, lib_ready, N):
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, lib_ready, N)
    delta = 2.0 ** 40
    M1 = synth.uniform_unit(N, 2, (N, N))
    M2 = synth.uniform_unit(N, 3, (N, N))
    c1, _, _ = C.encrypt_columns(oracle_mod, M1, s, delta, 11)
    c2, _, _ = C.encrypt_columns(oracle_mod, M2, s, delta, 12)
    want, _ = oracle_mod.cc_mm(c1, c2, keys, rk, C.PRP)
    got = C.from_batch(host(R.cc_mm(dev(C.to_batch(c1)), dev(C.to_batch(c2)), dkeys, drk)))
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    # and the product decrypts: column j of M1 @ M2 at scale Delta^2 / q_{L-1}
    scale = delta * delta / C.PR[-1]
    ref = M1 @ M2
    for j in range(0, N, max(1, N // 8)):
        dec = oracle_mod.rlwe_decrypt_rows(got[j, 0][:, None, :], got[j, 1][:, None, :], s,
                                           C.PR[:-1])[:, 0]
        val = oracle_mod.crt2(dec[0], dec[1], C.PR[0], C.PR[1]).astype(np.float64) / scale
        assert np.max(np.abs(val - ref[:, j])) <= 2.0 ** -20


def test_cc_mm_stage_timing(oracle_mod, lib_ready):
    from paper_2503_16080_gb300 import api
    N = 16
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, lib_ready, N)
    c = dev(C.to_batch(C.rand_cts(5, N, N, C.PR)))
    api.profile_enable(True)
    try:
        R.cc_mm(c, c, dkeys, drk)
        ms = R.cc_mm_stage_ms()
    finally:
        api.profile_enable(False)
    assert len(ms) == 4 and all(m >= 0 for m in ms)


def test_ring_rejects_bad_arguments(lib_ready):
    from paper_2503_16080_gb300.api import ModppError
    with pytest.raises(ModppError):
        lib_ready.Ring(16, C.PR[:2] + [C.PR[0]])          # repeated prime
    with pytest.raises(ModppError):
        lib_ready.Ring(12, C.PRP)                         # N not a power of two
    R = lib_ready.Ring(16, C.PRP)
    with pytest.raises(ValueError):
        R.transpose(dev(np.zeros((2, 3, 8, 16), dtype=np.uint64)),
                    dev(np.zeros((16, 3, 2, 4, 16), dtype=np.uint64)))


def test_ring_rejects_misaligned_pointers(lib_ready):
    # The ring kernels move coefficient pairs in 16-byte accesses: pointers
    # off a 16-byte boundary are refused on the host before any launch.
    from paper_2503_16080_gb300.api import lib
    N, L = 16, len(C.PR)
    R = lib_ready.Ring(N, C.PRP)
    buf = torch.zeros(2 * 2 * L * N + 4, dtype=torch.int64, device="cuda")
    base = buf.data_ptr()
    assert base % 16 == 0
    out = base + 8 * (2 * L * N + 2)
    assert lib().modpp_rescale(R._h, base + 8, out, 1, None) == -1
    assert lib().modpp_rescale(R._h, base, out + 8, 1, None) == -1
    assert lib().modpp_rescale(R._h, base, out, 1, None) == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("N", [2, 4, 8])
def test_transpose_small_degrees(oracle_mod, lib_ready, N):
    s = synth.ternary(N, 7, N)
    keys = C.aut_keys(oracle_mod, s, N, 5000 + N)
    R = lib_ready.Ring(N, C.PRP)
    L = len(C.PR)
    dkeys = R.prepare_keys(dev(C.stack_keys(keys, N, L)))
    cts = C.rand_cts(9 * N, N, N, C.PR)
    got = host(R.transpose(dev(C.to_batch(cts)), dkeys))
    assert np.array_equal(C.from_batch(got), oracle_mod.transpose(cts, keys, C.PRP))


def test_cc_mm_two_prime_chain(oracle_mod, lib_ready):
    # The shortest chain CC-MM accepts: L = 2 (one prime left after Rescale).
    N = 16
    prp = C.PR[:2] + [C.SP]
    s = synth.ternary(21, 1, N)
    keys = C.aut_keys(oracle_mod, s, N, 21000, prp)
    rk = C.relin_key(oracle_mod, s, N, 210, prp)
    R = lib_ready.Ring(N, prp)
    dkeys = R.prepare_keys(dev(C.stack_keys(keys, N, 2)))
    drk = R.prepare_keys(dev(rk[None]))
    c1 = C.rand_cts(31, N, N, C.PR[:2])
    c2 = C.rand_cts(32, N, N, C.PR[:2])
    want, _ = oracle_mod.cc_mm(c1, c2, keys, rk, prp)
    got = C.from_batch(host(R.cc_mm(dev(C.to_batch(c1)), dev(C.to_batch(c2)), dkeys, drk)))
    assert got.shape == (N, 2, 1, N)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("N,n", [(16, 16), (16, 4), (16, 1), (64, 24), (256, 256), (256, 100)])
def test_cc_mm_rowwise_bit_exact_and_decrypts(oracle_mod, lib_ready, N, n):
    # Alg. 8 with Step 1 skipped: column-wise M1 (N x n) times row-wise M2 (n x N).
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, lib_ready, N)
    delta = 2.0 ** 40
    M1 = synth.uniform_unit(N + n, 6, (N, n))
    M2 = synth.uniform_unit(N + n, 7, (n, N))
    c1, _, _ = C.encrypt_rows(oracle_mod, np.ascontiguousarray(M1.T), s, delta, 31)
    rw, _, _ = C.encrypt_rows(oracle_mod, M2, s, delta, 32)
    want, _ = oracle_mod.cc_mm_rowwise(c1, rw, keys, rk, C.PRP)
    got, mult = R.cc_mm_ex(dev(C.to_batch(c1)), dev(C.to_batch(rw)), dkeys, drk, m2_rowwise=True)
    got = C.from_batch(host(got))
    assert mult == 1.0 / C.PR[-1]
    assert np.array_equal(got, want)
    scale = delta * delta * mult
    ref = M1 @ M2
    for j in range(0, N, max(1, N // 8)):
        dec = oracle_mod.rlwe_decrypt_rows(got[j, 0][:, None, :], got[j, 1][:, None, :], s,
                                           C.PR[:-1])[:, 0]
        val = oracle_mod.crt2(dec[0], dec[1], C.PR[0], C.PR[1]).astype(np.float64) / scale
        assert np.max(np.abs(val - ref[:, j])) <= 2.0 ** -20


def test_cc_mm_rowwise_equals_cc_mm_after_transpose(oracle_mod, lib_ready):
    # Giving Alg. 8 the transposed (row-wise) right operand and skipping Step 1
    # is the same computation as the column-wise call.
    N = 64
    R, s, keys, rk, dkeys, drk = setup(oracle_mod, lib_ready, N)
    c1 = dev(C.to_batch(C.rand_cts(51, N, N, C.PR)))
    c2 = dev(C.to_batch(C.rand_cts(52, N, N, C.PR)))
    full = host(R.cc_mm(c1, c2, dkeys, drk))
    rw = R.transpose(c2, dkeys)
    part, _ = R.cc_mm_ex(c1, rw, dkeys, drk, m2_rowwise=True)
    assert np.array_equal(host(part), full)
    col, _ = R.cc_mm_ex(c1, c2, dkeys, drk)
    assert np.array_equal(host(col), full)


def test_cc_mm_ex_rejects_bad_shapes(lib_ready):
    from paper_2503_16080_gb300.api import lib
    N = 16
    R = lib_ready.Ring(N, C.PRP)
    assert lib().cc_mm_ex_workspace(R._h, 8, 0) == 0       # column-wise needs n = N
    assert lib().cc_mm_ex_workspace(R._h, 0, 1) == 0
    assert lib().cc_mm_ex_workspace(R._h, N + 1, 1) == 0
    assert lib().cc_mm_ex_workspace(R._h, 4, 2) == 0       # unknown flag
    assert lib().cc_mm_ex_workspace(R._h, 4, 1) > 0
    assert lib().cc_mm_ex_workspace(R._h, N, 0) == lib().cc_mm_workspace(R._h)
