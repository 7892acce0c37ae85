"""The seeded generators: the torch stream is bit-identical to the numpy one,
index-addressed draws match contiguous draws, and the distributions have the
ranges the workloads need."""
import numpy as np
import torch

from paper_2503_16080_gb300 import synth


def test_splitmix_reference_values():
    # SplitMix64 published sequence for state 0: the first outputs of the
    # generator with seed 0 (Steele et al.; Vigna's reference implementation).
    z = np.uint64(0)
    gamma = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        first = synth._mix(np.array([z + gamma, z + gamma * np.uint64(2)], dtype=np.uint64))
    assert int(first[0]) == 0xE220A8397B1DCDAF
    assert int(first[1]) == 0x6E789E6AA1B965F4


def test_torch_stream_matches_numpy():
    for seed, stream, q in [(1, 2, 2 ** 50 - 27), (123, 7, 97), (5, 3, 2 ** 62 - 57)]:
        a = synth.uniform_mod(seed, stream, (1000,), q)
        b = synth.uniform_mod_torch(seed, stream, (1000,), q, "cpu").numpy()
        assert np.array_equal(a, b)
        c = synth.uniform_mod_torch(seed, stream, (1000,), q, "cpu", chunk=97).numpy()
        assert np.array_equal(a, c)
    assert np.array_equal(synth.u64(9, 9, 50, start=10),
                          synth.u64_torch(9, 9, 50, "cpu", start=10).view(torch.uint64).numpy())


def test_torch_int8_matches_numpy():
    a = synth.uniform_int8(3, 4, (5000,))
    b = synth.uniform_int8_torch(3, 4, (5000,), "cpu", chunk=333).numpy()
    assert np.array_equal(a, b)
    idx = np.array([0, 17, 4999])
    assert np.array_equal(synth.uniform_int8_at(3, 4, idx), a[idx])


def test_indexed_draws_match_contiguous():
    q = synth.ntt_primes(50, 1)[0]
    full = synth.uniform_mod(4, 5, (30, 40), q)
    idx = np.array([[0, 7], [29, 39], [11, 3]])
    flat = idx[:, 0] * 40 + idx[:, 1]
    assert np.array_equal(synth.uniform_mod_at(4, 5, flat, q), full[idx[:, 0], idx[:, 1]])


def test_ranges():
    q = 1000003
    x = synth.uniform_mod(1, 1, (100000,), q)
    assert x.max() < q and x.min() >= 0 and abs(float(x.mean()) / q - 0.5) < 0.01
    u = synth.uniform_int8(1, 2, (100000,))
    assert u.min() == -128 and u.max() == 127
    z = synth.uniform_unit(1, 3, (100000,))
    assert z.min() >= -1 and z.max() < 1
    e = synth.rounded_gaussian(1, 4, (100000,))
    assert abs(float(e.std()) - 3.2) < 0.1 and np.abs(e).max() <= 20
    s = synth.ternary(1, 5, 100000)
    assert set(np.unique(s)) == {-1, 0, 1}
    for q in synth.ntt_primes(50, 3):
        assert synth.is_prime(q) and (q - 1) % 2 ** 17 == 0 and q.bit_length() == 50
