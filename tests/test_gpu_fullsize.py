"""Full-size parity at the workloads' own sizes, in the launch configuration
the benchmark times (pc_mm / pc_mv over all planes in one call).

The residue matrices are drawn on the GPU by the bit-identical torch stream of
``synth``; the oracle regenerates the sampled columns on the CPU through the
index-addressed stream and computes the sampled outputs one by one.  Samples:
rows and columns at tile boundaries (0, 127/128, the tile-column edges, the
last index) plus seeded random ones, and one whole boundary tile per plane."""
import numpy as np
import pytest
import torch

from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 2024


@pytest.fixture(scope="module")
def mp(cuda_ok):
    import paper_2503_16080_gb300 as m
    m.lib()
    return m


def _samples(n, extra, stream):
    edges = {0, 1, 31, 32, 39, 40, 47, 48, 63, 64, 127, 128, n // 2, n - 2, n - 1}
    rnd = synth.u64(SEED, stream, extra) % np.uint64(n)
    return np.array(sorted({e for e in edges if 0 <= e < n} | {int(x) for x in rnd}))


def _check_plane(oracle_mod, U_rows, got_plane, rows, cols, k, n, stream, q):
    idx = (np.arange(k, dtype=np.int64)[:, None] * n + cols[None, :]).ravel()
    A_cols = synth.uniform_mod_at(SEED, stream, idx, q).reshape(k, len(cols))
    want = oracle_mod.mod_pp_mm(U_rows.astype(np.int32), A_cols, [q])
    got = got_plane[np.ix_(rows, cols)]
    assert np.array_equal(got, want), f"stream {stream}: {np.count_nonzero(got != want)} mismatches"


def _run_pc(mp, oracle_mod, fn, d, k, n, primes, U_np, U_dev):
    P = len(primes)
    A = torch.stack([synth.uniform_mod_torch(SEED, 10 + j, (k, n), q, "cuda")
                     for j, q in enumerate(primes)])
    B = torch.stack([synth.uniform_mod_torch(SEED, 20 + j, (k, n), q, "cuda")
                     for j, q in enumerate(primes)])
    Aout, Bout = fn(U_dev, A, B, primes)
    torch.cuda.synchronize()
    assert mp.last_status() == 0
    del A, B
    rows = _samples(d, 6, 1)
    cols = _samples(n, 10, 2)
    # whole last tile (rows of the last 128-row block, last columns)
    tile_rows = np.arange(max(0, d - 128), d)
    tile_cols = np.arange(max(0, n - 48), n)
    U_rows = U_np(rows)
    U_tile = U_np(tile_rows)
    for j, q in enumerate(primes):
        for out, stream in ((Aout, 10 + j), (Bout, 20 + j)):
            plane = out[j]
            plane = plane.view(torch.int64)  # indexing is not implemented for uint64
            got_s = plane[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint64)
            _check_plane(oracle_mod, U_rows, got_s, np.arange(len(rows)), cols, k, n, stream, q)
            got_t = plane[torch.from_numpy(tile_rows).cuda()].cpu().numpy().view(np.uint64)
            _check_plane(oracle_mod, U_tile, got_t, np.arange(len(tile_rows)), tile_cols, k, n,
                         stream, q)


def test_pc_mm_n4096_three_50bit_primes(mp, oracle_mod):
    # The benchmark workload: U quantised N(0,1), six planes in one pc_mm call.
    d = k = n = 4096
    primes = synth.ntt_primes(50, 3)
    U = synth.quantised_normal_int8(SEED, 1, (d, k))
    _run_pc(mp, oracle_mod, mp.pc_mm, d, k, n, primes, lambda r: U[r], torch.from_numpy(U).cuda())


def test_pc_mm_n16384_four_50bit_primes(mp, oracle_mod):
    d = k = n = 16384
    primes = synth.ntt_primes(50, 4)
    U_dev = synth.uniform_int8_torch(SEED, 1, (d, k), "cuda")

    def U_rows(r):
        idx = (np.asarray(r, dtype=np.int64)[:, None] * k + np.arange(k)[None, :]).ravel()
        return synth.uniform_int8_at(SEED, 1, idx).reshape(len(r), k)

    _run_pc(mp, oracle_mod, mp.pc_mm, d, k, n, primes, U_rows, U_dev)
    torch.cuda.empty_cache()


def test_pc_mv_16384_batch32_four_50bit_primes(mp, oracle_mod):
    d = k = 16384
    n = 32
    primes = synth.ntt_primes(50, 4)
    U_dev = synth.uniform_int8_torch(SEED, 1, (d, k), "cuda")

    def U_rows(r):
        idx = (np.asarray(r, dtype=np.int64)[:, None] * k + np.arange(k)[None, :]).ravel()
        return synth.uniform_int8_at(SEED, 1, idx).reshape(len(r), k)

    _run_pc(mp, oracle_mod, mp.pc_mv, d, k, n, primes, U_rows, U_dev)
    torch.cuda.empty_cache()
