"""GPU parity of the Mod-PP-MM path against the CPU oracle (bit-exact).

Every case draws seeded inputs from ``synth``, runs the CUDA library through
the C ABI (Python binding) and compares all outputs, or sampled rows at full
size, with ``oracle.mod_pp_mm`` element by element."""
import numpy as np
import pytest
import torch

from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu

P50 = synth.ntt_primes(50, 4)
P40 = synth.ntt_primes(40, 2)
P60 = synth.ntt_primes(60, 2)
P62 = synth.ntt_primes(62, 1)


@pytest.fixture(scope="module")
def mp(cuda_ok):
    import paper_2503_16080_gb300 as m
    m.lib()
    return m


@pytest.fixture(params=[8, 9, 10])
def digit_bits(request, mp):
    mp.set_digit_bits(request.param)
    yield request.param
    mp.set_digit_bits(0)


def to_gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_and_compare(mp, oracle_mod, U, A, primes, path="f16", rows=None):
    C = mp.modpp_mm(to_gpu(U), to_gpu(A), primes, path=path)
    torch.cuda.synchronize()
    assert mp.last_status() == 0
    got = C.cpu().numpy()
    if rows is None:
        want = oracle_mod.mod_pp_mm(U.astype(np.int32), A, primes)
        assert np.array_equal(got, want)
    else:
        want = oracle_mod.mod_pp_mm_rows(U.astype(np.int32), A, primes, rows)
        assert np.array_equal(got[:, rows], want)
    return got


@pytest.mark.parametrize("shape", [(1, 1, 1), (256, 256, 256), (130, 300, 70), (257, 513, 33),
                                   (128, 64, 32), (5, 1000, 200), (384, 1024, 96), (129, 8, 31)])
def test_f16_exact_shapes(mp, oracle_mod, shape, digit_bits):
    d, k, n = shape
    U = synth.uniform_int8(sum(shape), 1, (d, k))
    A = synth.uniform_mod(sum(shape), 2, (2, k, n), P50[0])
    A[1] = synth.uniform_mod(sum(shape), 3, (k, n), P50[1])
    run_and_compare(mp, oracle_mod, U, A, P50[:2])


@pytest.mark.parametrize("primes", [P40, P60, P62, [97, 65537], [P50[0], P60[0], P40[0]]])
def test_f16_prime_widths(mp, oracle_mod, primes, digit_bits):
    d, k, n = 200, 700, 90
    U = synth.uniform_int8(11, 1, (d, k))
    A = np.stack([synth.uniform_mod(11, 2 + j, (k, n), q) for j, q in enumerate(primes)])
    run_and_compare(mp, oracle_mod, U, A, primes)


@pytest.mark.parametrize("k", [255, 256, 257, 1024, 4096])
def test_f16_extreme_accumulation(mp, oracle_mod, k, digit_bits):
    # U = -128 and residue q - 2^(b-1) (lowest digit -2^(b-1), others 0): every
    # chunk sum of digit 0 reaches +2^24, the edge of binary32's exact integers.
    q = P50[0]
    b = digit_bits
    h = 1 << (b - 1)
    d, n = 128, 64
    U = np.full((d, k), -128, dtype=np.int8)
    A = np.full((1, k, n), q - h, dtype=np.uint64)
    got = run_and_compare(mp, oracle_mod, U, A, [q])
    assert np.all(got == (128 * h * k) % q)
    # Mixed extremes: +127/-128 rows against digit patterns +-(2^(b-1)) in every position.
    L = -(-(q - 1).bit_length() // b)
    S = sum(1 << (b * i) for i in range(L))
    vals = np.array([((h - 1) * S) % q, (q - h * S) % q if h * S < q else 1, q - 1, 0, h - 1, q - h],
                    dtype=np.uint64)
    A2 = vals[synth.u64(k, 5, k * n) % np.uint64(len(vals))].reshape(1, k, n)
    U2 = np.where(synth.u64(k, 6, d * k).reshape(d, k) & np.uint64(1), 127, -128).astype(np.int8)
    run_and_compare(mp, oracle_mod, U2, A2, [q])


def test_int32_u_kind(mp, oracle_mod):
    U = synth.uniform_int8(3, 1, (70, 333)).astype(np.int32)
    A = synth.uniform_mod(3, 2, (1, 333, 45), P50[2])
    run_and_compare(mp, oracle_mod, U, A, [P50[2]])


def test_zero_k_and_empty(mp):
    U = torch.zeros((7, 0), dtype=torch.int8, device="cuda")
    A = torch.zeros((1, 0, 5), dtype=torch.uint64, device="cuda")
    C = mp.modpp_mm(U, A, [P50[0]])
    assert C.shape == (1, 7, 5) and int(C.cpu().numpy().max()) == 0
    U = torch.zeros((0, 4), dtype=torch.int8, device="cuda")
    A = torch.zeros((1, 4, 5), dtype=torch.uint64, device="cuda")
    assert mp.modpp_mm(U, A, [P50[0]]).shape == (1, 0, 5)


@pytest.mark.parametrize("path", ["fp64", "fp64_tight"])
def test_fp64_path_exact(mp, oracle_mod, path):
    U = synth.uniform_int8(21, 1, (96, 520))
    A = np.stack([synth.uniform_mod(21, 2 + j, (520, 40), q) for j, q in enumerate(P50[:2])])
    run_and_compare(mp, oracle_mod, U, A, P50[:2], path=path)


def test_strided_planes_and_leading_dims(mp, oracle_mod):
    q = P50[0]
    U_full = synth.uniform_int8(31, 1, (64, 300))
    A_full = synth.uniform_mod(31, 2, (2, 260, 100), q)
    U = to_gpu(U_full)[:, :250]
    A = to_gpu(A_full)[:, :250, :80]
    out = torch.zeros((2, 64, 96), dtype=torch.uint64, device="cuda")
    mp.modpp_mm(U, A, [q, q], out=out[:, :, :80])
    got = out.cpu().numpy()
    want = oracle_mod.mod_pp_mm(U_full[:, :250].astype(np.int32),
                                np.ascontiguousarray(A_full[:, :250, :80]), [q, q])
    assert np.array_equal(got[:, :, :80], want)
    assert np.all(got[:, :, 80:] == 0)


def test_repeat_calls_are_identical(mp):
    U = to_gpu(synth.uniform_int8(41, 1, (256, 512)))
    A = to_gpu(synth.uniform_mod(41, 2, (3, 512, 128), P50[0]))
    a = mp.modpp_mm(U, A, [P50[0]] * 3).clone()
    b = mp.modpp_mm(U, A, [P50[0]] * 3)
    assert torch.equal(a, b)


@pytest.fixture(params=["digits", "crt"])
def wide_path(request, mp):
    mp.set_wide_path(request.param)
    yield request.param
    mp.set_wide_path("auto")


@pytest.mark.parametrize("shape", [(1, 1, 1), (130, 300, 70), (256, 512, 96), (64, 1000, 33),
                                   (200, 300, 600)])
def test_wide_residue_products(mp, oracle_mod, shape, digit_bits, wide_path):
    # Both operands residues (Alg. 8 step 2): bit-exact per prime against the oracle.
    d, k, n = shape
    primes = [P50[0], P60[0], P40[0], 97]
    U = np.stack([synth.uniform_mod(sum(shape), 40 + j, (d, k), q) for j, q in enumerate(primes)])
    A = np.stack([synth.uniform_mod(sum(shape), 50 + j, (k, n), q) for j, q in enumerate(primes)])
    C = mp.modpp_mm_wide(to_gpu(U), to_gpu(A), primes)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    for j, q in enumerate(primes):
        assert np.array_equal(got[j], oracle_mod.mod_pp_mm_residues(U[j], A[j], q)), f"prime {q}"


def test_wide_extremes(mp, oracle_mod, wide_path):
    q = P62[0]
    d, k, n = 128, 600, 40
    U = np.full((1, d, k), q - 1, dtype=np.uint64)
    A = np.full((1, k, n), q - 1, dtype=np.uint64)
    got = mp.modpp_mm_wide(to_gpu(U), to_gpu(A), [q]).cpu().numpy()
    assert np.all(got == k % q)  # (-1)(-1) summed k times
    U2 = synth.uniform_mod(9, 1, (1, d, k), q)
    A2 = np.where(synth.u64(9, 2, k * n).reshape(1, k, n) & np.uint64(1), q - 1, (q - 1) // 2)
    got2 = mp.modpp_mm_wide(to_gpu(U2), to_gpu(A2.astype(np.uint64)), [q]).cpu().numpy()
    assert np.array_equal(got2[0], oracle_mod.mod_pp_mm_residues(U2[0], A2[0].astype(np.uint64), q))


@pytest.mark.parametrize("k", [8192, 6000, 4100])
def test_wide_crt_largest_products(mp, oracle_mod, k):
    # k = 8192, 6000 and 4100 run the inner dimension in several pieces (the
    # last one ragged at 6000 and 4100).
    # The CRT form at its bound: |X| = k ((q-1)/2)^2 for 50-bit primes (16 small
    # primes over four pieces of the inner dimension at k = 8192), both signs,
    # plus random rows; against the oracle.
    q = P50[0]
    mp.set_wide_path("crt")
    try:
        assert mp.wide_plan_info(k, [q]) > 0
        d, n = 130, 300
        hi, lo = (q - 1) // 2, (q + 1) // 2       # balanced lifts +(q-1)/2 and -(q-1)/2
        U = synth.uniform_mod(k, 1, (1, d, k), q)
        A = synth.uniform_mod(k, 2, (1, k, n), q)
        U[0, 0, :] = hi
        U[0, 1, :] = lo
        A[0, :, 0] = hi
        A[0, :, 1] = lo
        got = mp.modpp_mm_wide(to_gpu(U), to_gpu(A), [q]).cpu().numpy()
        assert np.array_equal(got[0], oracle_mod.mod_pp_mm_residues(U[0], A[0], q))
        X = k * ((q - 1) // 2) ** 2
        assert int(got[0, 0, 0]) == X % q and int(got[0, 1, 1]) == X % q
        assert int(got[0, 0, 1]) == (-X) % q
    finally:
        mp.set_wide_path("auto")


def test_bounded_wait_gives_up_and_context_survives(mp, oracle_mod):
    # A device wait that nothing satisfies gives up after its limit and
    # reports MODPP_ERR_TIMEOUT through the status word; the context is still
    # usable afterwards (the next product is exact).
    assert mp.selftest_bounded_wait(5.0) == -7
    assert mp.selftest_bounded_wait(20.0) == -7
    U = synth.uniform_int8(61, 1, (130, 200))
    A = synth.uniform_mod(61, 2, (1, 200, 70), P50[0])
    run_and_compare(mp, oracle_mod, U, A, [P50[0]])
