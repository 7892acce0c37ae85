"""GPU parity of Strategy 2 of Sec. 6.1 (truncation), modpp_mm_trunc, through
the C ABI.

The f16 form (the residue operand rounded to multiples of 2^s, then an exact
product) is bit-exact against the oracle's definition for every s, modulus
width and ragged shape, including a full-size 4096^3 product checked on
sampled rows.  The binary64 form (53-bit rounding, one DGEMM, exact residues
of the double products) is checked against the exact product within the
paper's bound, 2^-50 * k * max|U| * max|B|, and equal to it where every
double is exact."""
import numpy as np
import pytest
import torch

from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg(cuda_ok):
    import __graft_entry__ as g
    g.build()
    import paper_2503_16080_gb300 as p
    return p


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda().view(torch.uint64)


def _centred_diff(a, b, q):
    d = (a.astype(object) - b.astype(object)) % q
    return np.where(2 * d > q, d - q, d)


Q54 = synth.ntt_primes(54, 1)[0]
Q61_ODD = (1 << 61) - 1 - 2 * 12345          # odd, not required to be prime
Q31 = synth.ntt_primes(31, 1, two_adicity=1)[0]


@pytest.mark.parametrize("q,s", [(Q54, 0), (Q54, 1), (Q54, 9), (Q54, 18), (Q54, 27), (Q54, 40),
                                 (Q61_ODD, 25), (Q31, 4), (Q31, 31)])
@pytest.mark.parametrize("shape", [(300, 700, 130), (1, 1, 1), (129, 64, 65)])
def test_f16_trunc_bit_exact(oracle_mod, pkg, q, s, shape):
    d, k, n = shape
    U = synth.uniform_int8(s + 3, 1, (d, k))
    B = synth.uniform_mod(s + 3, 2, (k, n), q)
    got = pkg.modpp_mm_trunc(torch.from_numpy(U).cuda(), _dev(B), q, path="f16", drop_bits=s)
    want = oracle_mod.strategy2_trunc(U, B, q, s)
    assert np.array_equal(got.cpu().numpy(), want)


def test_f16_trunc_int32_plaintext_and_bound(oracle_mod, pkg):
    q, s, k = Q54, 20, 512
    U = synth.uniform_int8(7, 1, (96, k)).astype(np.int32)
    B = synth.uniform_mod(7, 2, (k, 80), q)
    got = pkg.modpp_mm_trunc(torch.from_numpy(U).cuda(), _dev(B), q, drop_bits=s).cpu().numpy()
    assert np.array_equal(got, oracle_mod.strategy2_trunc(U, B, q, s))
    exact = oracle_mod.mod_pp_mm(U, B[None], [q])[0]
    assert np.max(np.abs(_centred_diff(got, exact, q))) <= k * 128 * 2 ** (s - 1)


def test_f16_trunc_full_size_sampled_rows(oracle_mod, pkg):
    # 4096^3 with the paper's single modulus ~2^54, two digits dropped at b = 9.
    q, s, N = Q54, 18, 4096
    U = synth.uniform_int8_torch(11, 1, (N, N), "cuda")
    B = synth.uniform_mod_torch(11, 2, (N, N), q, "cuda")
    C = pkg.modpp_mm_trunc(U, B, q, drop_bits=s)
    rows = np.array([0, 1, 127, 128, 2047, 4000, 4095])
    cols = np.unique(np.r_[0, 63, 64, 4095, np.linspace(0, N - 1, 60).astype(np.int64)])
    Un = U.cpu().numpy()[rows]
    Bn = np.ascontiguousarray(B.view(torch.int64).cpu().numpy().view(np.uint64)[:, cols])
    want = oracle_mod.strategy2_trunc(Un, Bn, q, s)
    assert np.array_equal(C.cpu().numpy()[rows][:, cols], want)


def test_fp64_exact_when_everything_fits(oracle_mod, pkg):
    q = synth.ntt_primes(21, 1, two_adicity=1)[0]
    U = synth.uniform_int8(8, 1, (70, 64))
    B = synth.uniform_mod(8, 2, (64, 50), q)
    got = pkg.modpp_mm_trunc(torch.from_numpy(U).cuda(), _dev(B), q, path="fp64")
    assert np.array_equal(got.cpu().numpy(), oracle_mod.mod_pp_mm(U, B[None], [q])[0])


@pytest.mark.parametrize("ubits", [7, 19])
def test_fp64_within_papers_bound(oracle_mod, pkg, ubits):
    # The paper's setting: one modulus q ~ 2^54, k = 4096; U int8, or int32
    # with |U| <= 2^19 (the paper's ||U||).
    q, k = Q54, 4096
    if ubits == 7:
        U = synth.uniform_int8(9, 1, (64, k))
    else:
        U = (synth.uniform_mod(9, 1, (64, k), 1 << 20).astype(np.int64) - (1 << 19)).astype(np.int32)
    B = synth.uniform_mod(9, 2, (k, 96), q)
    got = pkg.modpp_mm_trunc(torch.from_numpy(U).cuda(), _dev(B), q, path="fp64").cpu().numpy()
    exact = oracle_mod.mod_pp_mm(U, B[None], [q])[0]
    err = int(np.max(np.abs(_centred_diff(got, exact, q))))
    normU = int(np.max(np.abs(U.astype(np.int64))))
    normB = int(np.max(np.abs(oracle_mod.centered(B, q))))
    assert err <= 2.0 ** -50 * k * normU * normB
    # the oracle's binary64 form obeys the same bound
    ref = oracle_mod.strategy2_fp64(U[:4], B, q)
    assert np.max(np.abs(_centred_diff(ref, exact[:4], q))) <= 2.0 ** -50 * k * normU * normB


def test_trunc_edge_cases_and_errors(pkg):
    from paper_2503_16080_gb300.api import ModppError
    q = Q54
    U = torch.ones((4, 0), dtype=torch.int8, device="cuda")
    B = torch.zeros((0, 5), dtype=torch.uint64, device="cuda")
    assert int(pkg.modpp_mm_trunc(U, B, q, drop_bits=9).view(torch.int64).abs().sum()) == 0  # k = 0
    U = torch.ones((4, 3), dtype=torch.int8, device="cuda")
    B = torch.ones((3, 5), dtype=torch.uint64, device="cuda")
    with pytest.raises(ModppError):
        pkg.modpp_mm_trunc(U, B, q, drop_bits=60)            # beyond bits(q)
    with pytest.raises(ModppError):
        pkg.modpp_mm_trunc(U, B, q, path="fp64", drop_bits=3)
    with pytest.raises(ModppError):
        pkg.modpp_mm_trunc(U, B, 1 << 40, drop_bits=3)       # even modulus
