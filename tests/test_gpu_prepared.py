"""GPU parity of the prepared-plaintext entry points (modpp_u_to_f16 +
pc_mm_u16): PC-MM and PC-Mv with U converted once are bit-exact against the
oracle and identical to the per-call conversion, for int8 and int32 U, ragged
shapes, both GEMM forms, and the full-size PC-Mv shape (16384^2 x 32)."""
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


@pytest.mark.parametrize("d,kct,N,P,kind", [(300, 700, 32, 2, "i8"), (513, 1000, 200, 3, "i8"),
                                            (129, 77, 65, 1, "i32"), (1, 1, 1, 1, "i8")])
def test_prepared_u_bit_exact(oracle_mod, pkg, d, kct, N, P, kind):
    primes = synth.ntt_primes(50, P)
    U = synth.uniform_int8(d, 1, (d, kct))
    A = np.stack([synth.uniform_mod(d, 2 + j, (kct, N), q) for j, q in enumerate(primes)])
    B = np.stack([synth.uniform_mod(d, 9 + j, (kct, N), q) for j, q in enumerate(primes)])
    Ut = torch.from_numpy(U).cuda()
    prep = pkg.PreparedU(Ut if kind == "i8" else Ut.to(torch.int32))
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    fn = pkg.pc_mv if N <= 32 else pkg.pc_mm
    Ao, Bo = fn(prep, At, Bt, primes)
    U32 = U.astype(np.int32)
    assert np.array_equal(Ao.cpu().numpy(), oracle_mod.mod_pp_mm(U32, A, primes))
    assert np.array_equal(Bo.cpu().numpy(), oracle_mod.mod_pp_mm(U32, B, primes))
    Ar, Br = fn(Ut, At, Bt, primes)
    assert torch.equal(Ao, Ar) and torch.equal(Bo, Br)


def test_prepared_u_pcmv_full_size(pkg):
    d = kct = 16384
    primes = synth.ntt_primes(50, 4)
    U = synth.uniform_int8_torch(21, 1, (d, kct), "cuda")
    A = torch.stack([synth.uniform_mod_torch(21, 10 + j, (kct, 32), q, "cuda")
                     for j, q in enumerate(primes)])
    B = torch.stack([synth.uniform_mod_torch(21, 20 + j, (kct, 32), q, "cuda")
                     for j, q in enumerate(primes)])
    prep = pkg.PreparedU(U)
    Ao, Bo = pkg.pc_mv(prep, A, B, primes)
    Ar, Br = pkg.pc_mv(U, A, B, primes)
    assert torch.equal(Ao, Ar) and torch.equal(Bo, Br)
    assert pkg.last_status() == 0


def test_prepared_u_rejects_fp64_path(pkg):
    U = torch.ones((4, 4), dtype=torch.int8, device="cuda")
    A = torch.zeros((1, 4, 4), dtype=torch.uint64, device="cuda")
    with pytest.raises(ValueError):
        pkg.pc_mm(pkg.PreparedU(U), A, A, synth.ntt_primes(50, 1), path="fp64")
