"""GPU parity of the CTA-pair form of the tensor-core GEMM (modpp_set_gemm_pair:
tcgen05.mma.cta_group::2, 256-row tiles computed by two CTAs of a cluster,
each staging its own U rows and half of the digit tile), bit-exact against
the oracle on shapes with ragged row, column and inner-dimension tails,
several digit counts, and a PC-MM."""
import numpy as np
import pytest
import torch

from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def pkg(cuda_ok):
    import __graft_entry__ as g
    g.build()
    import paper_2503_16080_gb300 as p
    old = p.get_gemm_pair()
    p.set_gemm_pair(True)
    yield p
    p.set_gemm_pair(old)


@pytest.mark.parametrize("d,k,n,bits,P", [(256, 128, 128, 50, 1), (300, 700, 130, 50, 2),
                                          (1000, 1100, 520, 50, 3), (513, 64, 65, 20, 1),
                                          (640, 900, 300, 62, 2), (384, 512, 200, 36, 2)])
def test_pair_gemm_bit_exact(oracle_mod, pkg, d, k, n, bits, P):
    primes = synth.ntt_primes(bits, P, two_adicity=1 if bits < 30 else 17)
    U = synth.uniform_int8(d + k, 1, (d, k))
    A = np.stack([synth.uniform_mod(d + n, 2 + j, (k, n), q) for j, q in enumerate(primes)])
    got = pkg.modpp_mm(torch.from_numpy(U).cuda(), torch.from_numpy(A).cuda(), primes)
    assert pkg.last_status() == 0
    assert np.array_equal(got.cpu().numpy(), oracle_mod.mod_pp_mm(U.astype(np.int32), A, primes))


def test_pair_pc_mm(oracle_mod, pkg):
    primes = synth.ntt_primes(50, 3)
    d = kct = N = 512
    U = synth.uniform_int8(9, 1, (d, kct))
    A = np.stack([synth.uniform_mod(9, 2 + j, (kct, N), q) for j, q in enumerate(primes)])
    B = np.stack([synth.uniform_mod(9, 6 + j, (kct, N), q) for j, q in enumerate(primes)])
    Ao, Bo = pkg.pc_mm(torch.from_numpy(U).cuda(), torch.from_numpy(A).cuda(),
                       torch.from_numpy(B).cuda(), primes)
    U32 = U.astype(np.int32)
    assert np.array_equal(Ao.cpu().numpy(), oracle_mod.mod_pp_mm(U32, A, primes))
    assert np.array_equal(Bo.cpu().numpy(), oracle_mod.mod_pp_mm(U32, B, primes))
