"""GPU parity of Alg. 7 (CP-MM with precomputation) with the key switches
back to one secret (pc_mm_precomp), bit-exact against the oracle: the one
Mod-PP-MM B * U per chain prime, the key switches of a batch sharing one
a-part (its digits transformed once), and the optional Rescale.  N = 1024
runs the register-blocked NTTs; smaller N the per-stage ones."""
import numpy as np
import pytest
import torch

import ckks_inputs as C
from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("N,d2,d3,rescale", [(16, 16, 16, False), (16, 7, 3, True),
                                             (64, 64, 20, False), (256, 256, 33, True),
                                             (1024, 1024, 16, False), (1024, 300, 5, True)])
def test_pc_mm_precomp_bit_exact(oracle_mod, ring_mod, N, d2, d3, rescale):
    seed = N + d3
    secrets = [synth.ternary(seed, 100 + j, N) for j in range(d2)]
    s = synth.ternary(seed, 99, N)
    U = synth.uniform_int8(seed, 1, (d2, d3))
    keys, _ = C.precomp_keys(oracle_mod, secrets, U, s, N, 700 + seed)
    M = synth.uniform_unit(seed, 2, (N, d2))
    cts, _, _ = C.encrypt_shared_a(oracle_mod, M, secrets, 2.0 ** 40, seed + 1)
    want, _ = oracle_mod.pcmm_precomp(cts, U, keys, C.PRP, rescale_out=rescale)
    R = ring_mod.Ring(N, C.PRP)
    L = len(C.PR)
    dk = R.prepare_keys(dev(np.stack(keys)))
    a = dev(cts[0, 0])                                           # (L, N)
    B = dev(np.transpose(cts[:, 1], (1, 0, 2)))                  # (L, d2, N)
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
    got = R.pc_mm_precomp(Ut, a, B, dk, rescale=rescale)
    assert tuple(got.shape) == (2, L - 1 if rescale else L, d3, N)
    assert np.array_equal(C.from_batch(host(got)), want)


def test_pc_mm_precomp_rejects_bad_arguments(ring_mod):
    from paper_2503_16080_gb300.api import lib
    N = 16
    R = ring_mod.Ring(N, C.PRP)
    assert lib().pc_mm_precomp_workspace(R._h, 0, 4, 0) == 0
    assert lib().pc_mm_precomp_workspace(R._h, 4, 0, 0) == 0
    assert lib().pc_mm_precomp_workspace(R._h, 4, 4, 2) == 0
    assert lib().pc_mm_precomp_workspace(R._h, 4, 4, 1) > lib().pc_mm_precomp_workspace(R._h, 4, 4, 0)
