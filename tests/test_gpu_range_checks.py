"""GPU tests of the debug-mode value-range checks (modpp_set_debug_checks).

Residue inputs must be canonical (every entry below its prime) and int32
plaintext entries must lie in [-128, 127]; the host cannot see the values, so
in debug mode a device pass reports a violation as MODPP_ERR_RANGE in the
call's status word (the ring's status word for the ring entry points).  Each
test plants one out-of-range value on the host side of the copy -- a value
check, nothing that touches memory out of bounds -- and checks the word; a
valid call afterwards reads MODPP_OK, and with debug mode off the same bad
input is not reported."""
import numpy as np
import pytest
import torch

import ckks_inputs as C
from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu

OK, RANGE = 0, -6


@pytest.fixture
def pkg(cuda_ok):
    import __graft_entry__ as g
    g.build()
    import paper_2503_16080_gb300 as p
    p.set_debug_checks(True)
    assert p.get_debug_checks()
    yield p
    p.set_debug_checks(False)


def _operands(d=64, k=96, n=80, P=2, seed=5):
    primes = synth.ntt_primes(50, P)
    U = torch.from_numpy(synth.uniform_int8(seed, 1, (d, k))).cuda()
    A = np.stack([synth.uniform_mod(seed, 2 + j, (k, n), q) for j, q in enumerate(primes)])
    return primes, U, A


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda().view(torch.uint64)


@pytest.mark.parametrize("path", ["f16", "fp64"])
def test_modpp_mm_residue_at_q(pkg, path):
    primes, U, A = _operands()
    ws = torch.empty(pkg.workspace_bytes(64, 96, 80, primes, path=path), dtype=torch.uint8,
                     device="cuda")
    pkg.modpp_mm(U, _dev(A), primes, path=path, workspace=ws)
    assert pkg.last_status(workspace=ws) == OK
    bad = A.copy()
    bad[1, 7, 5] = primes[1]              # exactly q: not canonical
    pkg.modpp_mm(U, _dev(bad), primes, path=path, workspace=ws)
    assert pkg.last_status(workspace=ws) == RANGE
    pkg.modpp_mm(U, _dev(A), primes, path=path, workspace=ws)   # cleared at the call's start
    assert pkg.last_status(workspace=ws) == OK
    pkg.set_debug_checks(False)
    pkg.modpp_mm(U, _dev(bad), primes, path=path, workspace=ws)
    assert pkg.last_status(workspace=ws) == OK                 # no check without debug mode


@pytest.mark.parametrize("value", [128, -129, 1 << 20])
def test_modpp_mm_int32_plaintext_out_of_range(pkg, value):
    primes, U, A = _operands()
    U32 = U.to(torch.int32)
    ws = torch.empty(pkg.workspace_bytes(64, 96, 80, primes), dtype=torch.uint8, device="cuda")
    pkg.modpp_mm(U32, _dev(A), primes, workspace=ws)
    assert pkg.last_status(workspace=ws) == OK
    U32[3, 90] = value
    pkg.modpp_mm(U32, _dev(A), primes, workspace=ws)
    assert pkg.last_status(workspace=ws) == RANGE


def test_pc_mm_b_part(pkg):
    primes, U, A = _operands(64, 96, 80, 3)
    B = np.stack([synth.uniform_mod(9, 5 + j, (96, 80), q) for j, q in enumerate(primes)])
    ws = torch.empty(pkg.workspace_bytes(64, 96, 80, primes, kind="pc_mm"), dtype=torch.uint8,
                     device="cuda")
    pkg.pc_mm(U, _dev(A), _dev(B), primes, workspace=ws)
    assert pkg.last_status(workspace=ws) == OK
    B[2, 95, 79] = np.uint64(1 << 63)
    pkg.pc_mm(U, _dev(A), _dev(B), primes, workspace=ws)
    assert pkg.last_status(workspace=ws) == RANGE


@pytest.mark.parametrize("mode", ["digits", "crt"])
def test_wide_left_operand(pkg, mode):
    primes = synth.ntt_primes(50, 2)
    d, k, n = 48, 64, 40
    Ures = np.stack([synth.uniform_mod(3, 1 + j, (d, k), q) for j, q in enumerate(primes)])
    A = np.stack([synth.uniform_mod(3, 5 + j, (k, n), q) for j, q in enumerate(primes)])
    pkg.set_wide_path(mode)
    try:
        ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
        pkg.modpp_mm_wide(_dev(Ures), _dev(A), primes, workspace=ws)
        assert pkg.last_status(workspace=ws) == OK
        Ures[0, 1, 2] = primes[0] + 1
        pkg.modpp_mm_wide(_dev(Ures), _dev(A), primes, workspace=ws)
        assert pkg.last_status(workspace=ws) == RANGE
    finally:
        pkg.set_wide_path("auto")


def test_grouped_plan(pkg):
    probs = []
    for i in range(3):
        primes, U, A = _operands(32 + 16 * i, 64, 48, 1 + i, seed=20 + i)
        probs.append((U, _dev(A), primes))
    plan = pkg.GroupedPlan(probs, tune=False)
    plan.run()
    assert plan.status() == OK
    primes, U, A = _operands(40, 64, 48, 2, seed=30)
    A[1, 0, 0] = primes[1]
    probs.append((U, _dev(A), primes))
    bad_plan = pkg.GroupedPlan(probs, tune=False)
    bad_plan.run()
    assert bad_plan.status() == RANGE
    plan.close()
    bad_plan.close()


def test_ring_inputs(pkg):
    from paper_2503_16080_gb300 import ring as ring_mod
    N = 16
    R = ring_mod.Ring(N, C.PRP)
    assert R.status() == OK
    # A raw switching key with one coefficient not below its prime (the
    # special prime's plane): prepare_keys reports it.
    key = synth.uniform_mod(4, 1, (1, len(C.PR), 2, len(C.PR) + 1, N), C.SP)
    for k, q in enumerate(C.PRP):
        key[..., k, :] %= np.uint64(q)
    good_key = _dev(key)
    R.prepare_keys(good_key)
    assert R.status() == OK
    key[0, 1, 0, len(C.PR), 3] = C.SP
    R.prepare_keys(_dev(key))
    assert R.status() == RANGE
    cts = C.rand_cts(8, 4, N, C.PR)
    R.keyswitch(_dev(C.to_batch(cts)), good_key)
    assert R.status() == OK
    cts[2, 1, 1, 7] = C.PR[1]
    R.keyswitch(_dev(C.to_batch(cts)), good_key)
    assert R.status() == RANGE
    assert R.status() == OK                # read clears the word
    R.tweak(_dev(C.to_batch(cts)))
    assert R.status() == RANGE
    R.close()
