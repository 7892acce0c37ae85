"""GPU test of modpp_mm_static, the Mod-PP-MM entry point for callers that
cannot allocate device memory (for example, applications whose memory manager
owns the whole GPU, or plugin hosts that forbid device allocation on the call
path).  It uses a fixed scratch array inside the library instead of a caller
workspace.

The test calls it through the C ABI twice in a row and checks each result,
element by element, against the regular entry point (modpp_mm with a caller
workspace) and against the oracle, and reads the device status word of the
static array after each call.  It also checks the documented edge cases and
error codes: k = 0 writes zeros, d = 0 is a no-op, a bad prime is
MODPP_ERR_PRIME, and a request larger than the fixed scratch is rejected
before anything runs.  This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu

OK, PRIME_ERROR, WORKSPACE_ERROR = 0, -2, -3


def _entry_points(pkg):
    lib = pkg.lib()
    fn = lib.modpp_mm_static
    I64, P = ctypes.c_int64, ctypes.c_void_p
    fn.argtypes = [I64, I64, I64, P, ctypes.c_int, I64, P, I64, I64, P, I64, I64, P,
                   ctypes.c_int, P]
    fn.restype = ctypes.c_int
    lib.modpp_mm_static_capacity.restype = ctypes.c_size_t
    lib.modpp_mm_static_status.argtypes = [P]
    lib.modpp_mm_static_status.restype = ctypes.c_int
    return fn, lib


def test_static_scratch_entry_point_matches_regular_entry_point(cuda_ok, oracle_mod):
    import paper_2503_16080_gb300 as pkg

    fn, lib = _entry_points(pkg)
    capacity = lib.modpp_mm_static_capacity()
    assert capacity == 64 << 20

    primes = synth.ntt_primes(50, 2)
    d, k, n = 300, 700, 130
    U_np = synth.uniform_int8(77, 1, (d, k))
    A_np = np.stack([synth.uniform_mod(77, 2 + j, (k, n), q) for j, q in enumerate(primes)])
    U = torch.from_numpy(U_np).cuda()
    A = torch.from_numpy(A_np).cuda()
    expected = pkg.modpp_mm(U, A, primes)  # regular entry point, caller workspace
    torch.cuda.synchronize()
    want = oracle_mod.mod_pp_mm(U_np.astype(np.int32), A_np, primes)
    assert np.array_equal(expected.cpu().numpy(), want)
    assert pkg.workspace_bytes(d, k, n, primes) <= capacity

    pr = np.ascontiguousarray(primes, dtype=np.uint64)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.from_numpy(np.full((2, d, n), 0xDEADBEEF, dtype=np.uint64)).cuda()
        rc = fn(d, k, n, U.data_ptr(), 0, k, A.data_ptr(), n, k * n, out.data_ptr(), n, d * n,
                pr.ctypes.data, 2, stream)
        assert rc == OK
        assert lib.modpp_mm_static_status(stream) == OK
        torch.cuda.synchronize()
        assert torch.equal(out, expected)
        assert np.array_equal(out.cpu().numpy(), want)

    # k = 0: the product is empty, every output is 0.
    out = torch.from_numpy(np.full((2, d, n), 5, dtype=np.uint64)).cuda()
    rc = fn(d, 0, n, U.data_ptr(), 0, 0, A.data_ptr(), n, 0, out.data_ptr(), n, d * n,
            pr.ctypes.data, 2, stream)
    assert rc == OK and lib.modpp_mm_static_status(stream) == OK
    assert int(out.view(torch.int64).abs().sum()) == 0
    # d = 0: nothing to compute.
    rc = fn(0, k, n, U.data_ptr(), 0, k, A.data_ptr(), n, k * n, out.data_ptr(), n, 0,
            pr.ctypes.data, 2, stream)
    assert rc == OK
    torch.cuda.synchronize()

    # An even "prime": the prime error of modpp_mm, before anything runs.
    bad = np.array([primes[0], 1 << 40], dtype=np.uint64)
    rc = fn(d, k, n, U.data_ptr(), 0, k, A.data_ptr(), n, k * n, out.data_ptr(), n, d * n,
            bad.ctypes.data, 2, stream)
    assert rc == PRIME_ERROR

    # 8192^3 needs about 1 GB of scratch: rejected before any pointer is used.
    big = 8192
    assert pkg.workspace_bytes(big, big, big, primes) > capacity
    rc = fn(big, big, big, 256, 0, big, 256, big, big * big, 256, big, big * big,
            pr.ctypes.data, 2, stream)
    assert rc == WORKSPACE_ERROR
