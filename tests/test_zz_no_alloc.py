"""GPU test of modpp_mm_static, the Mod-PP-MM entry point for callers that
cannot allocate device memory (for example, applications whose memory manager
owns the whole GPU, or plugin hosts that forbid device allocation on the call
path).  It uses a fixed scratch array inside the library instead of a caller
workspace.

The test calls it through the C ABI twice in a row and checks each result,
element by element, against the regular entry point (modpp_mm with a caller
workspace).  It also checks that a request larger than the fixed scratch is
rejected before anything runs.  This file is named so that pytest collects it
last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_16080_gb300 import synth

pytestmark = pytest.mark.gpu

WORKSPACE_ERROR = -3


def test_static_scratch_entry_point_matches_regular_entry_point(cuda_ok):
    import paper_2503_16080_gb300 as pkg

    lib = pkg.lib()
    fn = lib.modpp_mm_static
    I64, P = ctypes.c_int64, ctypes.c_void_p
    fn.argtypes = [I64, I64, I64, P, ctypes.c_int, I64, P, I64, I64, P, I64, I64, P,
                   ctypes.c_int, P]
    fn.restype = ctypes.c_int
    lib.modpp_mm_static_capacity.restype = ctypes.c_size_t
    capacity = lib.modpp_mm_static_capacity()
    assert capacity == 64 << 20

    primes = synth.ntt_primes(50, 2)
    d, k, n = 300, 700, 130
    U = torch.from_numpy(synth.uniform_int8(77, 1, (d, k))).cuda()
    A = torch.from_numpy(np.stack([synth.uniform_mod(77, 2 + j, (k, n), q)
                                   for j, q in enumerate(primes)])).cuda()
    expected = pkg.modpp_mm(U, A, primes)  # regular entry point, caller workspace
    torch.cuda.synchronize()
    assert pkg.workspace_bytes(d, k, n, primes) <= capacity

    pr = np.ascontiguousarray(primes, dtype=np.uint64)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.from_numpy(np.full((2, d, n), 0xDEADBEEF, dtype=np.uint64)).cuda()
        rc = fn(d, k, n, U.data_ptr(), 0, k, A.data_ptr(), n, k * n, out.data_ptr(), n, d * n,
                pr.ctypes.data, 2, stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(out, expected)

    # 8192^3 needs about 1 GB of scratch: rejected before any pointer is used.
    big = 8192
    assert pkg.workspace_bytes(big, big, big, primes) > capacity
    rc = fn(big, big, big, 256, 0, big, 256, big, big * big, 256, big, big * big,
            pr.ctypes.data, 2, stream)
    assert rc == WORKSPACE_ERROR
