"""CPU-side checks of the C ABI: the library loads, exports every function that
the headers under include/ declare, and its host logic (planning, workspace sizes,
argument validation) behaves as documented.  No call here reaches the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2503_16080_gb300 import build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADERS = sorted(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h"))


@pytest.fixture(scope="module")
def api():
    build.build()
    from paper_2503_16080_gb300 import api as a
    return a


def declared_functions():
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("modpp_mm", "modpp_mm_workspace", "pc_mm", "pc_mv", "pc_mm_workspace",
                     "modpp_plan_info", "modpp_status_read", "modpp_status_string", "cc_mm",
                     "cc_mm_workspace", "modpp_transpose", "modpp_tweak", "modpp_keyswitch",
                     "modpp_ring_create"):
        assert required in names


def test_library_exports_every_declared_symbol(api):
    L = ctypes.CDLL(api.library_path())
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(api):
    L = api.lib()
    assert L.modpp_status_string(0) == b"MODPP_OK"
    for code in range(-1, -8, -1):
        assert L.modpp_status_string(code).startswith(b"MODPP_ERR")
    assert L.modpp_abi_version() >> 16 == 1


@pytest.mark.parametrize("b", [8, 9, 10])
@pytest.mark.parametrize("bits", [8, 9, 10, 11, 40, 41, 50, 51, 60, 61, 62])
def test_f16_digit_counts(api, b, bits):
    q = synth.ntt_primes(bits, 1, two_adicity=1 if bits <= 11 else 17)[0]
    api.set_digit_bits(b)
    try:
        info = api.plan_info(4096, q, "f16")
    finally:
        api.set_digit_bits(0)
    # L balanced b-bit digits cover 2^(bL) consecutive integers: need q <= 2^(bL).
    L = -(-(q - 1).bit_length() // b)
    assert info == {"digits": L, "digit_bits": b, "k_chunk": 2 ** (18 - b)}
    assert q <= 2 ** (b * L) and q > 2 ** (b * (L - 1))
    # The chunk bound: chunk * 128 * 2^(b-1) = 2^24, the exact-integer range of binary32.
    assert info["k_chunk"] * 128 * 2 ** (b - 1) == 2 ** 24


def test_digit_bits_setting(api):
    assert api.get_digit_bits() in (8, 9, 10)
    with pytest.raises(api.ModppError):
        api.set_digit_bits(7)
    with pytest.raises(api.ModppError):
        api.set_digit_bits(11)
    api.set_digit_bits(10)
    assert api.get_digit_bits() == 10
    api.set_digit_bits(0)


def test_fp64_plan_matches_lemma(api):
    # Lemma le:strategy1 at d2 = 2^12: K = 1482910 (2^20.5), three digits for 50..62-bit q.
    for bits in (50, 54, 62):
        q = synth.ntt_primes(bits, 1)[0]
        info = api.plan_info(4096, q, "fp64")
        assert info["digits"] == 3 and info["digit_bits"] == 20 and info["k_chunk"] == 4096
    q = synth.ntt_primes(50, 1)[0]
    tight = api.plan_info(4096, q, "fp64_tight")  # base floor(2^53 / 2^19) = 2^34
    assert tight["digits"] == 2 and tight["digit_bits"] == 34


def test_workspace_sizes(api):
    q = synth.ntt_primes(50, 3)
    L = api.plan_info(4096, q[0])["digits"]
    # Tile columns per digit count (UMMA N = L * nc between 192 and 256).
    nc = 64 if L <= 3 else 48 if L <= 5 else 40 if L == 6 else 32
    nb = -(-4096 // nc)
    # f16: 256 B header + U16 (d x kp halves) + digits (planes x n_blocks x L x nc x kp halves)
    ws = api.workspace_bytes(4096, 4096, 4096, q[:1])
    assert ws == 256 + 4096 * 4096 * 2 + nb * L * nc * 4096 * 2
    pc = api.workspace_bytes(4096, 4096, 4096, q, kind="pc_mm")
    assert pc == 256 + 4096 * 4096 * 2 + 6 * nb * L * nc * 4096 * 2
    assert api.workspace_bytes(-1, 4, 4, q[:1]) == 0
    assert api.workspace_bytes(4, 4, 4, [4]) == 0


def _call(api, d=4, k=4, n=4, U=1, A=1, C=1, primes=(97,), path=0, ws=256, ws_bytes=1 << 20,
          ldu=None, lda=None, ldc=None, ukind=0):
    pr = np.ascontiguousarray(primes, dtype=np.uint64)
    return api.lib().modpp_mm(d, k, n, U, ukind, k if ldu is None else ldu, A,
                              n if lda is None else lda, k * n, C, n if ldc is None else ldc,
                              d * n, pr.ctypes.data if len(pr) else None, len(pr), path, ws,
                              ws_bytes, None)


def test_argument_errors_before_any_launch(api):
    ARG, PRIME, WS = -1, -2, -3
    assert _call(api, d=-1) == ARG
    assert _call(api, k=(1 << 20) + 1) == ARG
    assert _call(api, U=None) == ARG
    assert _call(api, A=None) == ARG
    assert _call(api, C=None) == ARG
    assert _call(api, ldu=3) == ARG
    assert _call(api, lda=3) == ARG
    assert _call(api, ldc=2) == ARG
    assert _call(api, ukind=7) == ARG
    assert _call(api, path=9) == ARG
    assert _call(api, primes=()) == ARG
    assert _call(api, primes=(98,)) == PRIME
    assert _call(api, primes=(1,)) == PRIME
    assert _call(api, primes=((1 << 62) + 1,)) == PRIME
    assert _call(api, primes=tuple([97] * 33)) == ARG
    assert _call(api, ws=None) == WS
    assert _call(api, ws=128) == WS          # not 256-byte aligned
    assert _call(api, ws_bytes=16) == WS     # too small


def test_static_entry_point_argument_errors_before_any_cuda_call(api):
    # modpp_mm_static checks its arguments with modpp_mm's codes before it
    # looks up its scratch array (no GPU here: a CUDA call would fail).
    L = api.lib()
    fn = L.modpp_mm_static
    I64, P = ctypes.c_int64, ctypes.c_void_p
    fn.argtypes = [I64, I64, I64, P, ctypes.c_int, I64, P, I64, I64, P, I64, I64, P,
                   ctypes.c_int, P]

    def call(d=4, k=4, n=4, primes=(97,), U=1, ldc=None):
        pr = np.ascontiguousarray(primes, dtype=np.uint64)
        return fn(d, k, n, U, 0, k, 1, n, k * n, 1, n if ldc is None else ldc, d * n,
                  pr.ctypes.data, len(pr), None)
    assert call(d=-1) == -1
    assert call(U=None) == -1
    assert call(ldc=3) == -1
    assert call(primes=(98,)) == -2
    assert call(primes=(97, 1 << 40)) == -2
    assert call(d=8192, k=8192, n=8192) == -3     # needs more than the 64 MiB array


def test_gemm_pair_setting(api):
    assert api.get_gemm_pair() in (False, True)
    old = api.get_gemm_pair()
    try:
        api.set_gemm_pair(True)
        assert api.get_gemm_pair()
        q = synth.ntt_primes(50, 3)
        # the pair tiles (32 columns at 6 digits) change the workspace layout
        assert api.workspace_bytes(4096, 4096, 4096, q) == 256 + 4096 * 4096 * 2 + \
            3 * 128 * 6 * 32 * 4096 * 2
        api.set_gemm_pair(False)
        assert not api.get_gemm_pair()
    finally:
        api.set_gemm_pair(old)
    assert api.lib().modpp_set_gemm_pair(2) == -1


def test_debug_checks_setting(api):
    assert not api.get_debug_checks()
    api.set_debug_checks(True)
    try:
        assert api.get_debug_checks()
    finally:
        api.set_debug_checks(False)
    assert not api.get_debug_checks()
    assert api.lib().modpp_set_debug_checks(2) == -1
    assert api.lib().modpp_ring_status_read(None, None) == -1


def test_pc_argument_errors(api):
    L = api.lib()
    pr = np.ascontiguousarray([97] * 17, dtype=np.uint64)
    assert L.pc_mm(4, 4, 4, 1, 1, 1, 1, 1, pr.ctypes.data, 17, 0, 256, 1 << 20, None) == -1
    assert L.pc_mv(4, 4, 4, 1, None, 1, 1, 1, pr.ctypes.data, 1, 0, 256, 1 << 20, None) == -1
    assert L.modpp_status_read(None, None) == -3


# ---------------------------------------------------------------- ring / CC-MM ABI (host side)

def _ring_lib(api):
    from paper_2503_16080_gb300 import ring
    return ring._register()


def test_ring_bytes_sizes(api):
    L = _ring_lib(api)
    assert L.modpp_ring_bytes(16, 3) > 0
    assert L.modpp_ring_bytes(8192, 4) > L.modpp_ring_bytes(4096, 4) > 0
    for N, Lc in ((12, 3), (1, 3), (32768, 3), (16, 0), (16, 17)):
        assert L.modpp_ring_bytes(N, Lc) == 0, (N, Lc)


def test_ring_bytes_gadgets(api):
    # Gadgets of dnum digits of at most two chain primes (every digit
    # non-empty) and one or two special primes; anything else is rejected.
    L = _ring_lib(api)
    assert L.modpp_ring_bytes_ks(16, 3, 1, 3) == L.modpp_ring_bytes(16, 3)
    for Lc, K, dnum in ((4, 2, 2), (3, 2, 2), (4, 2, 4), (2, 2, 1), (4, 1, 2), (16, 2, 8)):
        assert L.modpp_ring_bytes_ks(8192, Lc, K, dnum) > 0, (Lc, K, dnum)
    # two special primes need more table space than one
    assert L.modpp_ring_bytes_ks(8192, 4, 2, 2) > L.modpp_ring_bytes_ks(8192, 4, 1, 2)
    for Lc, K, dnum in ((4, 3, 2), (4, 0, 2), (4, 2, 0), (4, 2, 5), (5, 2, 2), (6, 2, 2),
                        (4, 2, 1), (17, 2, 9)):
        assert L.modpp_ring_bytes_ks(16, Lc, K, dnum) == 0, (Lc, K, dnum)


def test_ring_create_validates_before_touching_memory(api):
    import ctypes
    L = _ring_lib(api)
    good = synth.ntt_primes(50, 3) + synth.ntt_primes(60, 1)
    h = ctypes.c_void_p()

    def create(N, primes, mem=None, nbytes=0):
        arr = np.ascontiguousarray(primes, dtype=np.uint64)
        return L.modpp_ring_create(N, len(primes) - 1, arr.ctypes.data, mem, nbytes, None,
                                   ctypes.byref(h))
    assert create(12, good) == -1                      # N not a power of two
    assert create(16, good[:3] + [good[0]]) == -2      # repeated prime
    assert create(16, good[:3] + [good[3] + 2]) == -2  # not prime / not 1 mod 2N
    assert create(16, good[:3] + [(1 << 62) + 1]) == -2
    nt = [q for q in synth.ntt_primes(40, 4, two_adicity=1) if (q - 1) % 32 != 0]
    if nt:
        assert create(16, good[:3] + nt[:1]) == -2     # prime, but not 1 mod 2N
    assert create(16, good) == -3                      # valid, but no memory given
    assert not h.value


def test_wide_path_setting_and_plan(api):
    q = synth.ntt_primes(50, 4)
    api.set_wide_path("auto")
    assert api.get_wide_path() == 0
    assert api.wide_plan_info(8192, q) == 16          # CRT form: four pieces of k, 16 primes
    assert api.wide_plan_info(16384, q) == 19         # four pieces of 4096: primes <= 127
    assert api.wide_plan_info(1 << 20, q) == 0        # no prime set: digit form
    api.set_wide_path("digits")
    try:
        assert api.wide_plan_info(8192, q) == 0
    finally:
        api.set_wide_path("auto")
    with pytest.raises(api.ModppError):
        api.set_wide_path(3)
