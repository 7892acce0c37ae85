"""ctypes binding of ``libmodpp.so`` (C ABI in ``include/modpp.h``).

Argument marshalling only: tensors are passed as device pointers with their
sizes and strides, the stream is PyTorch's current CUDA stream, and the
caller-side workspace is a PyTorch allocation.  All arithmetic runs in the
library's CUDA kernels.  If the library was not built, every call raises
``ModppError``; there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import enum
import os
import threading
from typing import Sequence

import numpy as np
import torch

from .build import LIB_PATH

__all__ = ["ModppError", "Path", "lib", "library_path", "modpp_mm", "pc_mm", "pc_mv",
           "plan_info", "workspace_bytes", "last_status"]


class ModppError(RuntimeError):
    """A library call returned a negative modpp_status."""

    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_status_string(code)} ({code})")


class Path(enum.IntEnum):
    F16 = 0          # exact f16 digits on tcgen05 (default)
    FP64 = 1         # Strategy 1, base floor(sqrt(2^53/k)), cuBLAS DGEMM
    FP64_TIGHT = 2   # Strategy 1 with the asymmetric base floor(2^53/(128k))


_PATH_NAMES = {"f16": Path.F16, "fp64": Path.FP64, "fp64_tight": Path.FP64_TIGHT}

_lib = None
_lib_lock = threading.Lock()


def library_path() -> str:
    return LIB_PATH


def lib() -> ctypes.CDLL:
    """Load the compiled library (raises ModppError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ModppError(-5, f"libmodpp.so not built at {LIB_PATH} "
                                 "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I, U64, SZ = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                              ctypes.c_size_t)
        L.modpp_status_string.argtypes = [I]
        L.modpp_status_string.restype = ctypes.c_char_p
        L.modpp_abi_version.restype = I
        L.modpp_plan_info.argtypes = [I64, U64, I, P, P, P]
        L.modpp_mm_workspace.argtypes = [I64, I64, I64, P, I, I]
        L.modpp_mm_workspace.restype = SZ
        L.modpp_mm.argtypes = [I64, I64, I64, P, I, I64, P, I64, I64, P, I64, I64, P, I, I, P, SZ, P]
        L.pc_mm_workspace.argtypes = [I64, I64, I64, P, I, I]
        L.pc_mm_workspace.restype = SZ
        L.pc_mm.argtypes = [I64, I64, I64, P, P, P, P, P, P, I, I, P, SZ, P]
        L.pc_mv.argtypes = [I64, I64, I64, P, P, P, P, P, P, I, I, P, SZ, P]
        L.modpp_u16_bytes.argtypes = [I64, I64]
        L.modpp_u16_bytes.restype = SZ
        L.modpp_u_to_f16.argtypes = [I64, I64, P, I, I64, P, P]
        L.pc_mm_u16.argtypes = [I64, I64, I64, P, P, P, P, P, P, I, P, SZ, P]
        L.modpp_status_read.argtypes = [P, P]
        L.modpp_selftest_bounded_wait.argtypes = [P, ctypes.c_uint64, P]
        L.modpp_mm_wide_workspace.argtypes = [I64, I64, I64, P, I]
        L.modpp_mm_wide_workspace.restype = SZ
        L.modpp_mm_wide.argtypes = [I64, I64, I64, P, I64, I64, P, I64, I64, P, I64, I64, P, I, P,
                                    SZ, P]
        L.modpp_group_workspace.argtypes = [P, I]
        L.modpp_group_workspace.restype = SZ
        L.modpp_group_plan_create.argtypes = [P, I, P, SZ, I, P, P]
        L.modpp_group_run.argtypes = [P, P]
        L.modpp_group_run_graph.argtypes = [P, P]
        L.modpp_group_plan_info.argtypes = [P, P, P, P, P]
        L.modpp_group_plan_destroy.argtypes = [P]
        L.modpp_group_plan_destroy.restype = None
        L.modpp_set_digit_bits.argtypes = [I]
        L.modpp_get_digit_bits.restype = I
        L.modpp_set_wide_path.argtypes = [I]
        L.modpp_get_wide_path.restype = I
        L.modpp_wide_plan_info.argtypes = [I64, P, I, P]
        L.modpp_mm_trunc_workspace.argtypes = [I64, I64, I64, U64, I, I]
        L.modpp_mm_trunc_workspace.restype = SZ
        L.modpp_mm_trunc.argtypes = [I64, I64, I64, P, I, I64, P, I64, P, I64, U64, I, I, P, SZ,
                                     P]
        L.modpp_set_gemm_pair.argtypes = [I]
        L.modpp_get_gemm_pair.restype = I
        L.modpp_set_debug_checks.argtypes = [I]
        L.modpp_get_debug_checks.restype = I
        L.modpp_profile_enable.argtypes = [I]
        L.modpp_profile_read.argtypes = [I, P, P]
        _lib = L
        return L


def _status_string(code: int) -> str:
    try:
        return lib().modpp_status_string(int(code)).decode()
    except ModppError:
        return "library not loaded"


def _path(path) -> int:
    if isinstance(path, str):
        return int(_PATH_NAMES[path.lower()])
    return int(Path(path))


class _Primes:
    """A uint64 array of primes and its address, kept alive by the cache below."""
    __slots__ = ("arr", "data")

    def __init__(self, key: tuple):
        self.arr = np.ascontiguousarray(key, dtype=np.uint64)
        self.data = self.arr.ctypes.data

    def __len__(self) -> int:
        return len(self.arr)


# Prime lists seen so far: building the array and reading its address cost
# microseconds per call, which show in the small, latency-bound products.
_primes_cache: dict[tuple, _Primes] = {}


def _primes_arr(primes: Sequence[int]) -> _Primes:
    key = tuple(int(q) for q in primes)
    hit = _primes_cache.get(key)
    if hit is None:
        if len(_primes_cache) > 256:
            _primes_cache.clear()
        hit = _primes_cache[key] = _Primes(key)
    return hit


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


# Grow-only workspace cache, one per device.  Calls that share a device and
# run on different streams must pass their own workspace.
_ws_cache: dict[int, torch.Tensor] = {}


def _workspace(nbytes: int, device: torch.device, workspace: torch.Tensor | None) -> tuple[int, int]:
    if workspace is not None:
        ptr = workspace.data_ptr()
        if workspace.device != device or ptr % 256 or workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError("workspace: wrong device, misaligned or too small")
        return ptr, workspace.numel() * workspace.element_size()
    idx = device.index if device.index is not None else torch.cuda.current_device()
    buf = _ws_cache.get(idx)
    if buf is None or buf.numel() < nbytes:
        _ws_cache.pop(idx, None)
        buf = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=device)
        _ws_cache[idx] = buf
    assert buf.data_ptr() % 256 == 0
    return buf.data_ptr(), buf.numel()


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ModppError(rc, what)


def plan_info(k: int, q: int, path="f16") -> dict:
    """Digit split chosen for inner dimension k and prime q (host only)."""
    dg, bits, chunk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(lib().modpp_plan_info(int(k), int(q), _path(path), ctypes.byref(dg), ctypes.byref(bits),
                                 ctypes.byref(chunk)), "modpp_plan_info")
    return {"digits": dg.value, "digit_bits": bits.value, "k_chunk": chunk.value}


def workspace_bytes(d: int, k: int, n: int, primes: Sequence[int], path="f16",
                    kind: str = "modpp_mm") -> int:
    pr = _primes_arr(primes)
    fn = lib().modpp_mm_workspace if kind == "modpp_mm" else lib().pc_mm_workspace
    return int(fn(int(d), int(k), int(n), pr.data, len(pr), _path(path)))


def last_status(device: torch.device | int | None = None, stream=None,
                workspace: torch.Tensor | None = None) -> int:
    """Device status word of the last call that used this workspace (syncs the stream)."""
    if workspace is None:
        dev = torch.device("cuda", device if isinstance(device, int) else
                           (device.index if device is not None and device.index is not None
                            else torch.cuda.current_device()))
        workspace = _ws_cache.get(dev.index)
        if workspace is None:
            return 0
    return int(lib().modpp_status_read(ctypes.c_void_p(workspace.data_ptr()),
                                       ctypes.c_void_p(_stream_handle(stream))))


def selftest_bounded_wait(limit_ms: float = 10.0, device=None) -> int:
    """Runs the library's bounded-wait self-test (a device wait that nothing
    satisfies, limited to limit_ms) and returns the status word it leaves:
    MODPP_ERR_TIMEOUT (-7) when the wait gave up as designed."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)
    _check(lib().modpp_selftest_bounded_wait(ctypes.c_void_p(ws.data_ptr()),
                                             int(limit_ms * 1e6), ctypes.c_void_p(st.cuda_stream)),
           "modpp_selftest_bounded_wait")
    return int(lib().modpp_status_read(ctypes.c_void_p(ws.data_ptr()),
                                       ctypes.c_void_p(st.cuda_stream)))


KERNEL_GEMM, KERNEL_SPLIT, KERNEL_U16 = 0, 1, 2


def set_digit_bits(bits: int) -> None:
    """Digit width b in {8, 9, 10} of the f16 path (0 = default); process-wide."""
    _check(lib().modpp_set_digit_bits(int(bits)), "modpp_set_digit_bits")


def set_wide_path(mode) -> None:
    """Form of modpp_mm_wide's products: "auto" (0), "digits" (1) or "crt" (2)."""
    m = {"auto": 0, "digits": 1, "crt": 2}.get(mode, mode)
    _check(lib().modpp_set_wide_path(int(m)), "modpp_set_wide_path")


def get_wide_path() -> int:
    return int(lib().modpp_get_wide_path())


def wide_plan_info(k: int, primes: Sequence[int]) -> int:
    """Small primes of the CRT form for inner dimension k (0: digit form)."""
    pr = _primes_arr(primes)
    out = ctypes.c_int()
    _check(lib().modpp_wide_plan_info(int(k), pr.data, len(pr), ctypes.byref(out)),
           "modpp_wide_plan_info")
    return out.value


def set_gemm_pair(on: bool) -> None:
    """Kernel form of the f16 path for single-problem products: CTA pairs
    (tcgen05 cta_group::2, 256-row tiles) or one CTA per 128-row tile."""
    _check(lib().modpp_set_gemm_pair(1 if on else 0), "modpp_set_gemm_pair")


def get_gemm_pair() -> bool:
    return bool(lib().modpp_get_gemm_pair())


def set_debug_checks(on: bool) -> None:
    """Debug mode: device-side value-range checks of every call's inputs,
    reported as MODPP_ERR_RANGE in the call's status word (process-wide)."""
    _check(lib().modpp_set_debug_checks(1 if on else 0), "modpp_set_debug_checks")


def get_debug_checks() -> bool:
    return bool(lib().modpp_get_debug_checks())


def get_digit_bits() -> int:
    return int(lib().modpp_get_digit_bits())


def profile_enable(on: bool) -> None:
    """Bracket every launch of the library's kernels with CUDA events (measurement)."""
    _check(lib().modpp_profile_enable(1 if on else 0), "modpp_profile_enable")


def profile_read(kernel: int) -> tuple[float, int]:
    """(total milliseconds, launches) recorded for `kernel` since the last read."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().modpp_profile_read(int(kernel), ctypes.byref(ms), ctypes.byref(n)),
           "modpp_profile_read")
    return ms.value, n.value


def _check_residues(A: torch.Tensor, name: str) -> None:
    if not A.is_cuda or A.dtype != torch.uint64:
        raise TypeError(f"{name} must be a CUDA uint64 tensor")


def modpp_mm(U: torch.Tensor, A: torch.Tensor, primes: Sequence[int], *, path="f16",
             out: torch.Tensor | None = None, stream=None,
             workspace: torch.Tensor | None = None) -> torch.Tensor:
    """C[j] = U @ A[j] mod primes[j] (exact), on the GPU.

    U: (d, k) int8 or int32 CUDA tensor with values in [-128, 127], unit stride along k.
    A: (P, k, n) (or (k, n)) uint64 CUDA tensor of canonical residues, unit stride along n.
    Returns (P, d, n) (or (d, n)) uint64.
    """
    squeeze = A.dim() == 2
    A3 = A.unsqueeze(0) if squeeze else A
    _check_residues(A3, "A")
    if not U.is_cuda or U.dtype not in (torch.int8, torch.int32) or U.dim() != 2:
        raise TypeError("U must be a 2-D CUDA int8 or int32 tensor")
    if (U.numel() and U.stride(1) != 1) or (A3.numel() and A3.stride(2) != 1):
        raise ValueError("U and A need unit stride along their last dimension")
    P, k, n = A3.shape
    d = U.shape[0]
    if U.shape[1] != k or len(primes) != P:
        raise ValueError("shape mismatch between U, A and primes")
    if out is None:
        out = torch.empty((P, d, n), dtype=torch.uint64, device=A3.device)
    out3 = out.unsqueeze(0) if out.dim() == 2 else out
    if out3.shape != (P, d, n) or out3.stride(2) != 1:
        raise ValueError("out must be (P, d, n) with unit stride along n")
    pr = _primes_arr(primes)
    p = _path(path)
    need = int(lib().modpp_mm_workspace(d, k, n, pr.data, P, p))
    if need == 0:
        raise ModppError(-1, "modpp_mm_workspace")
    ws_ptr, ws_len = _workspace(need, A3.device, workspace)
    ukind = 0 if U.dtype == torch.int8 else 1
    ldu = U.stride(0) if U.numel() else k
    lda, sa = (A3.stride(1), A3.stride(0)) if A3.numel() else (n, k * n)
    ldc, sc = (out3.stride(1), out3.stride(0)) if out3.numel() else (n, d * n)
    rc = lib().modpp_mm(d, k, n, U.data_ptr(), ukind, ldu, A3.data_ptr(), lda, sa,
                        out3.data_ptr(), ldc, sc, pr.data, P, p, ws_ptr, ws_len,
                        _stream_handle(stream))
    _check(rc, "modpp_mm")
    return out3[0] if squeeze else out3


def modpp_mm_wide(U: torch.Tensor, A: torch.Tensor, primes: Sequence[int], *,
                  out: torch.Tensor | None = None, stream=None,
                  workspace: torch.Tensor | None = None) -> torch.Tensor:
    """C[j] = U[j] @ A[j] mod primes[j] with both operands residues (uint64, (P, d, k)
    and (P, k, n), canonical).  Returns (P, d, n) uint64."""
    _check_residues(U, "U")
    _check_residues(A, "A")
    if U.dim() != 3 or A.dim() != 3 or U.shape[0] != A.shape[0] or U.shape[2] != A.shape[1]:
        raise ValueError("U must be (P, d, k) and A (P, k, n)")
    P, d, k = U.shape
    n = A.shape[2]
    if (U.numel() and U.stride(2) != 1) or (A.numel() and A.stride(2) != 1):
        raise ValueError("unit stride along the last dimension required")
    if out is None:
        out = torch.empty((P, d, n), dtype=torch.uint64, device=A.device)
    pr = _primes_arr(primes)
    need = int(lib().modpp_mm_wide_workspace(d, k, n, pr.data, P))
    if need == 0:
        raise ModppError(-1, "modpp_mm_wide_workspace")
    ws_ptr, ws_len = _workspace(need, A.device, workspace)
    lu, su = (U.stride(1), U.stride(0)) if U.numel() else (k, d * k)
    la, sa = (A.stride(1), A.stride(0)) if A.numel() else (n, k * n)
    lc, sc = (out.stride(1), out.stride(0)) if out.numel() else (n, d * n)
    _check(lib().modpp_mm_wide(d, k, n, U.data_ptr(), lu, su, A.data_ptr(), la, sa,
                               out.data_ptr(), lc, sc, pr.data, P, ws_ptr, ws_len,
                               _stream_handle(stream)), "modpp_mm_wide")
    return out


def modpp_mm_trunc(U: torch.Tensor, B: torch.Tensor, q: int, *, path="f16", drop_bits: int = 0,
                   out: torch.Tensor | None = None, stream=None,
                   workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Strategy 2 of Sec. 6.1: C ~ U @ B mod q for one odd modulus q from the
    high-order bits of B.  path "f16": B rounded to multiples of 2^drop_bits,
    exact product of the rounded operand; path "fp64": B rounded to 53 bits,
    one DGEMM (drop_bits 0).  U: (d, k) int8/int32; B: (k, n) uint64 residues.
    Returns (d, n) uint64."""
    _check_residues(B, "B")
    if not U.is_cuda or U.dtype not in (torch.int8, torch.int32) or U.dim() != 2 or B.dim() != 2:
        raise TypeError("U must be 2-D int8/int32 and B 2-D uint64 CUDA tensors")
    if U.shape[1] != B.shape[0]:
        raise ValueError("inner dimensions differ")
    d, k = U.shape
    n = B.shape[1]
    if (U.numel() and U.stride(1) != 1) or (B.numel() and B.stride(1) != 1):
        raise ValueError("unit stride along the last dimension required")
    if out is None:
        out = torch.empty((d, n), dtype=torch.uint64, device=B.device)
    p = _path(path)
    need = int(lib().modpp_mm_trunc_workspace(d, k, n, int(q), p, int(drop_bits)))
    if need == 0:
        raise ModppError(-1, "modpp_mm_trunc_workspace")
    ws_ptr, ws_len = _workspace(need, B.device, workspace)
    ldu = U.stride(0) if U.numel() else k
    ldb = B.stride(0) if B.numel() else n
    ldc = out.stride(0) if out.numel() else n
    _check(lib().modpp_mm_trunc(d, k, n, U.data_ptr(), 0 if U.dtype == torch.int8 else 1, ldu,
                                B.data_ptr(), ldb, out.data_ptr(), ldc, int(q), p,
                                int(drop_bits), ws_ptr, ws_len, _stream_handle(stream)),
           "modpp_mm_trunc")
    return out


class PreparedU:
    """A plaintext U (d x k) converted once into the f16 layout the tensor
    cores read (modpp_u_to_f16), for reuse over many pc_mm / pc_mv calls."""

    def __init__(self, U: torch.Tensor, stream=None):
        if not U.is_cuda or U.dtype not in (torch.int8, torch.int32) or U.dim() != 2:
            raise TypeError("U must be a 2-D CUDA int8 or int32 tensor")
        if U.numel() and U.stride(1) != 1:
            raise ValueError("U needs unit stride along k")
        self.shape = tuple(U.shape)
        d, k = self.shape
        nbytes = int(lib().modpp_u16_bytes(d, k))
        self.data = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=U.device)
        _check(lib().modpp_u_to_f16(d, k, U.data_ptr(), 0 if U.dtype == torch.int8 else 1,
                                    U.stride(0) if U.numel() else k, self.data.data_ptr(),
                                    _stream_handle(stream)), "modpp_u_to_f16")

    @property
    def is_cuda(self):
        return True

    def data_ptr(self):
        return self.data.data_ptr()


def _pc(fn_name: str, U, A, B, primes, path, out, stream, workspace):
    _check_residues(A, "A")
    _check_residues(B, "B")
    prepared = isinstance(U, PreparedU)
    if prepared:
        if _path(path) != Path.F16:
            raise ValueError("a prepared U serves the f16 path only")
    elif not U.is_cuda or U.dtype != torch.int8 or U.dim() != 2 or not U.is_contiguous():
        raise TypeError("U must be a contiguous 2-D CUDA int8 tensor")
    if not (A.is_contiguous() and B.is_contiguous()) or A.shape != B.shape or A.dim() != 3:
        raise ValueError("A and B must be contiguous (P, kct, N) tensors of equal shape")
    P, kct, N = A.shape
    d = U.shape[0]
    if U.shape[1] != kct or len(primes) != P:
        raise ValueError("shape mismatch between U, A/B and primes")
    if out is None:
        out = (torch.empty((P, d, N), dtype=torch.uint64, device=A.device),
               torch.empty((P, d, N), dtype=torch.uint64, device=A.device))
    Aout, Bout = out
    if not (Aout.is_contiguous() and Bout.is_contiguous()) or Aout.shape != (P, d, N) \
            or Bout.shape != (P, d, N):
        raise ValueError("outputs must be contiguous (P, d, N) tensors")
    pr = _primes_arr(primes)
    p = _path(path)
    need = int(lib().pc_mm_workspace(d, kct, N, pr.data, P, p))
    if need == 0:
        raise ModppError(-1, "pc_mm_workspace")
    ws_ptr, ws_len = _workspace(need, A.device, workspace)
    if prepared:
        rc = lib().pc_mm_u16(d, kct, N, U.data_ptr(), A.data_ptr(), B.data_ptr(),
                             Aout.data_ptr(), Bout.data_ptr(), pr.data, P, ws_ptr, ws_len,
                             _stream_handle(stream))
        _check(rc, "pc_mm_u16")
        return Aout, Bout
    rc = getattr(lib(), fn_name)(d, kct, N, U.data_ptr(), A.data_ptr(), B.data_ptr(),
                                 Aout.data_ptr(), Bout.data_ptr(), pr.data, P, p, ws_ptr,
                                 ws_len, _stream_handle(stream))
    _check(rc, fn_name)
    return Aout, Bout


def pc_mm(U: torch.Tensor, A: torch.Tensor, B: torch.Tensor, primes: Sequence[int], *,
          path="f16", out=None, stream=None, workspace=None):
    """Row-format PC-MM: (U @ A[j] mod q_j, U @ B[j] mod q_j) for every prime."""
    return _pc("pc_mm", U, A, B, primes, path, out, stream, workspace)


def pc_mv(U: torch.Tensor, A: torch.Tensor, B: torch.Tensor, primes: Sequence[int], *,
          path="f16", out=None, stream=None, workspace=None):
    """PC-Mv on a thin batch: same products as pc_mm with a small column count."""
    return _pc("pc_mv", U, A, B, primes, path, out, stream, workspace)


# --------------------------------------------------------------------------
# Grouped Mod-PP-MM
# --------------------------------------------------------------------------

class _Problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int64), ("k", ctypes.c_int64), ("n", ctypes.c_int64),
                ("U", ctypes.c_void_p), ("ldu", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("strideA", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64), ("strideC", ctypes.c_int64),
                ("primes", ctypes.c_void_p), ("P", ctypes.c_int)]


class GroupedPlan:
    """A grouped Mod-PP-MM over problems (U_i, A_i, primes_i).

    U_i: (d, k) contiguous int8 CUDA tensor; A_i: (P, k, n) contiguous uint64 CUDA
    tensor; primes_i: P primes.  Outputs are allocated (``self.outputs[i]`` is
    (P, d, n) uint64) unless given.  ``tune`` lets the library time the digit
    widths on these problems and keep the fastest.
    """

    def __init__(self, problems, outputs=None, tune: bool = True, stream=None,
                 workspace: torch.Tensor | None = None):
        self._plan = ctypes.c_void_p()
        self._keep = []
        self.outputs = []
        arr = (_Problem * len(problems))()
        dev = None
        for i, (U, A, primes) in enumerate(problems):
            A3 = A.unsqueeze(0) if A.dim() == 2 else A
            _check_residues(A3, "A")
            if not U.is_cuda or U.dtype != torch.int8 or U.dim() != 2:
                raise TypeError("U must be a 2-D CUDA int8 tensor")
            if U.numel() and U.stride(1) != 1:
                raise ValueError("U needs unit stride along k")
            if A3.numel() and A3.stride(2) != 1:
                raise ValueError("A needs unit stride along n")
            P, k, n = A3.shape
            d = U.shape[0]
            if U.shape[1] != k or len(primes) != P:
                raise ValueError(f"problem {i}: shape mismatch")
            C = outputs[i] if outputs is not None else torch.empty(
                (P, d, n), dtype=torch.uint64, device=A3.device)
            if C.shape != (P, d, n) or C.stride(2) != 1:
                raise ValueError(f"problem {i}: output must be (P, d, n) with unit stride along n")
            pr = _primes_arr(primes)
            self._keep += [U, A3, C, pr]
            self.outputs.append(C)
            # Leading dimensions of empty operands are not meaningful: use the
            # dense ones so the library's checks hold.
            ldu = U.stride(0) if U.numel() else k
            lda, sa = (A3.stride(1), A3.stride(0)) if A3.numel() else (n, k * n)
            arr[i] = _Problem(d, k, n, U.data_ptr(), ldu, A3.data_ptr(), lda, sa,
                              C.data_ptr(), C.stride(1), C.stride(0), pr.data, P)
            dev = A3.device
        self._arr = arr
        need = int(lib().modpp_group_workspace(ctypes.byref(arr), len(problems)))
        if need == 0:
            raise ModppError(-1, "modpp_group_workspace")
        if workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=dev)
        if workspace.data_ptr() % 256 or workspace.numel() * workspace.element_size() < need:
            raise ValueError("workspace misaligned or too small")
        self.workspace = workspace
        _check(lib().modpp_group_plan_create(ctypes.byref(arr), len(problems),
                                             workspace.data_ptr(), need, 1 if tune else 0,
                                             _stream_handle(stream), ctypes.byref(self._plan)),
               "modpp_group_plan_create")

    def run(self, stream=None, graph: bool = False) -> list:
        fn = lib().modpp_group_run_graph if graph else lib().modpp_group_run
        _check(fn(self._plan, _stream_handle(stream)), "modpp_group_run")
        return self.outputs

    def info(self) -> dict:
        b, tiles, tuned = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * 3)()
        _check(lib().modpp_group_plan_info(self._plan, ctypes.byref(b), ctypes.byref(tiles),
                                           ctypes.byref(tuned), ms), "modpp_group_plan_info")
        return {"digit_bits": b.value, "tiles": tiles.value,
                "tuned": {0: "no", 1: "timed", 2: "cached"}[tuned.value],
                "tuned_ms": {8 + i: ms[i] for i in range(3)}}

    def status(self, stream=None) -> int:
        return int(lib().modpp_status_read(ctypes.c_void_p(self.workspace.data_ptr()),
                                           ctypes.c_void_p(_stream_handle(stream))))

    def close(self) -> None:
        if self._plan:
            lib().modpp_group_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def modpp_mm_grouped(problems, *, tune: bool = True, graph: bool = False, stream=None):
    """One-shot grouped Mod-PP-MM; returns the list of (P, d, n) outputs."""
    plan = GroupedPlan(problems, tune=tune, stream=stream)
    out = plan.run(stream=stream, graph=graph)
    torch.cuda.current_stream().synchronize()
    plan.close()
    return out
