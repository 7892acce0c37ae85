"""ctypes binding of the ring / CC-MM part of ``libmodpp.so`` (C ABI in
``include/modpp_ring.h``): KeySwitch, Tweak (Alg. 3), Transpose (Alg. 4),
Rescale and CC-MM (Alg. 8).

Argument marshalling only.  Ciphertext batches are uint64 CUDA tensors of
shape (2, L, n, N) -- part (a, b), prime, ciphertext, coefficient -- and
switching keys are (count, dnum, 2, L+K, N) for the ring's gadget of dnum
digits and K special primes (``Ring.key_shape``).  The ring tables and every
workspace are PyTorch allocations handed to the library as device pointers.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from .api import ModppError, _check, _stream_handle, _workspace, lib

__all__ = ["Ring"]

_registered = False


def _register():
    global _registered
    if _registered:
        return lib()
    L = lib()
    P, I64, I, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    L.modpp_ring_bytes.argtypes = [I64, I]
    L.modpp_ring_bytes.restype = SZ
    L.modpp_ring_bytes_ks.argtypes = [I64, I, I, I]
    L.modpp_ring_bytes_ks.restype = SZ
    L.modpp_ring_create.argtypes = [I64, I, P, P, SZ, P, P]
    L.modpp_ring_create_ks.argtypes = [I64, I, I, I, P, P, SZ, P, P]
    L.modpp_ring_destroy.argtypes = [P]
    L.modpp_ring_prepare_keys.argtypes = [P, P, I64, P]
    L.modpp_keyswitch_workspace.argtypes = [P, I64]
    L.modpp_keyswitch_workspace.restype = SZ
    L.modpp_keyswitch.argtypes = [P, P, P, I64, P, P, SZ, P]
    L.modpp_keyswitch_indexed.argtypes = [P, P, P, I64, P, P, P, SZ, P]
    L.modpp_tweak_workspace.argtypes = [P, I64]
    L.modpp_tweak_workspace.restype = SZ
    L.modpp_tweak.argtypes = [P, P, P, I64, P, SZ, P]
    L.modpp_transpose_workspace.argtypes = [P, I64]
    L.modpp_transpose_workspace.restype = SZ
    L.modpp_transpose.argtypes = [P, P, P, I64, P, P, SZ, P]
    L.modpp_rescale.argtypes = [P, P, P, I64, P]
    L.cc_mm_workspace.argtypes = [P]
    L.cc_mm_workspace.restype = SZ
    L.cc_mm.argtypes = [P, P, P, P, P, P, P, SZ, P]
    L.cc_mm_stage_ms.argtypes = [P, P]
    L.modpp_ring_status_read.argtypes = [P, P]
    L.cc_mm_ex_workspace.argtypes = [P, I64, I]
    L.cc_mm_ex_workspace.restype = SZ
    L.cc_mm_ex.argtypes = [P, I64, P, P, P, P, I, P, P, P, SZ, P]
    L.pc_mm_precomp_workspace.argtypes = [P, I64, I64, I]
    L.pc_mm_precomp_workspace.restype = SZ
    L.pc_mm_precomp.argtypes = [P, I64, I64, P, P, P, P, I, P, P, SZ, P]
    _registered = True
    return L


class Ring:
    """R_q = Z_q[X]/(X^N+1) over the chain primes[:L] with the K special
    primes primes[L:] for key switching, whose gadget has dnum digits (default
    K = 1, dnum = L).  Holds the library's ring tables on `device`."""

    def __init__(self, N: int, primes_with_P: Sequence[int], device="cuda", stream=None,
                 special: int = 1, dnum: int | None = None):
        L = _register()
        self.N = int(N)
        self.primes = [int(q) for q in primes_with_P]
        self.K = int(special)
        self.L = len(self.primes) - self.K
        self.dnum = self.L if dnum is None else int(dnum)
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        nbytes = int(L.modpp_ring_bytes_ks(self.N, self.L, self.K, self.dnum))
        if nbytes == 0:
            raise ModppError(-1, "modpp_ring_bytes_ks")
        self._mem = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._pr = np.ascontiguousarray(self.primes, dtype=np.uint64)
        h = ctypes.c_void_p()
        _check(L.modpp_ring_create_ks(self.N, self.L, self.K, self.dnum, self._pr.ctypes.data,
                                      self._mem.data_ptr(), nbytes, _stream_handle(stream),
                                      ctypes.byref(h)),
               "modpp_ring_create_ks")
        self._h = h

    def key_shape(self) -> tuple:
        """Shape of one switching key: (dnum, 2, L + K, N)."""
        return (self.dnum, 2, self.L + self.K, self.N)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().modpp_ring_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ checks
    def _batch(self, t: torch.Tensor, name: str, planes: int | None = None) -> int:
        planes = self.L if planes is None else planes
        if not (t.is_cuda and t.dtype == torch.uint64 and t.is_contiguous() and t.dim() == 4):
            raise TypeError(f"{name} must be a contiguous 4-D uint64 CUDA tensor")
        if t.shape[0] != 2 or t.shape[1] != planes or t.shape[3] != self.N:
            raise ValueError(f"{name} must have shape (2, {planes}, n, {self.N})")
        return int(t.shape[2])

    def _keys(self, k: torch.Tensor, name: str) -> int:
        if not (k.is_cuda and k.dtype == torch.uint64 and k.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous uint64 CUDA tensor")
        if k.dim() == 4:
            k = k.unsqueeze(0)
        if tuple(k.shape[1:]) != self.key_shape():
            raise ValueError(f"{name} must have shape (count,) + {self.key_shape()}")
        return int(k.shape[0])

    # ------------------------------------------------------------ calls
    def prepare_keys(self, keys: torch.Tensor, stream=None) -> torch.Tensor:
        """In place: coefficients -> evaluation-domain Montgomery form."""
        count = self._keys(keys, "keys")
        _check(lib().modpp_ring_prepare_keys(self._h, keys.data_ptr(), count,
                                             _stream_handle(stream)), "modpp_ring_prepare_keys")
        return keys

    def keyswitch(self, ct: torch.Tensor, key: torch.Tensor, out=None, stream=None,
                  workspace=None) -> torch.Tensor:
        n = self._batch(ct, "ct")
        self._keys(key, "key")
        out = torch.empty_like(ct) if out is None else out
        need = int(lib().modpp_keyswitch_workspace(self._h, n))
        wp, wl = _workspace(need, ct.device, workspace)
        _check(lib().modpp_keyswitch(self._h, ct.data_ptr(), out.data_ptr(), n, key.data_ptr(),
                                     wp, wl, _stream_handle(stream)), "modpp_keyswitch")
        return out

    def keyswitch_indexed(self, ct: torch.Tensor, keys: torch.Tensor, key_index: torch.Tensor,
                          out=None, stream=None, workspace=None) -> torch.Tensor:
        """Ciphertext c switched with keys[key_index[c]]; key_index[c] < 0 copies it."""
        n = self._batch(ct, "ct")
        count = self._keys(keys, "keys")
        if not (key_index.is_cuda and key_index.dtype == torch.int32 and key_index.is_contiguous()
                and key_index.numel() == n):
            raise TypeError("key_index must be a contiguous int32 CUDA tensor of n entries")
        if n and int(key_index.max()) >= count:
            raise ValueError("key_index refers past the last key")
        out = torch.empty_like(ct) if out is None else out
        need = int(lib().modpp_keyswitch_workspace(self._h, n))
        wp, wl = _workspace(need, ct.device, workspace)
        _check(lib().modpp_keyswitch_indexed(self._h, ct.data_ptr(), out.data_ptr(), n,
                                             keys.data_ptr(), key_index.data_ptr(), wp, wl,
                                             _stream_handle(stream)), "modpp_keyswitch_indexed")
        return out

    def tweak(self, ct: torch.Tensor, out=None, stream=None, workspace=None) -> torch.Tensor:
        n = self._batch(ct, "ct")
        out = torch.empty_like(ct) if out is None else out
        need = int(lib().modpp_tweak_workspace(self._h, n))
        wp, wl = _workspace(need, ct.device, workspace)
        _check(lib().modpp_tweak(self._h, ct.data_ptr(), out.data_ptr(), n, wp, wl,
                                 _stream_handle(stream)), "modpp_tweak")
        return out

    def transpose(self, ct: torch.Tensor, aut_keys: torch.Tensor, out=None, stream=None,
                  workspace=None) -> torch.Tensor:
        n = self._batch(ct, "ct")
        if n % self.N:
            raise ValueError("transpose needs a whole number of N-ciphertext matrices")
        if self._keys(aut_keys, "aut_keys") != self.N:
            raise ValueError("aut_keys must hold N keys (key j: s(X^(2j+1)) -> s)")
        groups = n // self.N
        out = torch.empty_like(ct) if out is None else out
        need = int(lib().modpp_transpose_workspace(self._h, groups))
        wp, wl = _workspace(need, ct.device, workspace)
        _check(lib().modpp_transpose(self._h, ct.data_ptr(), out.data_ptr(), groups,
                                     aut_keys.data_ptr(), wp, wl, _stream_handle(stream)),
               "modpp_transpose")
        return out

    def rescale(self, ct: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        n = self._batch(ct, "ct")
        if out is None:
            out = torch.empty((2, self.L - 1, n, self.N), dtype=torch.uint64, device=ct.device)
        _check(lib().modpp_rescale(self._h, ct.data_ptr(), out.data_ptr(), n,
                                   _stream_handle(stream)), "modpp_rescale")
        return out

    def cc_mm_workspace_bytes(self) -> int:
        return int(lib().cc_mm_workspace(self._h))

    def cc_mm(self, ct1: torch.Tensor, ct2: torch.Tensor, aut_keys: torch.Tensor,
              relin_key: torch.Tensor, out=None, stream=None, workspace=None) -> torch.Tensor:
        """Alg. 8 on column-wise encryptions (2, L, N, N); returns (2, L-1, N, N)."""
        for t, nm in ((ct1, "ct1"), (ct2, "ct2")):
            if self._batch(t, nm) != self.N:
                raise ValueError(f"{nm} must hold N ciphertexts")
        if self._keys(aut_keys, "aut_keys") != self.N:
            raise ValueError("aut_keys must hold N keys")
        self._keys(relin_key, "relin_key")
        if out is None:
            out = torch.empty((2, self.L - 1, self.N, self.N), dtype=torch.uint64,
                              device=ct1.device)
        need = self.cc_mm_workspace_bytes()
        if need == 0:
            raise ModppError(-1, "cc_mm_workspace")
        wp, wl = _workspace(need, ct1.device, workspace)
        _check(lib().cc_mm(self._h, ct1.data_ptr(), ct2.data_ptr(), aut_keys.data_ptr(),
                           relin_key.data_ptr(), out.data_ptr(), wp, wl, _stream_handle(stream)),
               "cc_mm")
        return out

    def cc_mm_ex(self, ct1: torch.Tensor, ct2: torch.Tensor, aut_keys: torch.Tensor,
                 relin_key: torch.Tensor, m2_rowwise: bool = False, out=None, stream=None,
                 workspace=None):
        """Alg. 8 with the right operand column-wise (as cc_mm) or, with
        m2_rowwise, row-wise and Step 1 skipped: ct1 (2, L, n, N) encrypts the
        columns of an N x n matrix, ct2 (2, L, n, N) the rows of an n x N
        matrix, 1 <= n <= N.  Returns (out (2, L-1, N, N), scale multiplier
        1/q_{L-1} of the output)."""
        n = self._batch(ct1, "ct1")
        if self._batch(ct2, "ct2") != n:
            raise ValueError("ct1 and ct2 must hold the same number of ciphertexts")
        if not m2_rowwise and n != self.N:
            raise ValueError("a column-wise ct2 needs N ciphertexts")
        if self._keys(aut_keys, "aut_keys") != self.N:
            raise ValueError("aut_keys must hold N keys")
        self._keys(relin_key, "relin_key")
        flags = 1 if m2_rowwise else 0
        if out is None:
            out = torch.empty((2, self.L - 1, self.N, self.N), dtype=torch.uint64,
                              device=ct1.device)
        need = int(lib().cc_mm_ex_workspace(self._h, n, flags))
        if need == 0:
            raise ModppError(-1, "cc_mm_ex_workspace")
        wp, wl = _workspace(need, ct1.device, workspace)
        mult = ctypes.c_double()
        _check(lib().cc_mm_ex(self._h, n, ct1.data_ptr(), ct2.data_ptr(), aut_keys.data_ptr(),
                              relin_key.data_ptr(), flags, out.data_ptr(), ctypes.byref(mult),
                              wp, wl, _stream_handle(stream)), "cc_mm_ex")
        return out, mult.value

    def pc_mm_precomp(self, Ut: torch.Tensor, a: torch.Tensor, B: torch.Tensor,
                      keys: torch.Tensor, rescale: bool = False, out=None, stream=None,
                      workspace=None) -> torch.Tensor:
        """Alg. 7 on a shared-a encryption, then the key switches back to one
        secret: Ut (d3, d2) int8 = U^T; a (L, N) the shared a-part; B (L, d2, N)
        the b-parts; keys (d3,) + key_shape() prepared, key k from column k of
        S*U.  Returns the batch (2, L or L-1, d3, N)."""
        if not (Ut.is_cuda and Ut.dtype == torch.int8 and Ut.dim() == 2 and Ut.is_contiguous()):
            raise TypeError("Ut must be a contiguous 2-D int8 CUDA tensor")
        d3, d2 = Ut.shape
        for t, nm, shp in ((a, "a", (self.L, self.N)), (B, "B", (self.L, d2, self.N))):
            if not (t.is_cuda and t.dtype == torch.uint64 and t.is_contiguous()):
                raise TypeError(f"{nm} must be a contiguous uint64 CUDA tensor")
            if tuple(t.shape) != shp:
                raise ValueError(f"{nm} must have shape {shp}")
        if self._keys(keys, "keys") != d3:
            raise ValueError("keys must hold d3 keys")
        flags = 1 if rescale else 0
        Lo = self.L - 1 if rescale else self.L
        if out is None:
            out = torch.empty((2, Lo, d3, self.N), dtype=torch.uint64, device=B.device)
        need = int(lib().pc_mm_precomp_workspace(self._h, d2, d3, flags))
        if need == 0:
            raise ModppError(-1, "pc_mm_precomp_workspace")
        wp, wl = _workspace(need, B.device, workspace)
        _check(lib().pc_mm_precomp(self._h, d2, d3, Ut.data_ptr(), a.data_ptr(), B.data_ptr(),
                                   keys.data_ptr(), flags, out.data_ptr(), wp, wl,
                                   _stream_handle(stream)), "pc_mm_precomp")
        return out

    def status(self, stream=None) -> int:
        """Reads and clears the ring's status word (syncs the stream):
        0, or MODPP_ERR_RANGE (-6) when debug checks found an input
        coefficient not below its prime since the last read."""
        return int(lib().modpp_ring_status_read(self._h, _stream_handle(stream)))

    def cc_mm_stage_ms(self) -> list[float]:
        """Stage times of the last cc_mm while profiling is on: transpose of ct2,
        the two Mod-PP-MMs, transpose of C00 | C10, relin + finish."""
        arr = (ctypes.c_double * 4)()
        _check(lib().cc_mm_stage_ms(self._h, arr), "cc_mm_stage_ms")
        return list(arr)
