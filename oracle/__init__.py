"""Test oracle for the Mod-PP-MM hot path (arXiv 2503.16080).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product library
(``paper_2503_16080_gb300``) never imports, loads or links anything here, and
this package imports nothing from it: the two share no code.

It is a plain, slow, obviously correct CPU restatement of what the hot path
computes:

* ``mod_pp_mm``      C = U*A mod q_j for every prime (Sec. 5, ModPPMM notation;
                     Thm th:pcmm). Plain definition, 128-bit accumulation in C.
* ``strategy1_*``    Strategy 1 of Sec. 6.1 (Lemma le:strategy1, Eq. decomp):
                     base-K signed digits, k1*k2 binary64 products, integer
                     recombination.  The FP64-limb path computes this.
* ``negacyclic_mul`` products in R_q = Z_q[X]/(X^N+1) (Sec. 2).
* ``ckks_encode`` / ``rlwe_encrypt_rows`` / ``rlwe_decrypt_rows`` / ``crt2``:
                     textbook coefficient-encoded CKKS (Sec. 2.2).
* ``toeplitz``       Toep(m) of Sec. 2 (the matrix of u -> u*m).

Pins against things other than itself live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "modpp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_modpp.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (OpenMP). Returns the .so path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I = ctypes.c_int64
    U64 = ctypes.c_uint64
    lib.or_mod_pp_mm_i32.argtypes = [I, I, I, P, I, P, I, P, I, U64]
    lib.or_mod_pp_mm_res.argtypes = [I, I, I, P, I, P, I, P, I, U64]
    lib.or_negacyclic_mul.argtypes = [I, P, P, P, U64]
    lib.or_negacyclic_mul_schoolbook.argtypes = [I, P, P, P, U64]
    lib.or_find_psi.argtypes = [U64, I]
    lib.or_find_psi.restype = U64
    lib.or_mulmod.argtypes = [U64, U64, U64]
    lib.or_mulmod.restype = U64
    lib.or_powmod.argtypes = [U64, U64, U64]
    lib.or_powmod.restype = U64
    lib.or_ckks_encode.argtypes = [I, P, ctypes.c_double, P]
    lib.or_ckks_encode.restype = None
    lib.or_ckks_decode.argtypes = [I, P, ctypes.c_double, P]
    lib.or_ckks_decode.restype = None
    lib.or_rlwe_encrypt_rows.argtypes = [I, I, ctypes.c_int, P, P, P, P, P, P]
    lib.or_rlwe_decrypt_rows.argtypes = [I, I, ctypes.c_int, P, P, P, P, P]
    lib.or_crt2_centered.argtypes = [I, P, P, U64, U64, P, P]
    lib.or_crt2_centered.restype = None
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed (rc={rc})")


# --------------------------------------------------------------------------
# Mod-PP-MM (the definition)
# --------------------------------------------------------------------------

def mod_pp_mm(U: np.ndarray, A: np.ndarray, primes: Sequence[int]) -> np.ndarray:
    """C[j] = U @ A[j] mod primes[j], canonical in [0, q_j).

    U: (d, k) small signed integers (|U| < 2^31), any integer dtype.
    A: (P, k, n) uint64 residues (or (k, n) for a single prime).
    Returns (P, d, n) uint64 (or (d, n) for 2-D A).
    """
    lib = _load()
    U32 = np.ascontiguousarray(U, dtype=np.int32)
    if not np.array_equal(U32.astype(np.int64), np.asarray(U, dtype=np.int64)):
        raise ValueError("U entries must fit in int32")
    squeeze = A.ndim == 2
    A3 = np.ascontiguousarray(A[None] if squeeze else A, dtype=np.uint64)
    P, k, n = A3.shape
    d = U32.shape[0]
    assert U32.shape[1] == k and len(primes) == P
    C = np.empty((P, d, n), dtype=np.uint64)
    for j, q in enumerate(primes):
        _check(lib.or_mod_pp_mm_i32(d, k, n, _ptr(U32), k, _ptr(A3[j]), n, _ptr(C[j]), n, int(q)),
               "mod_pp_mm")
    return C[0] if squeeze else C


def mod_pp_mm_rows(U: np.ndarray, A: np.ndarray, primes: Sequence[int],
                   rows: np.ndarray) -> np.ndarray:
    """The rows ``rows`` of mod_pp_mm(U, A, primes): shape (P, len(rows), n)."""
    return mod_pp_mm(np.ascontiguousarray(np.asarray(U)[rows]), A, primes)


def mod_pp_mm_residues(U: np.ndarray, A: np.ndarray, q: int) -> np.ndarray:
    """C = U @ A mod q with both operands residues mod q (Alg. 8, step 2)."""
    lib = _load()
    U64 = np.ascontiguousarray(U, dtype=np.uint64)
    A64 = np.ascontiguousarray(A, dtype=np.uint64)
    d, k = U64.shape
    n = A64.shape[1]
    C = np.empty((d, n), dtype=np.uint64)
    _check(lib.or_mod_pp_mm_res(d, k, n, _ptr(U64), k, _ptr(A64), n, _ptr(C), n, int(q)),
           "mod_pp_mm_res")
    return C


# --------------------------------------------------------------------------
# Strategy 1 of Sec. 6.1 (Lemma le:strategy1): the FP64-limb reduction
# --------------------------------------------------------------------------

def strategy1_base(d2: int) -> int:
    """K = floor(sqrt(2^53 / d2)) (Lemma le:strategy1)."""
    return math.isqrt((1 << 53) // d2)


def strategy1_digit_count(theta: int, K: int) -> int:
    """Number of base-K signed digits for integers of absolute value <= theta.

    The lemma states k = ceil(log(theta)/log(K)); its proof decomposes integers
    with |r| < K^k.  Both agree except when theta is an exact power of K, where
    the proof's condition needs one digit more; we take the smallest k with
    K^k > theta (at least 1)."""
    k = 1
    while K ** k <= theta:
        k += 1
    return k


def strategy1_signed_digits(X: np.ndarray, K: int, count: int) -> list[np.ndarray]:
    """Eq. decomp: X = sum_i X_i K^i with each X_i of the sign of X and |X_i| < K."""
    Xo = np.asarray(X, dtype=object)
    sign = np.where(Xo < 0, -1, 1)
    mag = np.abs(Xo)
    digits = []
    for _ in range(count):
        digits.append((sign * (mag % K)).astype(np.int64))
        mag = mag // K
    if np.any(mag != 0):
        raise ValueError("digit count too small for the operand")
    return digits


def centered(A: np.ndarray, q: int) -> np.ndarray:
    """Representative of each residue in (-q/2, q/2]."""
    Ao = np.asarray(A, dtype=object)
    return np.where(2 * Ao > q, Ao - q, Ao)


def strategy1_mod_pp_mm(U: np.ndarray, A: np.ndarray, q: int) -> tuple[np.ndarray, dict]:
    """Mod-PP-MM through Strategy 1, in the paper's order (Lemma le:strategy1):

    1. K = floor(sqrt(2^53/d2)); k1, k2 digit counts for theta1 = ||A||, theta2 = ||U||;
    2. signed base-K digits of both operands (Eq. decomp);
    3. the k1*k2 products U_j @ A_i in binary64 (numpy matmul), each exact
       because every partial sum stays below d2*K^2 <= 2^53;
    4. sum_{i,j} K^(i+j) * (U_j @ A_i) on integers, then reduce mod q.
    Returns (C, info) with info = {K, k1, k2, products}.
    """
    d, d2 = U.shape
    Ac = centered(A, q)
    theta1 = int(np.max(np.abs(Ac))) if Ac.size else 0
    theta2 = int(np.max(np.abs(np.asarray(U, dtype=object)))) if U.size else 0
    K = strategy1_base(d2)
    k1 = strategy1_digit_count(theta1, K)
    k2 = strategy1_digit_count(theta2, K)
    Ad = strategy1_signed_digits(Ac, K, k1)
    Ud = strategy1_signed_digits(np.asarray(U, dtype=object), K, k2)
    total = np.zeros((d, A.shape[1]), dtype=object)
    for i, Ai in enumerate(Ad):
        for j, Uj in enumerate(Ud):
            prod = Uj.astype(np.float64) @ Ai.astype(np.float64)
            assert np.all(np.abs(prod) < 2.0 ** 53)
            total = total + prod.astype(np.int64).astype(object) * (K ** (i + j))
    C = np.asarray(total % q, dtype=np.uint64)
    return C, {"K": K, "k1": k1, "k2": k2, "products": k1 * k2}


# --------------------------------------------------------------------------
# Ring R_q = Z_q[X]/(X^N+1) and textbook CKKS (Sec. 2)
# --------------------------------------------------------------------------

def toeplitz(m: Sequence[int]) -> np.ndarray:
    """Toep(m) of Sec. 2: column i holds the coefficients of X^i * m in Z[X]/(X^N+1).

    Entry (r, c) is m[r-c] when r >= c and -m[N+r-c] otherwise.  Python ints."""
    N = len(m)
    T = np.empty((N, N), dtype=object)
    for r in range(N):
        for c in range(N):
            T[r, c] = int(m[r - c]) if r >= c else -int(m[N + r - c])
    return T


def negacyclic_mul(a: np.ndarray, b: np.ndarray, q: int, schoolbook: bool = False) -> np.ndarray:
    lib = _load()
    a64 = np.ascontiguousarray(np.asarray(a, dtype=np.uint64) % np.uint64(q))
    b64 = np.ascontiguousarray(np.asarray(b, dtype=np.uint64) % np.uint64(q))
    c = np.empty_like(a64)
    fn = lib.or_negacyclic_mul_schoolbook if schoolbook else lib.or_negacyclic_mul
    _check(fn(a64.size, _ptr(a64), _ptr(b64), _ptr(c), int(q)), "negacyclic_mul")
    return c


def find_psi(q: int, N: int) -> int:
    return int(_load().or_find_psi(int(q), int(N)))


def ckks_encode(z: np.ndarray, delta: float) -> np.ndarray:
    """Ecd_coeff (Sec. 2.2): floor(Delta*z + 1/2), elementwise."""
    z64 = np.ascontiguousarray(z, dtype=np.float64)
    m = np.empty(z64.shape, dtype=np.int64)
    _load().or_ckks_encode(z64.size, _ptr(z64), float(delta), _ptr(m))
    return m


def ckks_decode(p: np.ndarray, delta: float) -> np.ndarray:
    p64 = np.ascontiguousarray(p, dtype=np.int64)
    z = np.empty(p64.shape, dtype=np.float64)
    _load().or_ckks_decode(p64.size, _ptr(p64), float(delta), _ptr(z))
    return z


def rlwe_encrypt_rows(a: np.ndarray, s: np.ndarray, m: np.ndarray, e: np.ndarray,
                      primes: Sequence[int]) -> np.ndarray:
    """b = -(a*s) + m + e mod q_j row by row (symmetric RLWE, Sec. 2.1).

    a: (P, rows, N) uniform residues; s: (N,) small signed; m, e: (rows, N).
    Returns b: (P, rows, N)."""
    P, rows, N = a.shape
    a64 = np.ascontiguousarray(a, dtype=np.uint64)
    s64 = np.ascontiguousarray(s, dtype=np.int64)
    m64 = np.ascontiguousarray(m, dtype=np.int64)
    e64 = np.ascontiguousarray(e, dtype=np.int64)
    pr = np.ascontiguousarray(primes, dtype=np.uint64)
    b = np.empty_like(a64)
    _check(_load().or_rlwe_encrypt_rows(rows, N, P, _ptr(pr), _ptr(a64), _ptr(s64), _ptr(m64),
                                        _ptr(e64), _ptr(b)), "rlwe_encrypt_rows")
    return b


def rlwe_decrypt_rows(a: np.ndarray, b: np.ndarray, s: np.ndarray,
                      primes: Sequence[int]) -> np.ndarray:
    """a*s + b mod q_j row by row. a, b: (P, rows, N). Returns (P, rows, N)."""
    P, rows, N = a.shape
    a64 = np.ascontiguousarray(a, dtype=np.uint64)
    b64 = np.ascontiguousarray(b, dtype=np.uint64)
    s64 = np.ascontiguousarray(s, dtype=np.int64)
    pr = np.ascontiguousarray(primes, dtype=np.uint64)
    out = np.empty_like(a64)
    _check(_load().or_rlwe_decrypt_rows(rows, N, P, _ptr(pr), _ptr(a64), _ptr(b64), _ptr(s64),
                                        _ptr(out)), "rlwe_decrypt_rows")
    return out


def crt2(r0: np.ndarray, r1: np.ndarray, q0: int, q1: int) -> np.ndarray:
    """Centred integers from residues mod q0 and q1 (raises if one exceeds int64)."""
    a = np.ascontiguousarray(r0, dtype=np.uint64)
    b = np.ascontiguousarray(r1, dtype=np.uint64)
    out = np.empty(a.shape, dtype=np.int64)
    ovf = np.empty(a.shape, dtype=np.int32)
    _load().or_crt2_centered(a.size, _ptr(a), _ptr(b), int(q0), int(q1), _ptr(out), _ptr(ovf))
    if ovf.any():
        raise OverflowError("CRT value outside int64")
    return out
