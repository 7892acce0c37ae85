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
* ``strategy2_*``    Strategy 2 of Sec. 6.1 (truncation): the product with the
                     high-order bits of the residue operand (an approximate
                     Mod-PP-MM for one modulus), in binary64 as printed and
                     as a rounding to a multiple of 2^s.
* ``negacyclic_mul`` products in R_q = Z_q[X]/(X^N+1) (Sec. 2).
* ``ckks_encode`` / ``rlwe_encrypt_rows`` / ``rlwe_decrypt_rows`` / ``crt2``:
                     textbook coefficient-encoded CKKS (Sec. 2.2).
* ``toeplitz``       Toep(m) of Sec. 2 (the matrix of u -> u*m).
* ``tweak_*``, ``automorphism``, ``ks_keygen``, ``keyswitch``, ``rescale``,
  ``transpose``, ``cc_mm``, ``cc_mm_rowwise``: the ring operations of the
  ciphertext-ciphertext product, Alg. 3 (Tweak), Alg. 4 (Transpose) and
  Alg. 8 (CC-MM), in the paper's order (``ccmm_oracle.c`` plus the
  compositions below).
* ``pcmm_precomp``   Alg. 7 (CP-MM with precomputation) on a shared-a
                     encryption, then the key switches back to one secret.

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
_SRCS = [os.path.join(_HERE, "modpp_oracle.c"), os.path.join(_HERE, "ccmm_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_modpp.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (OpenMP). Returns the .so path."""
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", *_SRCS, "-o", tmp, "-lm"]
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
    lib.or_monomial_mul.argtypes = [I, I, P, P, U64]
    lib.or_monomial_mul.restype = None
    lib.or_automorphism.argtypes = [I, I, P, P, U64]
    lib.or_automorphism.restype = None
    lib.or_tweak_def.argtypes = [I, I, ctypes.c_int, P, P, P]
    lib.or_tweak_def.restype = None
    lib.or_tweak_alg.argtypes = [I, I, ctypes.c_int, P, P, P]
    lib.or_tweak_alg.restype = None
    C = ctypes.c_int
    lib.or_ks_keygen_g.argtypes = [I, C, C, C, P, P, P, P, P, P]
    lib.or_keyswitch_g.argtypes = [I, C, C, C, P, P, P, P]
    lib.or_rescale.argtypes = [I, ctypes.c_int, P, P, P]
    lib.or_rescale.restype = None
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
# Strategy 2 of Sec. 6.1 (truncation): an approximate product from the
# high-order bits of the residue operand, for one modulus q
# --------------------------------------------------------------------------

def strategy2_round_high(B: np.ndarray, q: int, s: int) -> np.ndarray:
    """The residues' high-order bits: each entry of B (mod q) taken as its
    centred representative x in (-q/2, q/2] and rounded to the nearest
    multiple of 2^s, ties upward: 2^s * floor((x + 2^(s-1)) / 2^s).  s = 0
    keeps x.  Python integers (object array)."""
    x = centered(B, q)
    if s == 0:
        return x
    return ((x + (1 << (s - 1))) // (1 << s)) * (1 << s)


def strategy2_trunc(U: np.ndarray, B: np.ndarray, q: int, s: int) -> np.ndarray:
    """Mod-PP-MM of U with B's high-order bits (the truncation of Sec. 6.1
    with the decomposition of Eq. decomp started from the top, keeping the
    bits above 2^s): C = U * strategy2_round_high(B, q, s) mod q, canonical.
    Every entry differs from the exact (U * B mod q) by at most
    k * max|U| * 2^(s-1) (centred)."""
    Bs = strategy2_round_high(B, q, s)
    return mod_pp_mm(np.asarray(U), np.asarray(Bs % q, dtype=np.uint64)[None], [q])[0]


def strategy2_fp64(U: np.ndarray, B: np.ndarray, q: int) -> np.ndarray:
    """Strategy 2 as the paper states it for binary64: B's centred entries
    rounded to 53 bits (the nearest double), one floating-point product with
    U, and the product's value reduced modulo q.  The double products are
    integers; their residues are taken exactly, so the only errors are the
    rounding of B and of the floating-point sums (the paper's bound:
    about 2^-50 * k * ||U|| * ||B||)."""
    Bf = np.array([[float(v) for v in row] for row in centered(B, q)], dtype=np.float64) \
        if B.size else np.zeros(B.shape)
    P = np.asarray(U, dtype=np.float64) @ Bf
    out = np.empty(P.shape, dtype=np.uint64)
    for idx, v in np.ndenumerate(P):
        out[idx] = int(v) % q
    return out


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


# --------------------------------------------------------------------------
# Ring operations of the ciphertext-ciphertext product (Alg. 3, 4, 8)
# Ciphertexts: uint64 arrays [..., 2, L, N] (part 0 = a, part 1 = b).
# Switching keys: [L, 2, L+1, N] modulo the chain plus the special prime P.
# --------------------------------------------------------------------------

def _u64(x):
    return np.ascontiguousarray(x, dtype=np.uint64)


def monomial_mul(m, t: int, q: int) -> np.ndarray:
    """X^t * m in Z_q[X]/(X^N+1)."""
    m64 = _u64(m)
    out = np.empty_like(m64)
    _load().or_monomial_mul(m64.size, int(t), _ptr(m64), _ptr(out), int(q))
    return out


def automorphism(m, ell: int, q: int) -> np.ndarray:
    """m(X) -> m(X^ell) for odd ell (Aut, Sec. 2.2)."""
    m64 = _u64(m)
    out = np.empty_like(m64)
    _load().or_automorphism(m64.size, int(ell), _ptr(m64), _ptr(out), int(q))
    return out


def ct_map(ct, primes, fn) -> np.ndarray:
    """Apply fn(poly, q) to every part and plane of a ciphertext."""
    ct = _u64(ct)
    out = np.empty_like(ct)
    for part in range(2):
        for pl, q in enumerate(primes):
            out[part, pl] = fn(ct[part, pl], q)
    return out


def tweak_def(cts, primes) -> np.ndarray:
    """ct'_j = sum_{i<n} X^(2ijN/n) ct_i (the definition in Alg. 3)."""
    cts = _u64(cts)
    n, _, L, N = cts.shape
    out = np.empty_like(cts)
    pr = _u64(primes[:L])
    _load().or_tweak_def(n, N, L, _ptr(pr), _ptr(cts), _ptr(out))
    return out


def tweak_alg(cts, primes) -> np.ndarray:
    """Alg. 3 (Tweak), its recursion as stated."""
    cts = _u64(cts)
    n, _, L, N = cts.shape
    out = np.empty_like(cts)
    pr = _u64(primes[:L])
    _load().or_tweak_alg(n, N, L, _ptr(pr), _ptr(cts), _ptr(out))
    return out


def gadget_digits(L: int, dnum: int) -> list[range]:
    """Chain primes of each digit of the RNS gadget with dnum digits:
    consecutive groups of alpha = ceil(L / dnum) primes, the last one shorter."""
    alpha = -(-L // dnum)
    return [range(d * alpha, min(L, (d + 1) * alpha)) for d in range(dnum)]


def ks_keygen(s_old, s_new, primes_with_P, a, e, L=None, dnum=None) -> np.ndarray:
    """Switching key s_old -> s_new modulo P*Q with the RNS gadget of dnum
    digits (SWKGen of Sec. 2.2 with gadget rank dnum).  primes_with_P: the L
    chain primes, then the K special primes whose product is P (L defaults
    to K = 1; dnum to L, one digit per chain prime).  a: [dnum, L+K, N]
    uniform; e: [dnum, N] small.  Returns [dnum, 2, L+K, N]."""
    Lp = len(primes_with_P)
    L = Lp - 1 if L is None else L
    dnum = L if dnum is None else dnum
    N = len(s_old)
    key = np.empty((dnum, 2, Lp, N), dtype=np.uint64)
    pr = _u64(primes_with_P)
    so = np.ascontiguousarray(s_old, dtype=np.int64)
    sn = np.ascontiguousarray(s_new, dtype=np.int64)
    a64 = _u64(a)
    e64 = np.ascontiguousarray(e, dtype=np.int64)
    assert a64.shape == (dnum, Lp, N) and e64.shape == (dnum, N)
    _check(_load().or_ks_keygen_g(N, L, Lp - L, dnum, _ptr(pr), _ptr(so), _ptr(sn), _ptr(a64),
                                  _ptr(e64), _ptr(key)),
           "ks_keygen")
    return key


def keyswitch(ct, key, primes_with_P) -> np.ndarray:
    """KeySwitch: digit d = [a]_{Q_d} (exact CRT lift of a's residues on the
    digit's primes), sum digit_d * key_d mod PQ, divide by P (rounded).  The
    gadget is read off the key: [dnum, 2, L+K, N]."""
    ct = _u64(ct)
    _, L, N = ct.shape
    key64 = _u64(key)
    dnum, _, Lp, _ = key64.shape
    assert len(primes_with_P) == Lp
    out = np.empty_like(ct)
    pr = _u64(primes_with_P)
    _check(_load().or_keyswitch_g(N, L, Lp - L, dnum, _ptr(pr), _ptr(key64), _ptr(ct),
                                  _ptr(out)), "keyswitch")
    return out


def rescale(ct, primes) -> np.ndarray:
    """Rescale by the last prime of the chain: round(x / q_{L-1}), L-1 planes."""
    ct = _u64(ct)
    _, L, N = ct.shape
    out = np.empty((2, L - 1, N), dtype=np.uint64)
    pr = _u64(primes[:L])
    _load().or_rescale(N, L, _ptr(pr), _ptr(ct), _ptr(out))
    return out


def negacyclic_int(a, b) -> np.ndarray:
    """Product in Z[X]/(X^N+1) of two small integer polynomials (exact, int64)."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    N = len(a)
    full = np.convolve(a, b)
    out = full[:N].copy()
    out[: N - 1] -= full[N:]
    return out


def aut_key_secret(s, ell: int) -> np.ndarray:
    """s(X^ell) over the integers (the secret an automorphism key switches from)."""
    N = len(s)
    out = np.zeros(N, dtype=np.int64)
    for i, v in enumerate(np.asarray(s, dtype=np.int64)):
        p = (i * ell) % (2 * N)
        if p < N:
            out[p] += v
        else:
            out[p - N] -= v
    return out


def aut_ct(ct, ell: int, key, primes_with_P) -> np.ndarray:
    """Aut (Sec. 2.2): ct(X^ell), then KeySwitch s(X^ell) -> s (none for ell = 1)."""
    L = ct.shape[1]
    sig = ct_map(ct, primes_with_P[:L], lambda m, q: automorphism(m, ell, q))
    if ell == 1:
        return sig
    return keyswitch(sig, key, primes_with_P)


def transpose(cts, aut_keys, primes_with_P) -> np.ndarray:
    """Alg. 4 (Transpose) on N ciphertexts [N, 2, L, N].  aut_keys[j] switches
    s(X^(2j+1)) -> s (aut_keys[0] unused)."""
    cts = _u64(cts)
    N, _, L, _ = cts.shape
    primes = list(primes_with_P[:L])
    # Step 1: aux = Tweak((X^i ct_i)_i)
    shifted = np.stack([ct_map(cts[i], primes, lambda m, q, i=i: monomial_mul(m, i, q))
                        for i in range(N)])
    aux = tweak_alg(shifted, primes)
    # Steps 2-5: aux'_j = Aut(N^-1 * aux_{((2j+1)^-1 mod 2N - 1)/2}, 2j+1)
    auxp = np.empty_like(aux)
    ninv = [pow(N, -1, q) for q in primes]
    for j in range(N):
        ell = 2 * j + 1
        src = (pow(ell, -1, 2 * N) - 1) // 2
        scaled = aux[src].copy()
        for pl, q in enumerate(primes):
            for part in range(2):
                scaled[part, pl] = (scaled[part, pl].astype(object) * ninv[pl] % q).astype(np.uint64)
        auxp[j] = aut_ct(scaled, ell, aut_keys[j], primes_with_P)
    # Step 6: ct'' = Tweak(aux')
    ctpp = tweak_alg(auxp, primes)
    # Steps 7-9: ct'_{j mod N} = -X^(N-j) ct''_{N-j}, j = 1..N  (-X^(N-j) = X^(2N-j)).
    # Reading of the last iteration (j = N, ct'_0): the proof of the transpose
    # theorem uses -Tr(X^j m)/N = m_{N-j}, which holds for 1 <= j < N (the
    # constant term of X^j m is -m_{N-j}); for j = 0 the constant term is +m_0,
    # so the ensured ct'_0 (column 0) is +ct''_0, without the minus sign.
    out = np.empty_like(ctpp)
    for j in range(1, N):
        out[j] = ct_map(ctpp[N - j], primes, lambda m, q, j=j: monomial_mul(m, 2 * N - j, q))
    out[0] = ctpp[0]
    return out


def ct_add(x, y, primes) -> np.ndarray:
    out = np.empty_like(x)
    for pl, q in enumerate(primes):
        out[..., pl, :] = ((x[..., pl, :].astype(object) + y[..., pl, :].astype(object)) % q
                           ).astype(np.uint64)
    return out


def cc_mm(ct1, ct2, aut_keys, relin_key, primes_with_P):
    """Alg. 8 (CC-MM) on column-wise encryptions [N, 2, L, N] (ciphertext j is
    column j of the matrix).  Returns the column-wise encryption of M1*M2 after
    Rescale by q_{L-1}, [N, 2, L-1, N], and the intermediate blocks."""
    rw = transpose(ct2, aut_keys, primes_with_P)                     # Step 1
    out, blocks = cc_mm_rowwise(ct1, rw, aut_keys, relin_key, primes_with_P)
    blocks["row_wise"] = rw
    return out, blocks


def cc_mm_rowwise(ct1, rw, aut_keys, relin_key, primes_with_P):
    """Alg. 8 with Step 1 omitted, for a row-wise encrypted right operand (the
    "row or column" remark after Thm th:ccmm): ct1 holds n column-wise
    encryptions [n, 2, L, N] of an N x n matrix M (ciphertext j is column j),
    rw holds n row-wise encryptions [n, 2, L, N] of an n x N matrix M'
    (ciphertext t is row t), 1 <= n <= N.  Steps 2-5 as in Alg. 8; returns the
    column-wise encryption of M*M' (N x N) after Rescale, [N, 2, L-1, N], and
    the intermediate blocks."""
    ct1 = _u64(ct1)
    rw = _u64(rw)
    n, _, L, N = ct1.shape
    assert rw.shape == (n, 2, L, N)
    primes = list(primes_with_P[:L])
    C = np.empty((L, 2 * N, 2 * N), dtype=np.uint64)
    for pl, q in enumerate(primes):
        # [A; B] (2N x n): row r of A holds coefficient r of every column ciphertext.
        Ub = np.concatenate([ct1[:, 0, pl, :].T, ct1[:, 1, pl, :].T])
        # [A~' B~'] (n x 2N): row t is the row-wise ciphertext t (a-part then b-part).
        Wb = np.concatenate([rw[:, 0, pl, :], rw[:, 1, pl, :]], axis=1)
        C[pl] = mod_pp_mm_residues(Ub, Wb, q)                      # Step 2
    C00, C01 = C[:, :N, :N], C[:, :N, N:]
    C10, C11 = C[:, N:, :N], C[:, N:, N:]

    def rows_as_cts(Cx):  # row i of Cx is the a-part of ciphertext i, b = 0
        cts = np.zeros((N, 2, L, N), dtype=np.uint64)
        cts[:, 0] = np.transpose(Cx, (1, 0, 2))
        return cts

    D01 = transpose(rows_as_cts(C00), aut_keys, primes_with_P)      # Step 3
    D23 = transpose(rows_as_cts(C10), aut_keys, primes_with_P)      # Step 4
    out = np.empty((N, 2, L - 1, N), dtype=np.uint64)
    for j in range(N):                                               # Step 5
        r = np.zeros((2, L, N), dtype=np.uint64)
        r[0] = D01[j, 0]
        rl = keyswitch(r, relin_key, primes_with_P)                  # Relin(D0, 0)
        extra = np.zeros((2, L, N), dtype=np.uint64)
        extra[0] = ct_add(D01[j, 1], D23[j, 0], primes)              # D1 + D2
        extra[0] = ct_add(extra[0], C01[:, :, j], primes)            # + C01 (column j)
        extra[1] = ct_add(D23[j, 1], C11[:, :, j], primes)           # D3 + C11
        out[j] = rescale(ct_add(rl, extra, primes), primes)
    return out, {"C": C, "D01": D01, "D23": D23}


def pcmm_precomp(cts, U, keys, primes_with_P, rescale_out: bool = False):
    """Alg. 7 (CP-MM with precomputation) on a shared-a RLWE encryption,
    followed by the key switches back to one secret (Thm th:pcmm-with-precomp
    and the remark after it: switching before Rescale keeps more precision).

    cts: [d2, 2, L, N] ciphertexts (a, b_j) that share one a-part; ciphertext
         j encrypts column j of M under the secret s_j (column j of S), so
         Toep(a) * S + B = Delta * M + E with B's columns the b_j.
    U:   (d2, d3) integers, the plaintext known beforehand.
    keys: d3 switching keys [L, 2, L+1, N]; key k switches
         s'_k = sum_j U[j, k] s_j (column k of S * U) to the target secret.
    Step 1 (Alg. 7): B' = B * U mod q, so that Toep(a) * (S * U) + B' =
    Delta * M * U + E * U: ciphertext k, (a, column k of B'), encrypts column
    k of M * U under s'_k.  Then each (a, b'_k) is key-switched with key k,
    and Rescale by q_{L-1} is applied when rescale_out is set.
    Returns (out [d3, 2, L or L-1, N], {"B1": B' as [d3, L, N]})."""
    cts = _u64(cts)
    d2, _, L, N = cts.shape
    primes = list(primes_with_P[:L])
    a = cts[0, 0]
    if not all(np.array_equal(cts[j, 0], a) for j in range(d2)):
        raise ValueError("the ciphertexts must share one a-part")
    U = np.asarray(U)
    d3 = U.shape[1]
    Bt = np.ascontiguousarray(np.transpose(cts[:, 1], (1, 0, 2)))    # [L, d2, N]: row j = b_j
    B1 = mod_pp_mm(np.ascontiguousarray(U.T), Bt, primes)           # row k = sum_j U[j,k] b_j
    out = np.empty((d3, 2, L - 1 if rescale_out else L, N), dtype=np.uint64)
    for k in range(d3):
        ct = np.empty((2, L, N), dtype=np.uint64)
        ct[0] = a
        ct[1] = B1[:, k, :]
        sw = keyswitch(ct, keys[k], primes_with_P)
        out[k] = rescale(sw, primes) if rescale_out else sw
    return out, {"B1": np.ascontiguousarray(np.transpose(B1, (1, 0, 2)))}
