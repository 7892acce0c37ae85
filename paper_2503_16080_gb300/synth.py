"""Seeded synthetic inputs for the Mod-PP-MM path.

This module draws numbers and nothing else.  It holds none of the method's
arithmetic (no modular products, no encoding, no encryption).  Both the CUDA
path (tests, benchmark) and the test oracle take their inputs from here.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based stream: the i-th draw of
stream ``s`` under seed ``seed`` is mix(seed * G1 + s * G2 + (i + 1) * GAMMA).
It is vectorised over numpy uint64 with wrap-around arithmetic, so the
same (seed, stream, index) gives the same bits on every machine.

The distributions follow the paper's workloads (Sec. 6: i.i.d. uniform [-1, 1]
messages) and the symmetric RLWE recipe of Sec. 2.1: uniform a, ternary
secret, rounded Gaussian error.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_G1 = np.uint64(0xD1B54A32D192ED03)
_G2 = np.uint64(0xABC98388FB8FAC03)
_MASK32 = np.uint64(0xFFFFFFFF)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """`count` uniform 64-bit words: draws start .. start+count-1 of the stream."""
    with np.errstate(over="ignore"):
        base = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _G1
                + np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _G2)
        idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        return _mix(base + idx * _GAMMA)


def u64_at(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """The draws of the stream at the given flat indices (same bits as u64)."""
    with np.errstate(over="ignore"):
        base = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _G1
                + np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _G2)
        idx = np.asarray(index, dtype=np.uint64) + np.uint64(1)
        return _mix(base + idx * _GAMMA)


def _mulhi(x: np.ndarray, q: int) -> np.ndarray:
    """floor(x * q / 2^64) for uint64 x and q < 2^64, exactly, in uint64 pieces."""
    qh, ql = np.uint64(q >> 32), np.uint64(q & 0xFFFFFFFF)
    xh, xl = x >> np.uint64(32), x & _MASK32
    with np.errstate(over="ignore"):
        ll = xl * ql
        hl = xh * ql
        lh = xl * qh
        mid = (ll >> np.uint64(32)) + (hl & _MASK32) + (lh & _MASK32)
        return xh * qh + (hl >> np.uint64(32)) + (lh >> np.uint64(32)) + (mid >> np.uint64(32))


def uniform_mod(seed: int, stream: int, shape, q: int) -> np.ndarray:
    """Uniform residues in [0, q) (multiply-high mapping, bias < 2^-64 * q)."""
    n = int(np.prod(shape))
    return _mulhi(u64(seed, stream, n), int(q)).reshape(shape)


def uniform_mod_at(seed: int, stream: int, index: np.ndarray, q: int) -> np.ndarray:
    """Entries of uniform_mod(seed, stream, shape, q) at the given flat indices."""
    return _mulhi(u64_at(seed, stream, index), int(q))


def uniform_int8(seed: int, stream: int, shape) -> np.ndarray:
    """Uniform integers in [-128, 127] (int8 range)."""
    n = int(np.prod(shape))
    return (u64(seed, stream, n) >> np.uint64(56)).astype(np.uint8).view(np.int8).reshape(shape)


def uniform_int8_at(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Entries of uniform_int8(seed, stream, shape) at the given flat indices."""
    return (u64_at(seed, stream, index) >> np.uint64(56)).astype(np.uint8).view(np.int8)


def uniform_unit(seed: int, stream: int, shape) -> np.ndarray:
    """Uniform doubles in [-1, 1): multiples of 2^-52 (53-bit draws)."""
    n = int(np.prod(shape))
    v = (u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -52)
    return (v - 1.0).reshape(shape)


def _open01(seed: int, stream: int, n: int, start: int) -> np.ndarray:
    return ((u64(seed, stream, n, start) >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def normal(seed: int, stream: int, shape) -> np.ndarray:
    """Standard normal draws (Box-Muller on two independent halves of the stream)."""
    n = int(np.prod(shape))
    u1 = _open01(seed, stream, n, 0)
    u2 = _open01(seed, stream, n, n)
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).reshape(shape)


def quantised_normal_int8(seed: int, stream: int, shape, scale: float = 32.0) -> np.ndarray:
    """N(0,1) draws scaled by `scale`, rounded half-up and clamped to [-128, 127]:
    the 8-bit signed plaintext matrix of the PC-MM workloads."""
    x = np.floor(normal(seed, stream, shape) * scale + 0.5)
    return np.clip(x, -128, 127).astype(np.int8)


def ternary(seed: int, stream: int, n: int) -> np.ndarray:
    """Dense uniform ternary secret in {-1, 0, 1}."""
    return ((u64(seed, stream, n) % np.uint64(3)).astype(np.int64) - 1)


def rounded_gaussian(seed: int, stream: int, shape, sigma: float = 3.2,
                     tail: float = 6.0) -> np.ndarray:
    """Rounded Gaussian error of width sigma, tail-cut at tail*sigma."""
    x = np.clip(normal(seed, stream, shape) * sigma, -tail * sigma, tail * sigma)
    return np.floor(x + 0.5).astype(np.int64)


# --------------------------------------------------------------------------
# RNS primes (parameters, not arithmetic of the method)
# --------------------------------------------------------------------------

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (first twelve prime bases)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(bits: int, count: int, two_adicity: int = 17, exclude: Sequence[int] = ()) -> list[int]:
    """The `count` largest primes q < 2^bits with q = 1 mod 2^two_adicity,
    in descending order (NTT-friendly up to ring degree 2^(two_adicity-1))."""
    step = 1 << two_adicity
    q = ((1 << bits) - 1) // step * step + 1
    out: list[int] = []
    while len(out) < count and q > (1 << (bits - 1)):
        if q not in exclude and is_prime(q):
            out.append(q)
        q -= step
    if len(out) < count:
        raise ValueError("not enough primes of that shape")
    return out


def random_primes(seed: int, stream: int, count: int, lo_bits: int, hi_bits: int) -> list[int]:
    """`count` distinct primes whose bit lengths are drawn uniformly in [lo_bits, hi_bits]."""
    out: list[int] = []
    words = u64(seed, stream, 64 * count)
    i = 0
    while len(out) < count:
        b = lo_bits + int(words[i] % np.uint64(hi_bits - lo_bits + 1))
        c = (1 << (b - 1)) | (int(words[i + 1]) & ((1 << (b - 1)) - 1)) | 1
        i += 2
        while not is_prime(c):
            c += 2
            if c >= (1 << b):
                c = (1 << (b - 1)) + 1
        if c not in out:
            out.append(c)
    return out


# --------------------------------------------------------------------------
# The same streams drawn on a torch device (bit-identical to the numpy ones).
# Large residue matrices are generated where they are used; the CPU can
# regenerate any sampled entry through the *_at functions above.
# --------------------------------------------------------------------------

def _to_i64(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _shr(x, k: int):
    """Logical right shift of an int64 tensor holding uint64 bits."""
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(x, k), _to_i64((1 << (64 - k)) - 1))


def u64_torch(seed: int, stream: int, count: int, device, start: int = 0):
    """Same bits as u64(seed, stream, count, start), as an int64 tensor on `device`."""
    import torch
    base = _to_i64((seed & 0xFFFFFFFFFFFFFFFF) * 0xD1B54A32D192ED03
                   + (stream & 0xFFFFFFFFFFFFFFFF) * 0xABC98388FB8FAC03)
    z = torch.arange(start + 1, start + 1 + count, dtype=torch.int64, device=device)
    z = z * _to_i64(0x9E3779B97F4A7C15) + base
    z = torch.bitwise_xor(z, _shr(z, 30)) * _to_i64(0xBF58476D1CE4E5B9)
    z = torch.bitwise_xor(z, _shr(z, 27)) * _to_i64(0x94D049BB133111EB)
    return torch.bitwise_xor(z, _shr(z, 31))


def uniform_mod_torch(seed: int, stream: int, shape, q: int, device, chunk: int = 1 << 26):
    """uniform_mod(seed, stream, shape, q) generated on `device` (torch.uint64)."""
    import torch
    n = int(np.prod(shape))
    out = torch.empty(n, dtype=torch.int64, device=device)
    qh, ql = int(q) >> 32, int(q) & 0xFFFFFFFF
    m32 = 0xFFFFFFFF
    for s0 in range(0, n, chunk):
        cnt = min(chunk, n - s0)
        x = u64_torch(seed, stream, cnt, device, start=s0)
        xh, xl = _shr(x, 32), torch.bitwise_and(x, m32)
        ll, hl, lh = xl * ql, xh * ql, xl * qh
        mid = _shr(ll, 32) + torch.bitwise_and(hl, m32) + torch.bitwise_and(lh, m32)
        out[s0:s0 + cnt] = xh * qh + _shr(hl, 32) + _shr(lh, 32) + _shr(mid, 32)
    return out.view(torch.uint64).reshape(shape)


def uniform_int8_torch(seed: int, stream: int, shape, device, chunk: int = 1 << 26):
    """uniform_int8(seed, stream, shape) generated on `device` (torch.int8)."""
    import torch
    n = int(np.prod(shape))
    out = torch.empty(n, dtype=torch.int8, device=device)
    for s0 in range(0, n, chunk):
        cnt = min(chunk, n - s0)
        x = u64_torch(seed, stream, cnt, device, start=s0)
        # top byte as a signed int8: arithmetic shift keeps the sign bit
        out[s0:s0 + cnt] = torch.bitwise_right_shift(x, 56).to(torch.int8)
    return out.reshape(shape)


def uniform_unit_torch(seed: int, stream: int, shape, device, chunk: int = 1 << 26):
    """uniform_unit(seed, stream, shape) generated on `device` (float64, same values)."""
    import torch
    n = int(np.prod(shape))
    out = torch.empty(n, dtype=torch.float64, device=device)
    for s0 in range(0, n, chunk):
        cnt = min(chunk, n - s0)
        x = u64_torch(seed, stream, cnt, device, start=s0)
        out[s0:s0 + cnt] = _shr(x, 11).to(torch.float64) * (2.0 ** -52) - 1.0
    return out.reshape(shape)


def rounded_gaussian_torch(seed: int, stream: int, shape, device, sigma: float = 3.2,
                           tail: float = 6.0, chunk: int = 1 << 25):
    """The rounded_gaussian draw generated on `device` (int8; |e| <= tail * sigma < 128).
    Same Box-Muller formula on the same uniform bits; the device's log and cos
    may differ from the host's in the last bit, so a value can differ where
    the scaled draw sits on a rounding boundary."""
    import torch
    n = int(np.prod(shape))
    out = torch.empty(n, dtype=torch.int8, device=device)
    for s0 in range(0, n, chunk):
        cnt = min(chunk, n - s0)
        u1 = (_shr(u64_torch(seed, stream, cnt, device, start=s0), 11).to(torch.float64) + 0.5) \
            * 2.0 ** -53
        u2 = (_shr(u64_torch(seed, stream, cnt, device, start=n + s0), 11).to(torch.float64)
              + 0.5) * 2.0 ** -53
        x = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2) * sigma
        x = torch.clamp(x, -tail * sigma, tail * sigma)
        out[s0:s0 + cnt] = torch.floor(x + 0.5).to(torch.int8)
    return out.reshape(shape)
