// Device-side modular arithmetic on 64-bit residues.
//   Barrett reduction (P. Barrett, CRYPTO 1986) with mu = floor(2^64/q);
//   Shoup's precomputed-quotient multiplication (V. Shoup, NTL) for a fixed
//   multiplier w with w' = floor(w * 2^64 / q).
// Moduli satisfy 2 < q < 2^62, so 3q fits in 64 bits.
#pragma once
#include <cstdint>

namespace modpp {

// t mod q for any 64-bit t.  floor(t*mu/2^64) underestimates floor(t/q) by
// at most 2, so at most two corrections follow.
__device__ __forceinline__ uint64_t barrett_u64(uint64_t t, uint64_t q, uint64_t mu) {
    uint64_t r = t - __umul64hi(t, mu) * q;
    if (r >= q) r -= q;
    if (r >= q) r -= q;
    return r;
}

// Canonical residue of a signed 64-bit value.
__device__ __forceinline__ uint64_t smod_i64(int64_t x, uint64_t q, uint64_t mu) {
    const uint64_t mag = x < 0 ? static_cast<uint64_t>(-(x + 1)) + 1u : static_cast<uint64_t>(x);
    const uint64_t r = barrett_u64(mag, q, mu);
    return (x < 0 && r != 0) ? q - r : r;
}

// a * w mod q for a < 2^64 and w < q, given ws = floor(w * 2^64 / q).
__device__ __forceinline__ uint64_t shoup_mulmod(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    const uint64_t qh = __umul64hi(a, ws);
    uint64_t r = a * w - qh * q;
    if (r >= q) r -= q;
    return r;
}

// a * w mod q up to one multiple of q: the result lies in [0, 2q).
__device__ __forceinline__ uint64_t shoup_lazy(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    return a * w - __umul64hi(a, ws) * q;
}

// a * w mod q up to three multiples of q, [0, 4q), for any 64-bit a: Shoup's
// quotient from three of the four 32 x 32-bit partial products of a * ws.
// The low product and the low halves of the two middle ones are each below
// 2^64 after scaling, so the quotient falls short of floor(a * ws / 2^64) by
// at most 2, and the remainder of the exact quotient is below 2q.
__device__ __forceinline__ uint64_t shoup_lazy3(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
    const uint32_t a0 = static_cast<uint32_t>(a), a1 = static_cast<uint32_t>(a >> 32);
    const uint32_t s0 = static_cast<uint32_t>(ws), s1 = static_cast<uint32_t>(ws >> 32);
    const uint64_t qh = static_cast<uint64_t>(a1) * s1 + __umulhi(a1, s0) + __umulhi(a0, s1);
    return a * w - qh * q;
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    const uint64_t s = a + b;
    return s >= q ? s - q : s;
}

// Montgomery product a * b * 2^-64 mod q for any 64-bit a and b < q, q odd
// < 2^62 (a * b + t * q < 2^65 q, so one subtraction reaches [0, q));
// qinv = -q^-1 mod 2^64.
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t q, uint64_t qinv) {
    const uint64_t lo = a * b;
    const uint64_t hi = __umul64hi(a, b);
    const uint64_t t = lo * qinv;
    const uint64_t th = __umul64hi(t, q);
    // (lo + t*q) is a multiple of 2^64; its carry out of the low word is 1
    // unless lo == 0.
    uint64_t r = hi + th + (lo != 0 ? 1u : 0u);
    if (r >= q) r -= q;
    return r;
}

}  // namespace modpp
