// Device side of the key-switching gadget (KsGadget, ring_internal.h): the
// digits of an a-part (ModUp) and the centred residue [u]_P (ModDown).
#pragma once
#include <cstdint>

#include "modarith.cuh"
#include "ring_internal.h"

namespace modpp {

// First chain prime and prime count of digit d.
__host__ __device__ __forceinline__ int gadget_lo(const KsGadget &g, int d) { return d * g.alpha; }
__host__ __device__ __forceinline__ int gadget_count(const KsGadget &g, int d) {
    const int hi = (d + 1) * g.alpha;
    return (hi < g.L ? hi : g.L) - d * g.alpha;
}

// Garner's second mixed-radix digit of a two-prime gadget digit at one
// coefficient: v1 = (a_j1 - a_j0) * q_j0^-1 mod q_j1, canonical, so that the
// digit is the integer a_j0 + q_j0 * v1 in [0, q_j0 q_j1).
__device__ __forceinline__ uint64_t garner_v1(const KsGadget &g, const NttPlane *tab, int d,
                                              uint64_t a_j0, uint64_t a_j1) {
    const NttPlane &t1 = tab[gadget_lo(g, d) + 1];
    return shoup_mulmod(sub_mod(a_j1, barrett_u64(a_j0, t1.q, t1.mu), t1.q), g.ginv[d],
                        g.ginv_s[d], t1.q);
}

// Digit d of one a-part for target plane k: a0 points to the a-part's
// coefficients mod q_j0, v1 (two-prime digits only) to their Garner digits.
struct DigitSrc {
    const uint64_t *a0, *v1;  // v1 null: one-prime digit
    uint64_t c, c_s;          // q_j0 mod q_k, Shoup quotient
};

__device__ __forceinline__ DigitSrc make_digit_src(const KsGadget &g, const uint64_t *a_j0,
                                                   const uint64_t *v1, int d, int k) {
    DigitSrc s{};
    s.a0 = a_j0;
    if (gadget_count(g, d) == 2) {
        const int Lp = g.L + g.K;
        s.v1 = v1;
        s.c = g.cq[d * Lp + k];
        s.c_s = g.cq_s[d * Lp + k];
    }
    return s;
}

// The digit at coefficient j modulo q.  Unreduced (reduce false), a
// one-prime digit is below the largest chain prime and a two-prime digit
// below q_j0 + 4q; reduced, the canonical residue.
// TWO: the digit is known to have two primes (v1 present).
template <bool TWO = false>
__device__ __forceinline__ uint64_t digit_at(const DigitSrc &s, int64_t j, uint64_t q, uint64_t mu,
                                             bool reduce) {
    uint64_t x = s.a0[j];
    if (TWO || s.v1) x += shoup_lazy3(s.v1[j], s.c, s.c_s, q);
    return reduce ? barrett_u64(x, q, mu) : x;
}

// Largest unreduced digit value for target prime q.
__host__ __device__ __forceinline__ uint64_t digit_bound(const KsGadget &g, uint64_t q) {
    return g.alpha == 2 ? g.chain_max + 4 * q : g.chain_max;
}

// ModDown's [u]_P centred, as a residue mod chain prime k, for the special
// residues u0 (mod p0) and u1 (mod p1, two special primes only); tab holds
// the special primes at planes L, L+1.
struct CentredP {
    uint64_t v0, v1;
    bool neg;
};
__device__ __forceinline__ CentredP centred_p_digits(const KsGadget &g, const NttPlane *tab,
                                                     uint64_t u0, uint64_t u1) {
    CentredP c{};
    c.v0 = u0;
    if (g.K == 1) {
        c.neg = u0 > tab[g.L].q / 2;
    } else {
        const NttPlane &p1 = tab[g.L + 1];
        c.v1 = shoup_mulmod(sub_mod(u1, barrett_u64(u0, p1.q, p1.mu), p1.q), g.p0inv, g.p0inv_s,
                            p1.q);
        c.neg = c.v1 > g.m1 || (c.v1 == g.m1 && c.v0 >= g.h0);
    }
    return c;
}
__device__ __forceinline__ uint64_t centred_p_mod(const KsGadget &g, const NttPlane *tab,
                                                  const CentredP &c, int k) {
    const uint64_t q = tab[k].q, mu = tab[k].mu;
    if (g.K == 1) {
        const uint64_t P = tab[g.L].q;
        if (c.neg) {
            const uint64_t mag = barrett_u64(P - c.v0, q, mu);
            return mag == 0 ? 0 : q - mag;
        }
        return barrett_u64(c.v0, q, mu);
    }
    uint64_t r = add_mod(barrett_u64(c.v0, q, mu), shoup_mulmod(c.v1, g.p0k[k], g.p0k_s[k], q), q);
    return c.neg ? sub_mod(r, g.Pk[k], q) : r;
}

}  // namespace modpp
