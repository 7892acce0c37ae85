// Multi-modular (CRT) form of the wide Mod-PP-MM; see rns_wide.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace modpp {

constexpr int kMaxRnsPrimes = 32;
constexpr int kMaxRnsChunks = 4;  // pieces of the inner dimension

struct RnsPrime {
    uint32_t p;    // odd prime < 256
    uint32_t mag;  // floor(2^32 / p)
    uint32_t t21;  // 2^21 mod p
    uint32_t t42;  // 2^42 mod p
};
struct RnsPrimes {
    int R;
    int chunks;         // the inner dimension runs as 1..kMaxRnsChunks products (chunk_len each)
    int64_t chunk_len;  // multiple of 64 when chunks > 1
    RnsPrime p[kMaxRnsPrimes];
};
// Constants of the CRT recombination modulo one chain prime q.
struct RnsCrt {
    int R;
    int chunks;                   // residue planes per prime, summed before the CRT
    uint64_t q;
    uint64_t mq, mqs;             // M mod q and its Shoup quotient
    int p[kMaxRnsPrimes];
    int c[kMaxRnsPrimes];         // (M / p_i)^-1 mod p_i
    uint32_t wlo[kMaxRnsPrimes];  // (M / p_i) mod q, low and high 32 bits
    uint32_t whi[kMaxRnsPrimes];
    uint64_t mu;                  // Barrett constant of q
    uint64_t t32, t32s;           // 2^32 mod q and its Shoup quotient
};
struct RnsLayout {
    int64_t kp, nblk;
    size_t off_u16, off_d, off_res, total;
};

// Small primes for inner dimension k and the chain primes qs, product
// M >= 2.8 k ((q-1)/2)^2.  The inner dimension runs in c = 1..kMaxRnsChunks
// pieces of length len with len B^2 < 2^24 (residues |r| <= B <= 125),
// choosing the c with the fewest primes (5% cost per extra piece).  False
// when no set of at most kMaxRnsPrimes primes exists.
bool rns_choose(int64_t k, const uint64_t *qs, int P, RnsPrimes *out);
RnsCrt rns_crt_consts(const RnsPrimes &pr, uint64_t q);
// Workspace of one chain prime's products (reused across chain primes).
RnsLayout rns_layout(int64_t d, int64_t k, int64_t n, const RnsPrimes &pr);
// Rows of the U map (R * d) and of the residue matrix map (R * nblk * 256).
constexpr int kRnsTileCols = 256;
// The three passes of C = U * A mod q for one chain prime (U d x k, A k x n
// residues): residue planes of U (skipped when split_u is false: the planes
// from the previous call are reused) and of A; the small-prime products
// (tmU / tmD describe the f16 planes at ws + off_u16 / off_d); the CRT
// recombination into C.  Each returns 0 or a negative modpp_status.
int rns_split(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu, const uint64_t *A,
              int64_t lda, uint64_t q, const RnsPrimes &pr, const RnsLayout &lay, uint8_t *ws,
              bool split_u, cudaStream_t st);
// tmU / tmD: one pair of maps per chunk (base at the chunk's first inner
// index, inner extent the chunk's length).
int rns_gemm(int64_t d, int64_t k, int64_t n, const RnsPrimes &pr, const RnsLayout &lay,
             uint8_t *ws, int *status, uint64_t timeout_ns, int num_sms, const CUtensorMap *tmU,
             const CUtensorMap *tmD, cudaStream_t st);
int rns_crt(int64_t d, int64_t n, uint64_t *C, int64_t ldc, uint64_t q, const RnsPrimes &pr,
            const RnsLayout &lay, uint8_t *ws, cudaStream_t st);

}  // namespace modpp
