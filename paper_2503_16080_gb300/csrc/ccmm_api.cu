// Host side of the ring / CC-MM ABI declared in include/modpp_ring.h: ring
// tables, workspace layouts and the kernel sequence of KeySwitch, Tweak
// (Alg. 3), Transpose (Alg. 4) and CC-MM (Alg. 8).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "modpp.h"
#include "modpp_internal.h"
#include "modpp_ring.h"
#include "ring_internal.h"

using namespace modpp;

struct modpp_ring_s {
    int64_t N = 0;
    int L = 0;
    int K = 1;                     // special primes
    int Dg = 0;                    // gadget digits (dnum)
    int logN = 0;
    std::vector<uint64_t> primes;  // L + K: chain, then the special primes
    char *mem = nullptr;           // caller's device memory holding the tables
    const NttPlane *tab = nullptr; // [L + K]
    KsGadget g{};                  // the key-switching gadget (device pointers into mem)
    const uint64_t *pinv = nullptr, *pinv_s = nullptr;    // P^-1 mod q_k, k < L
    const uint64_t *qlinv = nullptr, *qlinv_s = nullptr;  // q_{L-1}^-1 mod q_k, k < L-1
    const uint64_t *ninv = nullptr, *ninv_s = nullptr;    // N^-1 mod q_k, k < L
    const int *t2_src = nullptr, *t2_ellinv = nullptr, *t2_kid = nullptr;
    const int *kid_zero = nullptr;
    int *status = nullptr;         // status word of the ring (debug range checks)
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool timed = false;
};

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxChain = 16;
constexpr int64_t kMaxN = 16384;
// Bytes of key-switching scratch (digits and products) one chunk may use;
// MODPP_KS_CHUNK_BYTES overrides it.
constexpr size_t kKsChunkBytes = size_t(1) << 31;
size_t ks_chunk_budget() {
    if (const char *v = std::getenv("MODPP_KS_CHUNK_BYTES")) {
        const long long x = std::atoll(v);
        if (x > 0) return static_cast<size_t>(x);
    }
    return kKsChunkBytes;
}

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
int cuda_status(cudaError_t e) { return e == cudaSuccess ? MODPP_OK : MODPP_ERR_CUDA; }

using u128 = unsigned __int128;
uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return static_cast<uint64_t>(static_cast<u128>(a) * b % q);
}
uint64_t powmod(uint64_t b, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}
// Inverse modulo a prime by Fermat's little theorem.
uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a % q, q - 2, q); }
uint64_t shoup(uint64_t w, uint64_t q) {
    return static_cast<uint64_t>((static_cast<u128>(w) << 64) / q);
}
bool is_prime_u64(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull})
        if (n % p == 0) return n == p;
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    // Miller-Rabin with the first 12 prime bases is deterministic below 3.3e24.
    for (uint64_t a : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}
// A primitive 2N-th root of unity mod q (q = 1 mod 2N, N a power of two):
// x = g^((q-1)/2N) has order dividing 2N, and exactly 2N when x^N = -1.
uint64_t find_psi(uint64_t q, uint64_t N) {
    for (uint64_t g = 2; g < q; ++g) {
        const uint64_t x = powmod(g, (q - 1) / (2 * N), q);
        if (powmod(x, N, q) == q - 1) return x;
    }
    return 0;
}
unsigned bitrev(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}
int log2_exact(int64_t x) {
    int l = 0;
    while ((int64_t(1) << l) < x) ++l;
    return (int64_t(1) << l) == x ? l : -1;
}

// Layout of the ring tables inside the caller's memory.
struct RingLayout {
    size_t tab, tables, consts, gadget, ints, status, total;
};
RingLayout ring_layout(int64_t N, int L, int K) {
    RingLayout r{};
    const int Lp = L + K;
    size_t off = 0;
    r.tab = off;
    off = align_up(off + sizeof(NttPlane) * Lp);
    r.tables = off;
    off = align_up(off + sizeof(uint64_t) * 8 * Lp * N);
    r.consts = off;
    off = align_up(off + sizeof(uint64_t) * 6 * Lp);
    r.gadget = off;  // cq, cq_s [kMaxGadgetDigits][L+K]; p0k, p0k_s, Pk [L]
    off = align_up(off + sizeof(uint64_t) * (2 * kMaxGadgetDigits * Lp + 3 * L));
    r.ints = off;
    off = align_up(off + sizeof(int) * (3 * N + 1));
    r.status = off;
    off = align_up(off + sizeof(int));
    r.total = off;
    return r;
}

int64_t batch_words(const modpp_ring_s *r, int64_t n, int L) { return 2 * L * n * r->N; }

// Planes of key switching: chain and special primes.
int ks_planes(const modpp_ring_s *r) { return r->L + r->K; }
// Words of one switching key: [D][2][L+K][N].
int64_t key_words(const modpp_ring_s *r) {
    return static_cast<int64_t>(r->Dg) * 2 * ks_planes(r) * r->N;
}

// Garner digits (two-prime gadget digits): one row per digit and ciphertext.
bool ks_two_prime(const modpp_ring_s *r) { return r->g.alpha == 2; }

// Ciphertexts per key-switching chunk and the chunk's scratch words.
int64_t ks_chunk(const modpp_ring_s *r, int64_t n) {
    const int64_t Lp = ks_planes(r);
    const int64_t per_ct = static_cast<int64_t>(r->Dg) * Lp * r->N + 2 * Lp * r->N +
                           (ks_two_prime(r) ? r->Dg * r->N : 0);
    int64_t nb = static_cast<int64_t>(ks_chunk_budget() / 8) / per_ct;
    nb = std::max<int64_t>(1, std::min(nb, n));
    return nb;
}
size_t ks_scratch_bytes(const modpp_ring_s *r, int64_t n) {
    if (n == 0) return 0;
    const int64_t nb = ks_chunk(r, n);
    const int64_t Lp = ks_planes(r);
    return align_up(sizeof(uint64_t) * nb * r->Dg * Lp * r->N) +
           align_up(sizeof(uint64_t) * nb * 2 * Lp * r->N) +
           (ks_two_prime(r) ? align_up(sizeof(uint64_t) * nb * r->Dg * r->N) : 0);
}

// KeySwitch of ciphertexts [0, count) of a batch with plane stride n, written
// to a batch with plane stride n_out; key of ciphertext c: keys[kid[c % kper]]
// (kid < 0: copied unchanged).
int ks_run(const modpp_ring_s *r, const uint64_t *ct, int64_t n, int64_t count, uint64_t *out,
           int64_t n_out, const uint64_t *keys, const int *kid, int kper, int b_zero, char *scratch,
           cudaStream_t st) {
    if (count == 0) return MODPP_OK;
    const int Lp = ks_planes(r);
    const int N = static_cast<int>(r->N);
    const int64_t nb = ks_chunk(r, count);
    uint64_t *D = reinterpret_cast<uint64_t *>(scratch);
    uint64_t *U = reinterpret_cast<uint64_t *>(
        scratch + align_up(sizeof(uint64_t) * nb * r->Dg * Lp * r->N));
    uint64_t *V = ks_two_prime(r) ? U + align_up(sizeof(uint64_t) * nb * 2 * Lp * r->N) / 8
                                  : nullptr;
    for (int64_t c0 = 0; c0 < count; c0 += nb) {
        const int64_t m = std::min(nb, count - c0);
        cudaError_t e = cudaSuccess;
        if (V) e = launch_ks_garner(ct, n, N, c0, m, r->tab, r->g, V, st);
        if (e != cudaSuccess) return MODPP_ERR_CUDA;
        // One key for every ciphertext (relinearisation, modpp_keyswitch):
        // the fused kernel, whose key reads then hit L2.  One key per
        // ciphertext (the automorphisms of Alg. 4): the streaming
        // multiply-accumulate kernel reads the keys at full bandwidth.
        if (kper == 1 && ks_fused_supported(N)) {
            e = launch_ks_fused(ct, n, N, c0, m, r->tab, r->g, V, keys, kid, kper, U, st);
        } else {
            if (ntt_fast_supported(N)) {
                e = launch_ks_digits_ntt(ct, n, N, c0, m, r->tab, r->g, V, D, st);
            } else {
                e = launch_ks_decompose(ct, n, N, c0, m, r->tab, r->g, V, D, st);
                if (e == cudaSuccess)
                    e = launch_ntt(D, m * r->Dg * Lp, N, 1, Lp, r->tab, false, st);
            }
            if (e == cudaSuccess)
                e = launch_ks_multacc(D, keys, kid, kper, r->g, N, c0, m, r->tab, U, st);
            if (e == cudaSuccess) e = launch_ntt(U, m * 2 * Lp, N, 1, Lp, r->tab, true, st);
        }
        if (e == cudaSuccess)
            e = launch_ks_moddown(U, ct, n, N, c0, m, kid, kper, b_zero, r->tab, r->g, r->pinv,
                                  r->pinv_s, out, n_out, st);
        if (e != cudaSuccess) return MODPP_ERR_CUDA;
    }
    return MODPP_OK;
}

// A Tweak is log2(size) radix-2 stages (Alg. 3) over blocks of `size`
// ciphertexts in bit-reversed order; its passes run one to three stages each.
// Stages the next Tweak pass takes at stage half `half`: three (radix 8) or
// two (radix 4) while the group of 8h or 4h ciphertexts fits both the Tweak's
// size and the ring degree (even rotations), else one.
int tweak_pass_stages(int64_t half, int64_t size, int64_t N) {
    if (8 * half <= size && 8 * half <= N) return 3;
    if (4 * half <= size && 4 * half <= N) return 2;
    return 1;
}

// Where a Tweak's passes read first and write last.
struct TweakIO {
    const uint64_t *src = nullptr;  // the first pass reads here, through `in`, instead of a
    TweakMap in;                    // input map of the first pass
    uint64_t *dst = nullptr;        // the last pass writes here, through out_t3, instead of a / b
    int out_t3 = 0;
    uint64_t *land = nullptr;       // without dst: a or b, where the last pass must write
};

// The Tweak's passes on a batch of n ciphertexts (n / size independent Tweaks
// of size ciphertexts each), ping-ponging between a and b; returns the buffer
// holding the result.  Without io.src the first pass reads a (and writes b).
uint64_t *tweak_stages(const modpp_ring_s *r, uint64_t *a, uint64_t *b, int64_t n, int64_t size,
                       int L, cudaStream_t st, int *rc, int parts = 2,
                       const TweakIO &io = TweakIO{}) {
    *rc = MODPP_OK;
    const int N = static_cast<int>(r->N);
    int passes = 0;
    for (int64_t half = 1; half < size; ++passes) half <<= tweak_pass_stages(half, size, N);
    const uint64_t *in = io.src ? io.src : a;
    uint64_t *o = b;
    if (io.land && io.src) o = ((passes - 1) % 2 == 0) ? io.land : (io.land == a ? b : a);
    int p = 0;
    for (int64_t half = 1; half < size; ++p) {
        cudaError_t e;
        const int k = tweak_pass_stages(half, size, N);
        TweakMap mp{};
        if (p == 0) mp = io.in;
        uint64_t *dst = o;
        if (p == passes - 1 && io.dst) {
            dst = io.dst;
            mp.out_t3 = io.out_t3;
        }
        if (k == 3)
            e = launch_tweak_radix8(in, dst, n, L, N, half, r->tab, st, parts, mp);
        else if (k == 2)
            e = launch_tweak_radix4(in, dst, n, L, N, half, r->tab, st, parts, mp);
        else
            e = launch_tweak_stage(in, dst, n, L, N, half, r->tab, st, parts, mp);
        half <<= k;
        if (e != cudaSuccess) {
            *rc = MODPP_ERR_CUDA;
            return a;
        }
        in = dst;
        o = o == a ? b : a;
    }
    return const_cast<uint64_t *>(in);
}

size_t transpose_scratch(const modpp_ring_s *r, int64_t groups) {
    const int64_t n = groups * r->N;
    return 2 * align_up(sizeof(uint64_t) * batch_words(r, n, r->L)) + ks_scratch_bytes(r, n);
}

// Alg. 4 on `groups` matrices of N ciphertexts; scratch of transpose_scratch bytes.
// b_zero: every input b-part is zero (the (C00, 0) and (C10, 0) of Alg. 8):
// the first Tweak and the gather before the key switches then run on the
// a-parts only (a Tweak and Aut of zero are zero), the input's b-parts are
// never read, and the key switches produce the b-parts.
int transpose_run(const modpp_ring_s *r, const uint64_t *ct, uint64_t *out, int64_t groups,
                  const uint64_t *aut_keys, char *scratch, cudaStream_t st, bool b_zero = false) {
    const int parts1 = b_zero ? 1 : 2;
    const int L = r->L;
    const int N = static_cast<int>(r->N);
    const int64_t n = groups * r->N;
    if (n == 0) return MODPP_OK;
    const size_t bb = align_up(sizeof(uint64_t) * batch_words(r, n, L));
    uint64_t *x1 = reinterpret_cast<uint64_t *>(scratch);
    uint64_t *x2 = reinterpret_cast<uint64_t *>(scratch + bb);
    char *ks = scratch + 2 * bb;
    // Step 1: aux = Tweak((X^i ct_i)_i): the first pass reads ciphertext
    // brev(i) times X^brev(i) for position i (the stages' bit-reversed input).
    int rc = MODPP_OK;
    TweakIO io1;
    io1.src = ct;
    io1.in.in_bits = r->logN;
    io1.in.in_shift = 1;
    uint64_t *aux = tweak_stages(r, x1, x2, n, r->N, L, st, &rc, parts1, io1);
    if (rc) return rc;
    uint64_t *other = aux == x1 ? x2 : x1;
    // Steps 2-5: aux'_j = Aut(N^-1 aux_{((2j+1)^-1 - 1)/2}, 2j+1), written in
    // bit-reversed order for the second Tweak; then the key switches.
    GatherTables t2{};
    t2.per = N;
    t2.src = r->t2_src;
    t2.ellinv = r->t2_ellinv;
    t2.scale = r->ninv;
    t2.scale_s = r->ninv_s;
    if (launch_ct_gather(aux, other, n, L, N, t2, r->tab, st, parts1) != cudaSuccess)
        return MODPP_ERR_CUDA;
    rc = ks_run(r, other, n, n, other, n, aut_keys, r->t2_kid, N, b_zero ? 1 : 0, ks, st);
    if (rc) return rc;
    // Step 6: ct'' = Tweak(aux'); steps 7-9 in its last pass:
    // ct'_j = X^(2N-j) ct''_{N-j} (1 <= j < N), ct'_0 = ct''_0, written to out.
    TweakIO io2;
    io2.dst = out;
    io2.out_t3 = 1;
    tweak_stages(r, other, aux, n, r->N, L, st, &rc, 2, io2);
    return rc;
}

struct CcLayout {
    size_t wide, scratch, rw, ut, x, y, z, total;
};
// Workspace of CC-MM with inner dimension n (n = N for Alg. 8 as printed).
CcLayout cc_layout(const modpp_ring_s *r, int64_t n) {
    CcLayout c{};
    const int64_t N = r->N;
    const int L = r->L;
    const size_t wide = modpp_mm_wide_workspace(2 * N, n, N, r->primes.data(), L);
    const size_t tr = transpose_scratch(r, 2);
    size_t off = 0;
    // The Mod-PP-MM workspace (whose first word is the status word) and the
    // transpose scratch are used at different times and share one region.
    c.wide = off;
    c.scratch = off;
    off = align_up(off + std::max(wide, tr));
    c.rw = off;  // row-wise encryption of M2 (column-wise input); later the relinearised D0
    off = align_up(off + sizeof(uint64_t) * batch_words(r, N, L));
    c.ut = off;  // [L][2N][n]: [A; B] of ct1 per prime
    off = align_up(off + sizeof(uint64_t) * L * 2 * N * n);
    c.x = off;   // batch of 2N: a-parts [C00; C10]; b-parts zero (never written or read)
    off = align_up(off + sizeof(uint64_t) * batch_words(r, 2 * N, L));
    c.y = off;   // [L][2N][N]: [C01; C11]
    off = align_up(off + sizeof(uint64_t) * L * 2 * N * N);
    c.z = off;   // Transpose of x
    off = align_up(off + sizeof(uint64_t) * batch_words(r, 2 * N, L));
    c.total = off;
    return c;
}

// Ciphertext, key and output pointers: present and 16-byte aligned.
bool a16(const void *p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool ws_ok(const void *ws, size_t have, size_t need) {
    if (need == 0) return true;
    return ws != nullptr && (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) == 0 && have >= need;
}

// Debug-mode range checks of ring inputs (off unless debug_checks_on()): a
// batch [2][Lc][n][N] of coefficients below the chain primes, and switching
// keys [count][D][2][L+K][N] below q_0 .. q_{L-1} and the special primes.  A violation sets
// MODPP_ERR_RANGE in the ring's status word (sticky until read).
int check_batch(const modpp_ring_s *r, const uint64_t *ct, int64_t n, int Lc, cudaStream_t st) {
    if (!debug_checks_on() || n == 0) return MODPP_OK;
    const int64_t plane = n * r->N;
    return cuda_status(range_planes(ct, 2 * Lc, 1, plane, plane, plane, r->primes.data(), Lc,
                                    r->status, st));
}
int check_keys(const modpp_ring_s *r, const uint64_t *keys, int64_t count, cudaStream_t st) {
    if (!debug_checks_on() || count == 0) return MODPP_OK;
    return cuda_status(range_planes(keys, count * r->Dg * 2 * ks_planes(r), 1, r->N, r->N, r->N,
                                    r->primes.data(), ks_planes(r), r->status, st));
}


}  // namespace

extern "C" {

// Gadget limits: 1 <= D <= L digits of at most two primes (every digit
// non-empty), one or two special primes.
bool gadget_args_ok(int L, int K, int D) {
    if (L < 1 || L > kMaxChain || K < 1 || K > 2 || D < 1 || D > L || D > kMaxGadgetDigits) return false;
    const int alpha = (L + D - 1) / D;
    return alpha <= 2 && (D - 1) * alpha < L;
}

size_t modpp_ring_bytes_ks(int64_t N, int L, int K, int dnum) {
    if (N < 2 || N > kMaxN || log2_exact(N) < 0 || !gadget_args_ok(L, K, dnum)) return 0;
    return ring_layout(N, L, K).total;
}

size_t modpp_ring_bytes(int64_t N, int L) { return modpp_ring_bytes_ks(N, L, 1, L); }

int modpp_ring_create_ks(int64_t N, int L, int K, int dnum, const uint64_t *primes_host, void *mem,
                         size_t mem_bytes, void *stream, modpp_ring *ring) {
    if (ring == nullptr || primes_host == nullptr) return MODPP_ERR_ARG;
    *ring = nullptr;
    if (N < 2 || N > kMaxN || log2_exact(N) < 0 || !gadget_args_ok(L, K, dnum))
        return MODPP_ERR_ARG;
    const int Lp = L + K;
    for (int i = 0; i < Lp; ++i) {
        const uint64_t q = primes_host[i];
        if (q < 3 || (q & 1) == 0 || q >= (uint64_t(1) << 62) || (q - 1) % (2 * N) != 0 ||
            !is_prime_u64(q))
            return MODPP_ERR_PRIME;
        for (int j = 0; j < i; ++j)
            if (primes_host[j] == q) return MODPP_ERR_PRIME;
    }
    const RingLayout lay = ring_layout(N, L, K);
    if (!ws_ok(mem, mem_bytes, lay.total)) return MODPP_ERR_WORKSPACE;
    auto *r = new (std::nothrow) modpp_ring_s;
    if (!r) return MODPP_ERR_ARG;
    r->N = N;
    r->L = L;
    r->K = K;
    r->Dg = dnum;
    r->logN = log2_exact(N);
    r->primes.assign(primes_host, primes_host + Lp);
    r->mem = static_cast<char *>(mem);

    std::vector<char> host(lay.total, 0);
    auto *tabs = reinterpret_cast<uint64_t *>(host.data() + lay.tables);
    const uint64_t *dtabs = reinterpret_cast<const uint64_t *>(r->mem + lay.tables);
    auto *tab = reinterpret_cast<NttPlane *>(host.data() + lay.tab);
    for (int k = 0; k < Lp; ++k) {
        const uint64_t q = primes_host[k];
        const uint64_t psi = find_psi(q, N);
        if (psi == 0) {
            delete r;
            return MODPP_ERR_PRIME;
        }
        const uint64_t psi_inv = invmod(psi, q);
        uint64_t *fwd = tabs + (static_cast<int64_t>(8 * k) + 0) * N;
        uint64_t *fwd_s = tabs + (static_cast<int64_t>(8 * k) + 1) * N;
        uint64_t *inv = tabs + (static_cast<int64_t>(8 * k) + 2) * N;
        uint64_t *inv_s = tabs + (static_cast<int64_t>(8 * k) + 3) * N;
        uint64_t *fwd2 = tabs + (static_cast<int64_t>(8 * k) + 4) * N;  // 2N words
        uint64_t *inv2 = tabs + (static_cast<int64_t>(8 * k) + 6) * N;  // 2N words
        uint64_t pw = 1, pwi = 1;
        for (int64_t i = 0; i < N; ++i) {  // psi^i, placed at bitrev(i)
            const unsigned j = bitrev(static_cast<unsigned>(i), r->logN);
            fwd[j] = pw;
            fwd_s[j] = shoup(pw, q);
            inv[j] = pwi;
            inv_s[j] = shoup(pwi, q);
            fwd2[2 * j] = fwd[j];
            fwd2[2 * j + 1] = fwd_s[j];
            inv2[2 * j] = inv[j];
            inv2[2 * j + 1] = inv_s[j];
            pw = mulmod(pw, psi, q);
            pwi = mulmod(pwi, psi_inv, q);
        }
        NttPlane &t = tab[k];
        t.q = q;
        t.mu = static_cast<uint64_t>((static_cast<u128>(1) << 64) / q);
        uint64_t y = q;  // -q^-1 mod 2^64 by Newton's iteration
        for (int it = 0; it < 6; ++it) y *= 2 - q * y;
        t.qinv_neg = ~y + 1;
        t.ninv = invmod(static_cast<uint64_t>(N) % q, q);
        t.ninv_s = shoup(t.ninv, q);
        t.r64 = static_cast<uint64_t>((static_cast<u128>(1) << 64) % q);
        t.r64_s = shoup(t.r64, q);
        t.fwd = dtabs + (static_cast<int64_t>(8 * k) + 0) * N;
        t.fwd_s = dtabs + (static_cast<int64_t>(8 * k) + 1) * N;
        t.inv = dtabs + (static_cast<int64_t>(8 * k) + 2) * N;
        t.inv_s = dtabs + (static_cast<int64_t>(8 * k) + 3) * N;
        t.fwd2 = reinterpret_cast<const ulonglong2 *>(dtabs + (static_cast<int64_t>(8 * k) + 4) * N);
        t.inv2 = reinterpret_cast<const ulonglong2 *>(dtabs + (static_cast<int64_t>(8 * k) + 6) * N);
    }
    auto *consts = reinterpret_cast<uint64_t *>(host.data() + lay.consts);
    const uint64_t ql = primes_host[L - 1];
    // P mod q: the product of the special primes
    auto p_mod = [&](uint64_t q) {
        uint64_t v = 1 % q;
        for (int t = 0; t < K; ++t) v = mulmod(v, primes_host[L + t] % q, q);
        return v;
    };
    for (int k = 0; k < Lp; ++k) {
        const uint64_t q = primes_host[k];
        consts[0 * Lp + k] = k < L ? invmod(p_mod(q), q) : 0;
        consts[1 * Lp + k] = shoup(consts[0 * Lp + k], q);
        consts[2 * Lp + k] = k < L - 1 ? invmod(ql % q, q) : 0;
        consts[3 * Lp + k] = k < L - 1 ? shoup(consts[2 * Lp + k], q) : 0;
        consts[4 * Lp + k] = tab[k].ninv;
        consts[5 * Lp + k] = tab[k].ninv_s;
    }
    const uint64_t *dconsts = reinterpret_cast<const uint64_t *>(r->mem + lay.consts);
    r->tab = reinterpret_cast<const NttPlane *>(r->mem + lay.tab);
    r->pinv = dconsts;
    r->pinv_s = dconsts + Lp;
    r->qlinv = dconsts + 2 * Lp;
    r->qlinv_s = dconsts + 3 * Lp;
    r->ninv = dconsts + 4 * Lp;
    r->ninv_s = dconsts + 5 * Lp;
    // The key-switching gadget: digit constants (Garner's lift of two-prime
    // digits) and ModDown's constants for two special primes.
    KsGadget &g = r->g;
    g.L = L;
    g.K = K;
    g.D = dnum;
    g.alpha = (L + dnum - 1) / dnum;
    g.chain_max = *std::max_element(primes_host, primes_host + L);
    auto *gad = reinterpret_cast<uint64_t *>(host.data() + lay.gadget);
    const uint64_t *dgad = reinterpret_cast<const uint64_t *>(r->mem + lay.gadget);
    uint64_t *cq = gad, *cq_s = gad + kMaxGadgetDigits * Lp, *p0k = gad + 2 * kMaxGadgetDigits * Lp;
    uint64_t *p0k_s = p0k + L, *Pk = p0k + 2 * L;
    for (int d = 0; d < dnum; ++d) {
        const int j0 = d * g.alpha;
        if (std::min(L, j0 + g.alpha) - j0 < 2) continue;
        const uint64_t q0 = primes_host[j0], q1 = primes_host[j0 + 1];
        g.ginv[d] = invmod(q0 % q1, q1);
        g.ginv_s[d] = shoup(g.ginv[d], q1);
        for (int k = 0; k < Lp; ++k) {
            const uint64_t q = primes_host[k];
            cq[d * Lp + k] = q0 % q;
            cq_s[d * Lp + k] = shoup(q0 % q, q);
        }
    }
    g.cq = dgad;
    g.cq_s = dgad + kMaxGadgetDigits * Lp;
    if (K == 2) {
        const uint64_t p0 = primes_host[L], p1 = primes_host[L + 1];
        g.p0inv = invmod(p0 % p1, p1);
        g.p0inv_s = shoup(g.p0inv, p1);
        g.m1 = (p1 - 1) / 2;
        g.h0 = (p0 + 1) / 2;
        for (int k = 0; k < L; ++k) {
            const uint64_t q = primes_host[k];
            p0k[k] = p0 % q;
            p0k_s[k] = shoup(p0 % q, q);
            Pk[k] = p_mod(q);
        }
    }
    g.p0k = dgad + 2 * kMaxGadgetDigits * Lp;
    g.p0k_s = g.p0k + L;
    g.Pk = g.p0k + 2 * L;
    // Index tables of Alg. 4 (ints, period N).
    auto *ints = reinterpret_cast<int *>(host.data() + lay.ints);
    const int *dints = reinterpret_cast<const int *>(r->mem + lay.ints);
    int *t2_src = ints, *t2_ellinv = ints + N, *t2_kid = ints + 2 * N;
    const uint64_t twoN = 2 * static_cast<uint64_t>(N);
    for (int64_t c = 0; c < N; ++c) {
        // position c of the bit-reversed second Tweak input holds aux'_j, j = bitrev(c)
        const int64_t j = bitrev(static_cast<unsigned>(c), r->logN);
        const uint64_t ell = 2 * static_cast<uint64_t>(j) + 1;
        // ell^-1 modulo 2^64 by Newton's iteration (each step doubles the
        // correct low bits; ell is odd, so ell is its own inverse mod 8),
        // then modulo 2N.
        uint64_t inv = ell;
        for (int it = 0; it < 5; ++it) inv *= 2 - ell * inv;
        inv &= twoN - 1;
        t2_src[c] = static_cast<int>((inv - 1) / 2);
        t2_ellinv[c] = static_cast<int>(inv);
        t2_kid[c] = j == 0 ? -1 : static_cast<int>(j);
    }
    ints[3 * N] = 0;
    r->t2_src = dints;
    r->t2_ellinv = dints + N;
    r->t2_kid = dints + 2 * N;
    r->kid_zero = dints + 3 * N;
    r->status = reinterpret_cast<int *>(r->mem + lay.status);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(mem, host.data(), lay.total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreate(&r->ev[i]);
    if (e != cudaSuccess) {
        for (auto &ev : r->ev)
            if (ev) cudaEventDestroy(ev);
        delete r;
        return MODPP_ERR_CUDA;
    }
    *ring = r;
    return MODPP_OK;
}

int modpp_ring_create(int64_t N, int L, const uint64_t *primes_host, void *mem, size_t mem_bytes,
                      void *stream, modpp_ring *ring) {
    return modpp_ring_create_ks(N, L, 1, L, primes_host, mem, mem_bytes, stream, ring);
}

int modpp_ring_destroy(modpp_ring ring) {
    if (ring == nullptr) return MODPP_ERR_ARG;
    for (auto &ev : ring->ev)
        if (ev) cudaEventDestroy(ev);
    delete ring;
    return MODPP_OK;
}

int modpp_ring_prepare_keys(modpp_ring r, uint64_t *keys, int64_t count, void *stream) {
    if (r == nullptr || count < 0 || (count > 0 && !a16(keys))) return MODPP_ERR_ARG;
    const int Lp = ks_planes(r);
    const int64_t polys = count * r->Dg * 2 * Lp;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc = check_keys(r, keys, count, st);
    if (rc) return rc;
    cudaError_t e = launch_ntt(keys, polys, static_cast<int>(r->N), 1, Lp, r->tab, false, st);
    if (e == cudaSuccess) e = launch_to_montgomery(keys, polys, static_cast<int>(r->N), 1, Lp, r->tab, st);
    return cuda_status(e);
}

size_t modpp_keyswitch_workspace(modpp_ring r, int64_t n) {
    if (r == nullptr || n < 0) return 0;
    return std::max<size_t>(kAlign, ks_scratch_bytes(r, n));
}

int modpp_keyswitch(modpp_ring r, const uint64_t *ct, uint64_t *out, int64_t n, const uint64_t *key,
                    void *ws, size_t ws_bytes, void *stream) {
    if (r == nullptr || n < 0) return MODPP_ERR_ARG;
    if (n > 0 && (!a16(ct) || !a16(out) || !a16(key))) return MODPP_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, ks_scratch_bytes(r, n))) return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_batch(r, ct, n, r->L, st);
    if (rc == MODPP_OK && n > 0) rc = check_keys(r, key, 1, st);
    if (rc) return rc;
    return ks_run(r, ct, n, n, out, n, key, r->kid_zero, 1, 0, static_cast<char *>(ws), st);
}

int modpp_keyswitch_indexed(modpp_ring r, const uint64_t *ct, uint64_t *out, int64_t n,
                            const uint64_t *keys, const int *key_index, void *ws, size_t ws_bytes,
                            void *stream) {
    if (r == nullptr || n < 0 || n > (int64_t(1) << 30)) return MODPP_ERR_ARG;
    if (n == 0) return MODPP_OK;
    if (!a16(ct) || !a16(out) || !a16(keys) || key_index == nullptr) return MODPP_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, ks_scratch_bytes(r, n))) return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc = check_batch(r, ct, n, r->L, st);
    if (rc) return rc;
    return ks_run(r, ct, n, n, out, n, keys, key_index, static_cast<int>(n), 0,
                  static_cast<char *>(ws), st);
}

size_t modpp_tweak_workspace(modpp_ring r, int64_t n) {
    if (r == nullptr || n < 0) return 0;
    return std::max<size_t>(kAlign, align_up(sizeof(uint64_t) * batch_words(r, n, r->L)));
}

int modpp_tweak(modpp_ring r, const uint64_t *ct, uint64_t *out, int64_t n, void *ws,
                size_t ws_bytes, void *stream) {
    if (r == nullptr || n < 0) return MODPP_ERR_ARG;
    if (n == 0) return MODPP_OK;
    const int ln = log2_exact(n);
    if (ln < 0 || n > 2 * r->N || !a16(ct) || !a16(out)) return MODPP_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, align_up(sizeof(uint64_t) * batch_words(r, n, r->L))))
        return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int crc = check_batch(r, ct, n, r->L, st);
    if (crc) return crc;
    uint64_t *w = static_cast<uint64_t *>(ws);
    if (n == 1)  // no stage: the Tweak of one ciphertext is itself
        return cudaMemcpyAsync(out, ct, sizeof(uint64_t) * batch_words(r, 1, r->L),
                               cudaMemcpyDeviceToDevice, st) == cudaSuccess
                   ? MODPP_OK
                   : MODPP_ERR_CUDA;
    // The first pass reads the inputs in bit-reversed order; the passes
    // alternate between the workspace and out so that the last lands in out.
    int rc = MODPP_OK;
    TweakIO io;
    io.src = ct;
    io.in.in_bits = ln;
    io.land = out;
    tweak_stages(r, w, out, n, n, r->L, st, &rc, 2, io);
    return rc;
}

size_t modpp_transpose_workspace(modpp_ring r, int64_t groups) {
    if (r == nullptr || groups < 0) return 0;
    return std::max<size_t>(kAlign, transpose_scratch(r, groups));
}

int modpp_transpose(modpp_ring r, const uint64_t *ct, uint64_t *out, int64_t groups,
                    const uint64_t *aut_keys, void *ws, size_t ws_bytes, void *stream) {
    if (r == nullptr || groups < 0) return MODPP_ERR_ARG;
    if (groups == 0) return MODPP_OK;
    if (!a16(ct) || !a16(out) || !a16(aut_keys)) return MODPP_ERR_ARG;
    if (!ws_ok(ws, ws_bytes, transpose_scratch(r, groups))) return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_batch(r, ct, groups * r->N, r->L, st);
    if (rc == MODPP_OK) rc = check_keys(r, aut_keys, r->N, st);
    if (rc) return rc;
    return transpose_run(r, ct, out, groups, aut_keys, static_cast<char *>(ws), st);
}

int modpp_rescale(modpp_ring r, const uint64_t *ct, uint64_t *out, int64_t n, void *stream) {
    if (r == nullptr || n < 0 || r->L < 2) return MODPP_ERR_ARG;
    if (n == 0) return MODPP_OK;
    if (!a16(ct) || !a16(out)) return MODPP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc = check_batch(r, ct, n, r->L, st);
    if (rc) return rc;
    return cuda_status(launch_rescale(ct, out, r->L, n * r->N, r->tab, r->qlinv, r->qlinv_s, st));
}

size_t cc_mm_ex_workspace(modpp_ring r, int64_t n, int flags) {
    if (r == nullptr || r->L < 2 || (flags & ~MODPP_CC_M2_ROWWISE) != 0) return 0;
    if ((flags & MODPP_CC_M2_ROWWISE) ? (n < 1 || n > r->N) : n != r->N) return 0;
    return cc_layout(r, n).total;
}

size_t cc_mm_workspace(modpp_ring r) {
    if (r == nullptr) return 0;
    return cc_mm_ex_workspace(r, r->N, 0);
}

int cc_mm_ex(modpp_ring r, int64_t n, const uint64_t *ct1, const uint64_t *ct2,
             const uint64_t *aut_keys, const uint64_t *relin_key, int flags, uint64_t *out,
             double *out_scale_mult, void *ws, size_t ws_bytes, void *stream) {
    if (r == nullptr || r->L < 2 || (flags & ~MODPP_CC_M2_ROWWISE) != 0) return MODPP_ERR_ARG;
    const bool rowwise = (flags & MODPP_CC_M2_ROWWISE) != 0;
    if (rowwise ? (n < 1 || n > r->N) : n != r->N) return MODPP_ERR_ARG;
    if (!a16(ct1) || !a16(ct2) || !a16(aut_keys) || !a16(relin_key) || !a16(out))
        return MODPP_ERR_ARG;
    const CcLayout lay = cc_layout(r, n);
    if (!ws_ok(ws, ws_bytes, lay.total)) return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    const int L = r->L;
    const int64_t N = r->N, NN = N * N, nN = n * N;
    uint64_t *rw = reinterpret_cast<uint64_t *>(base + lay.rw);
    uint64_t *ut = reinterpret_cast<uint64_t *>(base + lay.ut);
    uint64_t *x = reinterpret_cast<uint64_t *>(base + lay.x);
    uint64_t *y = reinterpret_cast<uint64_t *>(base + lay.y);
    uint64_t *z = reinterpret_cast<uint64_t *>(base + lay.z);
    char *scratch = base + lay.scratch;
    {
        int rc = check_batch(r, ct1, n, L, st);
        if (rc == MODPP_OK) rc = check_batch(r, ct2, n, L, st);
        if (rc == MODPP_OK) rc = check_keys(r, aut_keys, N, st);
        if (rc == MODPP_OK) rc = check_keys(r, relin_key, 1, st);
        if (rc) return rc;
    }
    const bool timed = profile_active();
    r->timed = timed;
    auto mark = [&](int i) {
        if (timed) cudaEventRecord(r->ev[i], st);
    };
    mark(0);
    // Step 1: row-wise encryption of M2, unless it is given row-wise (the
    // row-or-column remark after Thm th:ccmm: Step 1 is skipped).
    const uint64_t *m2 = ct2;
    if (!rowwise) {
        const int rc = transpose_run(r, ct2, rw, 1, aut_keys, scratch, st);
        if (rc) return rc;
        m2 = rw;
    }
    mark(1);
    // Step 2: [A; B] per prime (2N x n; row r of A: coefficient r of every
    // column ciphertext), then C[:, :N] = [A; B] * A~' and C[:, N:] = [A; B] * B~'.
    cudaError_t e = launch_transpose_u64(ct1, ut, static_cast<int>(n), static_cast<int>(N), N, n,
                                         nN, 2 * N * n, L, st);
    if (e == cudaSuccess)
        e = launch_transpose_u64(ct1 + L * nN, ut + N * n, static_cast<int>(n),
                                 static_cast<int>(N), N, n, nN, 2 * N * n, L, st);
    if (e != cudaSuccess) return MODPP_ERR_CUDA;
    const size_t wide_bytes = modpp_mm_wide_workspace(2 * N, n, N, r->primes.data(), L);
    void *wws = base + lay.wide;
    int rc = modpp_mm_wide_pair(2 * N, n, N, ut, n, 2 * N * n, m2, m2 + L * nN, N, nN, x, y, N,
                                2 * NN, r->primes.data(), L, wws, wide_bytes, st);
    if (rc) return rc;
    mark(2);
    // Steps 3-4: Transpose((C00, 0)) and Transpose((C10, 0)) as one batch.
    rc = transpose_run(r, x, z, 2, aut_keys, scratch, st, /*b_zero=*/true);
    if (rc) return rc;
    mark(3);
    // Step 5: Relin(D0, 0) into rw (free now), then the sums and Rescale.
    char *ks = scratch;
    rc = ks_run(r, z, 2 * N, N, rw, N, relin_key, r->kid_zero, 1, 1, ks, st);
    if (rc) return rc;
    CcFinishParams fp{};
    fp.R = rw;
    fp.Z = z;
    fp.Y = y;
    fp.out = out;
    fp.L = L;
    fp.N = static_cast<int>(N);
    fp.tab = r->tab;
    fp.qlinv = r->qlinv;
    fp.qlinv_s = r->qlinv_s;
    if (launch_cc_finish(fp, st) != cudaSuccess) return MODPP_ERR_CUDA;
    mark(4);
    if (out_scale_mult) *out_scale_mult = 1.0 / static_cast<double>(r->primes[L - 1]);
    return MODPP_OK;
}

int cc_mm(modpp_ring r, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *aut_keys,
          const uint64_t *relin_key, uint64_t *out, void *ws, size_t ws_bytes, void *stream) {
    if (r == nullptr) return MODPP_ERR_ARG;
    return cc_mm_ex(r, r->N, ct1, ct2, aut_keys, relin_key, 0, out, nullptr, ws, ws_bytes, stream);
}

// ---------------------------------------------------------------- Alg. 7
// CP-MM with precomputation on a shared-a encryption, then the key switches
// back to one secret.  Workspace: the Mod-PP-MM workspace (status word
// first), the shared digits D of a (D * (L+K) transforms), key-switch
// products for a chunk of output ciphertexts, and, with the Rescale flag,
// the unrescaled batch.
struct PrecompLayout {
    size_t mm = 0, dig = 0, v = 0, u = 0, x = 0, total = 0;
    int64_t chunk = 0;
};
PrecompLayout precomp_layout(const modpp_ring_s *r, int64_t d2, int64_t d3, int flags) {
    PrecompLayout p{};
    const int L = r->L, Lp = ks_planes(r);
    const int64_t N = r->N;
    size_t off = 0;
    p.mm = off;
    off = align_up(off + modpp_mm_workspace(d3, d2, N, r->primes.data(), L, MODPP_PATH_F16));
    p.dig = off;
    off = align_up(off + sizeof(uint64_t) * r->Dg * Lp * N);
    p.v = off;  // Garner digits of the shared a-part (two-prime digits)
    off = align_up(off + sizeof(uint64_t) * r->Dg * N);
    const int64_t per_ct = 2 * static_cast<int64_t>(Lp) * N;
    p.chunk = std::max<int64_t>(1, std::min<int64_t>(d3, static_cast<int64_t>(ks_chunk_budget() / 8) / per_ct));
    p.u = off;
    off = align_up(off + sizeof(uint64_t) * p.chunk * per_ct);
    p.x = off;
    if (flags & MODPP_PRECOMP_RESCALE) off = align_up(off + sizeof(uint64_t) * batch_words(r, d3, L));
    p.total = off;
    return p;
}

size_t pc_mm_precomp_workspace(modpp_ring r, int64_t d2, int64_t d3, int flags) {
    if (r == nullptr || d2 < 1 || d3 < 1 || d2 > (int64_t(1) << 20) || d3 >= (int64_t(1) << 31) ||
        (flags & ~MODPP_PRECOMP_RESCALE) != 0 || ((flags & MODPP_PRECOMP_RESCALE) && r->L < 2))
        return 0;
    return precomp_layout(r, d2, d3, flags).total;
}

int pc_mm_precomp(modpp_ring r, int64_t d2, int64_t d3, const int8_t *Ut, const uint64_t *a,
                  const uint64_t *B, const uint64_t *keys, int flags, uint64_t *out, void *ws,
                  size_t ws_bytes, void *stream) {
    if (r == nullptr || d2 < 1 || d3 < 1 || d2 > (int64_t(1) << 20) || d3 >= (int64_t(1) << 31) ||
        (flags & ~MODPP_PRECOMP_RESCALE) != 0)
        return MODPP_ERR_ARG;
    const bool resc = (flags & MODPP_PRECOMP_RESCALE) != 0;
    if (resc && r->L < 2) return MODPP_ERR_ARG;
    if (Ut == nullptr || !a16(a) || !a16(B) || !a16(keys) || !a16(out)) return MODPP_ERR_ARG;
    const PrecompLayout lay = precomp_layout(r, d2, d3, flags);
    if (!ws_ok(ws, ws_bytes, lay.total)) return MODPP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int L = r->L, Lp = ks_planes(r);
    const int N = static_cast<int>(r->N);
    char *base = static_cast<char *>(ws);
    int rc = MODPP_OK;
    if (debug_checks_on()) {  // a and B below their primes; the keys
        rc = cuda_status(range_planes(a, L, 1, N, N, N, r->primes.data(), L, r->status, st));
        if (rc == MODPP_OK)
            rc = cuda_status(range_planes(B, L, 1, d2 * N, d2 * N, d2 * N, r->primes.data(), L,
                                          r->status, st));
        if (rc == MODPP_OK) rc = check_keys(r, keys, d3, st);
        if (rc) return rc;
    }
    // Step 1 (Alg. 7): B' = B * U, i.e. row k of B'^T = sum_j U[j][k] b_j for
    // every chain prime: one Mod-PP-MM of U^T (d3 x d2, int8) times the b-parts
    // (d2 x N per prime), written as the b-parts of the output batch.
    uint64_t *X = resc ? reinterpret_cast<uint64_t *>(base + lay.x) : out;
    const int64_t plane = d3 * static_cast<int64_t>(N);
    const size_t mm_bytes = modpp_mm_workspace(d3, d2, N, r->primes.data(), L, MODPP_PATH_F16);
    rc = modpp_mm(d3, d2, N, Ut, MODPP_U_I8, d2, B, N, d2 * static_cast<int64_t>(N), X + L * plane,
                  N, plane, r->primes.data(), L, MODPP_PATH_F16, base + lay.mm, mm_bytes, st);
    if (rc) return rc;
    // Key switches of (a, b'_k) with key k, k < d3: the digits of the shared
    // a-part and their forward transforms once, then per chunk the key
    // products, the inverse transforms and ModDown (in place on X).
    uint64_t *D = reinterpret_cast<uint64_t *>(base + lay.dig);
    uint64_t *Ubuf = reinterpret_cast<uint64_t *>(base + lay.u);
    uint64_t *V = ks_two_prime(r) ? reinterpret_cast<uint64_t *>(base + lay.v) : nullptr;
    cudaError_t e = cudaSuccess;
    if (V) e = launch_ks_garner(a, 1, N, 0, 1, r->tab, r->g, V, st);
    if (e != cudaSuccess) return MODPP_ERR_CUDA;
    if (ntt_fast_supported(N)) {
        e = launch_ks_digits_ntt(a, 1, N, 0, 1, r->tab, r->g, V, D, st);
    } else {
        e = launch_ks_decompose(a, 1, N, 0, 1, r->tab, r->g, V, D, st);
        if (e == cudaSuccess) e = launch_ntt(D, r->Dg * Lp, N, 1, Lp, r->tab, false, st);
    }
    if (e != cudaSuccess) return MODPP_ERR_CUDA;
    for (int64_t c0 = 0; c0 < d3; c0 += lay.chunk) {
        const int64_t m = std::min(lay.chunk, d3 - c0);
        e = launch_ks_multacc(D, keys, nullptr, 1, r->g, N, c0, m, r->tab, Ubuf, st,
                              /*d_shared=*/1);
        if (e == cudaSuccess) e = launch_ntt(Ubuf, m * 2 * Lp, N, 1, Lp, r->tab, true, st);
        if (e == cudaSuccess)
            e = launch_ks_moddown(Ubuf, X, d3, N, c0, m, nullptr, 1, 0, r->tab, r->g, r->pinv,
                                  r->pinv_s, X, d3, st);
        if (e != cudaSuccess) return MODPP_ERR_CUDA;
    }
    if (resc)
        return cuda_status(launch_rescale(X, out, L, d3 * static_cast<int64_t>(N), r->tab,
                                          r->qlinv, r->qlinv_s, st));
    return MODPP_OK;
}

int modpp_ring_status_read(modpp_ring r, void *stream) {
    if (r == nullptr) return MODPP_ERR_ARG;
    return modpp_status_read(r->status, stream);
}

int cc_mm_stage_ms(modpp_ring r, double ms[4]) {
    if (r == nullptr || ms == nullptr) return MODPP_ERR_ARG;
    if (!r->timed) return MODPP_ERR_ARG;
    for (int i = 0; i < 4; ++i) {
        float v = 0.f;
        if (cudaEventSynchronize(r->ev[i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&v, r->ev[i], r->ev[i + 1]) != cudaSuccess)
            return MODPP_ERR_CUDA;
        ms[i] = v;
    }
    return MODPP_OK;
}

}  // extern "C"
