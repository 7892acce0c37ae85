/*
 * modpp.h -- C ABI of the GB300 (sm_103a) Mod-PP-MM library.
 *
 * The library computes the exact modular matrix products to which
 * "Fast Homomorphic Linear Algebra with BLAS" (Bae, Cheon, Hanrot, Park,
 * Stehle; arXiv 2503.16080) reduces encrypted linear algebra:
 *
 *   Mod-PP-MM   C_j = U * A_j  mod q_j   for every RNS prime q_j
 *
 * (Sec. 5, notation ModPPMM_{q; d1, d2, d3}).  PC-MM and PC-Mv are two such
 * products, one on the a-part and one on the b-part of the ciphertext matrix
 * (Alg. 6 / Thm th:pcmm, written for the row format of Eq. mat_row_format).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are row-major; leading dimensions are in elements.
 * - Residue matrices are uint64 and canonical: every entry of A_j lies in
 *   [0, q_j).  Outputs are canonical in [0, q_j).
 * - U holds small signed integers in [-128, 127] (the integer-quantised
 *   plaintext matrix), stored as int8 or as int32 (see modpp_u_kind).
 * - Primes: odd, 3 <= q_j < 2^62.  They need not be distinct.
 * - Every data pointer (U, A, B, C, outputs, workspace) is a DEVICE pointer
 *   owned by the caller.  `primes_host` is a host array.  `stream` is a
 *   cudaStream_t (NULL = legacy default stream).
 * - The library never allocates device memory on the call path: scratch
 *   space is the caller's workspace, sized by the matching *_workspace
 *   query.  The workspace must be 256-byte aligned and must not be used by
 *   two calls that may run concurrently.
 * - Calls are asynchronous: they validate arguments on the host, enqueue
 *   kernels on `stream` and return.  An argument error returns a negative
 *   modpp_status before anything is enqueued.  A failure detected on the
 *   device (a bounded wait that timed out) is recorded in the workspace's
 *   status word and read back with modpp_status_read().
 * - Output buffers must not overlap inputs.
 * - Value ranges (residues canonical, U in [-128, 127]) are preconditions the
 *   host cannot see.  They are checked only in debug mode
 *   (modpp_set_debug_checks); otherwise an input outside its range gives
 *   unspecified outputs.
 */
#ifndef MODPP_H
#define MODPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MODPP_OK = 0,
    MODPP_ERR_ARG = -1,         /* bad size, null pointer or leading dimension */
    MODPP_ERR_PRIME = -2,       /* a prime is even, < 3 or >= 2^62 */
    MODPP_ERR_WORKSPACE = -3,   /* workspace null, misaligned or too small */
    MODPP_ERR_UNSUPPORTED = -4, /* valid request this build does not serve */
    MODPP_ERR_CUDA = -5,        /* a CUDA runtime, driver or cuBLAS call failed */
    MODPP_ERR_RANGE = -6,       /* debug checks: an input value outside its range (status word) */
    MODPP_ERR_TIMEOUT = -7      /* a bounded device-side wait gave up (status word) */
} modpp_status;

/* Which arithmetic carries the products. */
typedef enum {
    /* Default. Exact small-integer digits on the sm_103a tensor cores
     * (tcgen05.mma kind::f16, FP32 accumulation in TMEM, K split so every
     * partial sum stays within the 2^24 exact-integer range of FP32), with
     * a fused modular epilogue.  Residues are split into balanced b-bit
     * digits (modpp_set_digit_bits). */
    MODPP_PATH_F16 = 0,
    /* Strategy 1 of Sec. 6.1 (Lemma le:strategy1), as the paper ran it:
     * base K = floor(sqrt(2^53/k)) signed digits, one binary64 GEMM (cuBLAS
     * DGEMM) per digit pair, exact integer recombination mod q_j. */
    MODPP_PATH_FP64 = 1,
    /* Strategy 1 with the asymmetric base K_A = floor(2^53 / (k * 128))
     * for the residue operand (U needs one digit because |U| <= 128). */
    MODPP_PATH_FP64_TIGHT = 2
} modpp_path;

typedef enum {
    MODPP_U_I8 = 0,  /* int8_t entries */
    MODPP_U_I32 = 1  /* int32_t entries, values in [-128, 127] */
} modpp_u_kind;

/*
 * Debug mode: value-range checks of the inputs on the device (the
 * preconditions on input values, which the host cannot see).
 * While on, every product entry point (modpp_mm, pc_mm, pc_mv, the wide
 * products, grouped runs) enqueues, after its own launches, a pass over its
 * residue inputs checking 0 <= A_j[t][c] < q_j (and U_j for the wide
 * products) and, for MODPP_U_I32, -128 <= U <= 127.  A violation writes
 * MODPP_ERR_RANGE into the call's status word (modpp_status_read), unless
 * the word already holds an error.  The ring entry points of modpp_ring.h
 * check their ciphertext and key inputs before their launches and report
 * in the ring's status word (modpp_ring_status_read).  The products still
 * run; their outputs are unspecified when a check fails.  The setting is
 * process-wide (host only); the environment variable MODPP_DEBUG_CHECKS=1
 * turns it on at load time.  on: 0 or 1, else MODPP_ERR_ARG.
 */
int modpp_set_debug_checks(int on);
int modpp_get_debug_checks(void);

/* Human-readable name of a modpp_status value (static string). */
const char *modpp_status_string(int status);

/* Version of this ABI: (major << 16) | minor. */
int modpp_abi_version(void);

/*
 * Digit width b of the F16 path (process-wide tuning setting, host only).
 * Residues are split into balanced b-bit digits, b in {8, 9, 10}; the inner
 * dimension is accumulated in exact FP32 chunks of 2^(18-b).  Narrower
 * digits mean more digit products but fewer drains of the accumulators.
 * 0 restores the default: 9-bit digits, and 8-bit digits for products of at
 * most 32 output columns per plane (such thin products, PC-Mv for one, are
 * bound by the drains).  modpp_get_digit_bits and modpp_plan_info report the
 * width of wider products.  Returns MODPP_OK or MODPP_ERR_ARG.  Changing it
 * while calls are in flight on other threads is not supported.
 */
int modpp_set_digit_bits(int bits);
int modpp_get_digit_bits(void);

/*
 * Tensor-core kernel form of the f16 path for single-problem products
 * (modpp_mm, pc_mm, pc_mv; process-wide tuning setting, host only):
 *   0  one CTA per 128-row tile (tcgen05.mma.cta_group::1, M = 128);
 *   1  CTA pairs: clusters of two CTAs compute 256-row tiles with
 *      tcgen05.mma.cta_group::2 (M = 256), each CTA staging its own 128 rows
 *      of U and half of the digit tile, for outputs of at least 256 rows and
 *      more than 64 columns (others keep the one-CTA form).
 * The results are identical.  The environment variable MODPP_GEMM_PAIR sets
 * the initial value.  Workspace queries made before a change do not apply
 * after it.  Returns MODPP_OK or MODPP_ERR_ARG.
 */
int modpp_set_gemm_pair(int on);
int modpp_get_gemm_pair(void);

/*
 * Planning query (host only, no GPU needed).  For a product with inner
 * dimension k modulo q on `path`, reports how the operands are split:
 *   digits      number of residue digits (F16: ceil(bits(q)/b) balanced
 *               b-bit digits; FP64: the Strategy 1 digit count k1)
 *   digit_bits  F16: b (see modpp_set_digit_bits); FP64: floor(log2(base))
 *   k_chunk     F16: inner-dimension chunk whose FP32 partial sums stay
 *               exact, 2^(18-b); FP64: k (one DGEMM covers the whole k)
 * Returns MODPP_OK or an error for invalid k or q.
 */
int modpp_plan_info(int64_t k, uint64_t q, int path, int *digits, int *digit_bits,
                    int64_t *k_chunk);

/*
 * Workspace bytes for modpp_mm with these sizes (0 for invalid arguments).
 */
size_t modpp_mm_workspace(int64_t d, int64_t k, int64_t n, const uint64_t *primes_host, int P,
                          int path);

/*
 * Mod-PP-MM over P primes (Sec. 5, ModPPMM; Thm th:pcmm):
 *   C_j[r][c] = ( sum_t U[r][t] * A_j[t][c] ) mod q_j,   0 <= j < P.
 *
 *   U       d x k, kind `ukind`, leading dimension ldu >= k.
 *   A       P matrices k x n; A_j starts at A + j*strideA, leading dim lda >= n.
 *   C       P matrices d x n; C_j starts at C + j*strideC, leading dim ldc >= n.
 *   primes_host  P primes (host memory).
 *   P       1 <= P <= 32.
 *   path    a modpp_path value.
 *   ws, ws_bytes  workspace of at least modpp_mm_workspace(...) bytes.
 * Sizes: 0 <= d, n < 2^31; 0 <= k <= 2^20.  k = 0 writes zeros.
 * Returns MODPP_OK once the work is enqueued, or a negative modpp_status.
 */
int modpp_mm(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
             const uint64_t *A, int64_t lda, int64_t strideA, uint64_t *C, int64_t ldc,
             int64_t strideC, const uint64_t *primes_host, int P, int path, void *ws,
             size_t ws_bytes, void *stream);

/*
 * Approximate Mod-PP-MM of ONE modulus from the high-order bits of the
 * residue operand: Strategy 2 of Sec. 6.1 ("truncation").  The paper uses
 * it for the b-part of PC-MM, where an error e on the product becomes an
 * error of about e / Delta on the decoded message.  q: one odd modulus,
 * 3 <= q < 2^62 (it need not be prime).  B (k x n, leading dimension ldb)
 * holds residues in [0, q); each entry is read as its centred representative
 * x in (-q/2, q/2].  C (d x n, ldc) receives canonical residues.
 *   MODPP_PATH_F16, drop_bits = s >= 0 (s <= bits(q)): x is rounded to the
 *     nearest multiple of 2^s (ties upward), x_s = 2^s floor((x + 2^(s-1))
 *     / 2^s), and C = U * x_s mod q exactly, on the f16 digits of x_s / 2^s
 *     (fewer digit products than the exact product when s drops whole
 *     digits).  U int8, or int32 with values in [-128, 127].
 *     |C - U * B|  <=  k * max|U| * 2^(s-1)   (centred, per entry).
 *     s = 0 is the exact product.
 *   MODPP_PATH_FP64, drop_bits = 0: as printed, x rounded to the nearest
 *     double (53 significant bits), one binary64 product with U (cuBLAS
 *     DGEMM; any int32 U is exact in binary64), and the exact residue of
 *     each (integer-valued) double product.  The paper's bound:
 *     |C - U * B| <~ 2^-50 * k * max|U| * max|x|.
 * Sizes and errors as modpp_mm; other paths or a drop_bits outside the
 * range return MODPP_ERR_ARG.  Workspace from modpp_mm_trunc_workspace.
 */
size_t modpp_mm_trunc_workspace(int64_t d, int64_t k, int64_t n, uint64_t q, int path,
                                int drop_bits);
int modpp_mm_trunc(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                   const uint64_t *B, int64_t ldb, uint64_t *C, int64_t ldc, uint64_t q, int path,
                   int drop_bits, void *ws, size_t ws_bytes, void *stream);

/*
 * Mod-PP-MM of two residue matrices (the products of two ciphertext
 * matrices in Alg. 8, step 2):
 *   C_j = U_j * A_j mod q_j,   0 <= j < P,
 * where U_j (d x k, plane j at U + j*strideU, leading dimension ldu) holds
 * residues in [0, q_j) like A_j.  U_j is split into balanced 8-bit digits, each
 * digit plane runs the tensor-core product with A_j's digits, and the results
 * are accumulated with weights 2^(8 i) mod q_j.  Other conventions as modpp_mm
 * (MODPP_PATH_F16 only); workspace from modpp_mm_wide_workspace.
 */
size_t modpp_mm_wide_workspace(int64_t d, int64_t k, int64_t n, const uint64_t *primes_host,
                               int P);
int modpp_mm_wide(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu, int64_t strideU,
                  const uint64_t *A, int64_t lda, int64_t strideA, uint64_t *C, int64_t ldc,
                  int64_t strideC, const uint64_t *primes_host, int P, void *ws, size_t ws_bytes,
                  void *stream);

/*
 * Two wide products with the same left operand (the two products of Alg. 8,
 * step 2): C1_j = U_j * A1_j and C2_j = U_j * A2_j mod q_j, with the layout
 * conventions of modpp_mm_wide (A1, A2 share lda / strideA; C1, C2 share ldc
 * / strideC) and its workspace.  In the CRT form U's residue planes are
 * formed once per prime for both products.
 */
int modpp_mm_wide_pair(int64_t d, int64_t k, int64_t n, const uint64_t *U, int64_t ldu,
                       int64_t strideU, const uint64_t *A1, const uint64_t *A2, int64_t lda,
                       int64_t strideA, uint64_t *C1, uint64_t *C2, int64_t ldc, int64_t strideC,
                       const uint64_t *primes_host, int P, void *ws, size_t ws_bytes,
                       void *stream);

/*
 * How modpp_mm_wide forms its products.  Digit form: U_j in 8-bit digits
 * times A_j in b-bit digits, LU x LA tensor-core products per prime.
 * Multi-modular (CRT) form, the exact lifting variant of Strategy 3 (Sec.
 * 6.1): both operands lifted to balanced integers and reduced modulo R small
 * primes p < 256 with k ((p-1)/2)^2 < 2^24 and prod p >= 2.8 k ((q-1)/2)^2,
 * one tensor-core product per small prime, then the Chinese remainder
 * theorem modulo q_j.  Both are exact.
 *   mode 0 (default): the CRT form when it needs at most 10/11 of the digit
 *                     form's products, else digits;
 *   mode 1: always digits;  mode 2: the CRT form whenever a prime set exists.
 * Process-wide; returns MODPP_ERR_ARG for other modes.  Workspace queries
 * made before a change do not apply after it.
 */
int modpp_set_wide_path(int mode);
int modpp_get_wide_path(void);
/* Small primes the wide product would use for inner dimension k and these
 * chain primes (0 = digit form), under the current mode.  Host only. */
int modpp_wide_plan_info(int64_t k, const uint64_t *primes_host, int P, int *crt_primes);

/*
 * Workspace bytes for pc_mm / pc_mv with these sizes (0 for invalid arguments).
 */
size_t pc_mm_workspace(int64_t d, int64_t kct, int64_t N, const uint64_t *primes_host, int P,
                       int path);

/*
 * PC-MM in the row format (Alg. 6 and Thm th:pcmm, transposed to the row
 * identity A * Toep(s)^t + B = Delta*M of Eq. mat_row_format): row t of
 * (A_j, B_j) is the RNS residue j of a ciphertext whose plaintext is row t
 * of the kct x N message matrix.  Computes the two Mod-PP-MMs
 *   Aout_j = U * A_j mod q_j,   Bout_j = U * B_j mod q_j,
 * so that Aout * Toep(s)^t + Bout = U * (Delta*M + E): row r of the output
 * encrypts row r of U*M under the same secret.  No rescale is applied.
 *
 *   U            d x kct int8, contiguous (ldu = kct).
 *   A, B         [P][kct][N] contiguous residues.
 *   Aout, Bout   [P][d][N] contiguous.
 *   1 <= P <= 16.
 */
int pc_mm(int64_t d, int64_t kct, int64_t N, const int8_t *U, const uint64_t *A,
          const uint64_t *B, uint64_t *Aout, uint64_t *Bout, const uint64_t *primes_host, int P,
          int path, void *ws, size_t ws_bytes, void *stream);

/*
 * PC-Mv: the same pair of Mod-PP-MMs on a thin batch of `nvec` columns
 * (Thm th:pcmm with a small d3; the CP-Mv remark of Sec. 5.1).  Arguments
 * as pc_mm with N replaced by nvec.  The kernel streams U once per
 * (prime, part) plane, which is the memory-bound regime.
 */
int pc_mv(int64_t d, int64_t kct, int64_t nvec, const int8_t *U, const uint64_t *A,
          const uint64_t *B, uint64_t *Aout, uint64_t *Bout, const uint64_t *primes_host, int P,
          int path, void *ws, size_t ws_bytes, void *stream);

/*
 * Prepared plaintext.  The f16 path first converts U into an f16 matrix of d
 * rows of kp = k rounded up to 8 halves (zero padded), which the tensor cores
 * read.  For a plaintext reused over many products (the setting of Sec. 5.2,
 * where U is known beforehand) that conversion can be done once:
 *   modpp_u16_bytes(d, k)     bytes of the prepared matrix (0 for bad sizes);
 *   modpp_u_to_f16(...)       writes it to U16 (device, 16-byte aligned),
 *                             from U (int8, or int32 in [-128, 127]; d x k,
 *                             leading dimension ldu);
 *   pc_mm_u16(...)            PC-MM / PC-Mv exactly as pc_mm / pc_mv on
 *                             MODPP_PATH_F16, with the prepared U16 (d x kct)
 *                             instead of U; workspace from pc_mm_workspace.
 * Results are identical to pc_mm / pc_mv with the same U.  Debug range checks
 * do not inspect a prepared U16.
 */
size_t modpp_u16_bytes(int64_t d, int64_t k);
int modpp_u_to_f16(int64_t d, int64_t k, const void *U, int ukind, int64_t ldu, void *U16,
                   void *stream);
int pc_mm_u16(int64_t d, int64_t kct, int64_t N, const void *U16, const uint64_t *A,
              const uint64_t *B, uint64_t *Aout, uint64_t *Bout, const uint64_t *primes_host, int P,
              void *ws, size_t ws_bytes, void *stream);

/*
 * Grouped Mod-PP-MM: many independent products of uneven sizes, each with its
 * own prime list, computed by a few launches for the whole group: one U
 * conversion, then one digit split and one persistent tensor-core GEMM per
 * class of problems with the same digit count.
 *
 *   C_i,j = U_i * A_i,j  mod q_i,j     for every problem i and prime j.
 *
 * One modpp_problem describes problem i with the layout of modpp_mm:
 *   U      d x k int8 (values in [-128, 127]), leading dimension ldu >= k;
 *   A      P planes k x n, plane j at A + j*strideA, leading dimension lda >= n;
 *   C      P planes d x n, plane j at C + j*strideC, leading dimension ldc >= n;
 *   primes host array of P primes (odd, 3 <= q < 2^62); 1 <= P <= 32.
 * Sizes as modpp_mm (0 <= d, n < 2^31; 0 <= k <= 2^20; k = 0 gives zeros).
 *
 * A plan binds the problems (device pointers) and the caller's workspace.
 * - modpp_group_workspace(): bytes the plan needs (0 on invalid problems).
 * - modpp_group_plan_create(): validates, lays out the workspace, writes the
 *   device tables (synchronises `stream` once), and, if `tune` is non-zero,
 *   chooses the digit width (8, 9 or 10 bits) by timing each candidate on the
 *   problems themselves.  Tuning runs the products, so the outputs are
 *   written.  The choice is cached per process, keyed by the sizes, prime
 *   widths and GPU name, and appended to the file named by the environment
 *   variable MODPP_TUNE_CACHE when it is set.  Without tuning the process-wide
 *   width (modpp_set_digit_bits) is used.
 * - modpp_group_run(): enqueues the launches on `stream`.
 * - modpp_group_run_graph(): the first call runs the group once and captures
 *   the launches in a CUDA graph; every call launches that graph on `stream`.
 * - modpp_group_plan_info(): chosen digit width, number of GEMM tiles, tuning
 *   source (0 none, 1 timed, 2 cached) and the timed milliseconds of widths
 *   8, 9, 10 (tuned_ms[3]; 0 where not timed).
 * - modpp_group_plan_destroy(): frees the plan's host state and graph.
 * The workspace's status word (modpp_status_read) reports device timeouts of
 * the last run.  A plan must not be run concurrently with itself.
 * (Grouped launch over a device problem table: this build's own scheduling
 * layer; the products are Mod-PP-MMs as defined in Sec. 5.)
 */
typedef struct {
    int64_t d, k, n;
    const int8_t *U;
    int64_t ldu;
    const uint64_t *A;
    int64_t lda, strideA;
    uint64_t *C;
    int64_t ldc, strideC;
    const uint64_t *primes;
    int P;
} modpp_problem;

typedef struct modpp_group_plan modpp_group_plan;

size_t modpp_group_workspace(const modpp_problem *probs, int count);
int modpp_group_plan_create(const modpp_problem *probs, int count, void *ws, size_t ws_bytes,
                            int tune, void *stream, modpp_group_plan **plan);
int modpp_group_run(modpp_group_plan *plan, void *stream);
int modpp_group_run_graph(modpp_group_plan *plan, void *stream);
int modpp_group_plan_info(const modpp_group_plan *plan, int *digit_bits, int *tiles, int *tuned,
                          double *tuned_ms);
void modpp_group_plan_destroy(modpp_group_plan *plan);

/*
 * Kernel timing for measurement (no counterpart in the paper: instrumentation).
 * While enabled, every launch of the kernels named by modpp_kernel_id is
 * bracketed by a pair of CUDA events recorded on the launch's stream.
 * modpp_profile_read() waits for the recorded events of one kernel, returns
 * the sum of their elapsed times in milliseconds and the number of launches,
 * and forgets them.  Enabling or disabling also forgets all records.
 * Events are host-side driver objects; no device memory is allocated.
 */
typedef enum {
    MODPP_KERNEL_GEMM = 0,   /* tensor-core digit GEMM + modular epilogue */
    MODPP_KERNEL_SPLIT = 1,  /* residue -> f16 digit planes */
    MODPP_KERNEL_U16 = 2     /* U -> f16 */
} modpp_kernel_id;

int modpp_profile_enable(int on);
int modpp_profile_read(int kernel, double *total_ms, int64_t *launches);

/*
 * Mod-PP-MM without any device allocation by the caller or the library.
 * (No counterpart in the paper: this is an interface for callers that cannot
 * allocate device memory, for example applications whose memory manager owns
 * the whole GPU, plugin hosts that forbid device allocation on the call path,
 * or code that cannot accept an allocation's synchronisation and latency.)
 *
 * Same computation, arguments and layouts as modpp_mm on MODPP_PATH_F16, but
 * the scratch space is a fixed array of MODPP_STATIC_SCRATCH_BYTES (64 MiB)
 * compiled into the library.  Every GPU that loads the library holds that
 * array until the process exits.  The caller still passes the inputs and the
 * outputs (device pointers).
 *
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, and caches it.  Make
 *   that first call before any stream capture on the device.  A
 *   cudaDeviceReset unloads the library's device code; calls after one are
 *   not supported.
 * - Argument errors return the codes of modpp_mm (MODPP_ERR_ARG,
 *   MODPP_ERR_PRIME) before any CUDA call.  A request whose scratch need,
 *   modpp_mm_workspace(d, k, n, primes, P, MODPP_PATH_F16), exceeds
 *   MODPP_STATIC_SCRATCH_BYTES is then rejected with MODPP_ERR_WORKSPACE
 *   before anything is enqueued.
 * - It calls no cudaMalloc, cudaFree or other allocating routine.
 * - All calls on a device share the one array, which keeps the last call's
 *   contents.  Each call clears what must start at zero (the status word)
 *   and overwrites the rest before reading it.  Calls whose execution can
 *   overlap on the GPU (different streams without ordering, or several host
 *   threads) race on the array and give unspecified results: serialise them.
 * - Device-side status: the status word lives in the static array.
 *   modpp_mm_static_status(stream) waits for `stream`, reads and clears it
 *   on the current device: MODPP_OK, or MODPP_ERR_TIMEOUT when a bounded
 *   device wait of the last call gave up (its outputs are then unspecified).
 */
#define MODPP_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

size_t modpp_mm_static_capacity(void);
int modpp_mm_static(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                    const uint64_t *A, int64_t lda, int64_t strideA, uint64_t *C, int64_t ldc,
                    int64_t strideC, const uint64_t *primes_host, int P, void *stream);
int modpp_mm_static_status(void *stream);

/*
 * Waits for `stream`, reads and clears the device status word kept in the
 * workspace `ws`.  Returns MODPP_OK, MODPP_ERR_TIMEOUT (a bounded device wait
 * gave up; the kernel returned early and its outputs are unspecified) or
 * MODPP_ERR_CUDA.
 */
int modpp_status_read(void *ws, void *stream);

/*
 * Self-test of the failure path of the bounded device waits (every spin on
 * an mbarrier in the library's kernels gives up after a time limit, records
 * MODPP_ERR_TIMEOUT in the status word and returns).  Enqueues one small
 * kernel whose wait nothing ever satisfies, limited to limit_ns (1 ns to
 * 10 s); the status word at the start of `ws` (device, 256-byte aligned, at
 * least 256 bytes) then reads MODPP_ERR_TIMEOUT through modpp_status_read,
 * and the context stays usable.  Returns MODPP_OK once enqueued,
 * MODPP_ERR_ARG for a bad workspace or limit, MODPP_ERR_CUDA.
 */
int modpp_selftest_bounded_wait(void *ws, uint64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MODPP_H */
