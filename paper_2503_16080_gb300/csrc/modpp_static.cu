// modpp_mm_static: Mod-PP-MM for callers that cannot allocate device memory.
//
// Some callers have no way to provide the scratch workspace that modpp_mm
// needs.  Examples: an application whose memory manager reserves the whole
// GPU up front, so that a cudaMalloc from a library fails; a plugin host
// whose interface forbids device allocation on the call path; code with hard
// latency bounds, where an allocation's implicit synchronisation and
// unpredictable cost are not acceptable.  This entry point takes the same
// inputs and outputs as modpp_mm (f16 path) but uses a fixed scratch array
// that is part of the library image itself.
//
// The array below is allocated by the CUDA runtime when this library's device
// code is loaded on a GPU, and every GPU that loads the library keeps it until
// the process exits.  In host code its name is only a host-side stand-in,
// never a device address: the device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, and cached.  A
// cudaDeviceReset unloads the module, so the cached address is then stale:
// calls after a reset are not supported.
#include <cuda_runtime.h>

#include <mutex>

#include "modpp.h"
#include "modpp_internal.h"

namespace {

constexpr size_t kScratchBytes = MODPP_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once per
// device on first use).
int scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MODPP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (g_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr)
            return MODPP_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MODPP_OK;
}

}  // namespace

extern "C" {

size_t modpp_mm_static_capacity(void) { return kScratchBytes; }

int modpp_mm_static(int64_t d, int64_t k, int64_t n, const void *U, int ukind, int64_t ldu,
                    const uint64_t *A, int64_t lda, int64_t strideA, uint64_t *C, int64_t ldc,
                    int64_t strideC, const uint64_t *primes_host, int P, void *stream) {
    // The argument checks of modpp_mm come first, with its error codes; no
    // CUDA call is made for a rejected request.
    const int rc = modpp::mm_check_args(d, k, n, U, ukind, ldu, A, lda, strideA, C, ldc, strideC,
                                        primes_host, P);
    if (rc != MODPP_OK) return rc;
    if (modpp_mm_workspace(d, k, n, primes_host, P, MODPP_PATH_F16) > kScratchBytes)
        return MODPP_ERR_WORKSPACE;  // larger than the static scratch
    void *ws = nullptr;
    const int arc = scratch_address(&ws);
    if (arc != MODPP_OK) return arc;
    // modpp_mm clears the status word at the start of every call and rewrites
    // every other scratch byte it reads, so stale contents of the previous
    // call do not leak into this one.
    return modpp_mm(d, k, n, U, ukind, ldu, A, lda, strideA, C, ldc, strideC, primes_host, P,
                    MODPP_PATH_F16, ws, kScratchBytes, stream);
}

int modpp_mm_static_status(void *stream) {
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != MODPP_OK) return rc;
    return modpp_status_read(ws, stream);
}

}  // extern "C"
