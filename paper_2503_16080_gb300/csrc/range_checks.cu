// Value-range checks of the inputs (debug mode).
//
// The entry points take residues that must be canonical (every entry of a
// plane modulo q lies in [0, q)) and plaintext entries in [-128, 127].  The
// host cannot check values it never reads, so these checks are a device
// pass over the inputs, enabled by modpp_set_debug_checks(1) or by the
// environment variable MODPP_DEBUG_CHECKS=1 at load time.  A violation
// writes MODPP_ERR_RANGE into the call's status word (compare-and-swap from
// MODPP_OK, so an earlier error such as a timeout is kept).  The product
// itself still runs: its outputs are then unspecified, as without the check.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>

#include "modpp.h"
#include "modpp_internal.h"

namespace modpp {
namespace {

std::atomic<int> g_debug_checks{[] {
    const char *v = std::getenv("MODPP_DEBUG_CHECKS");
    return (v != nullptr && v[0] != '\0' && v[0] != '0') ? 1 : 0;
}()};

__device__ __forceinline__ void flag_range(int *status, bool bad) {
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
        atomicCAS(status, MODPP_OK, MODPP_ERR_RANGE);
}

// Element (p, r, c) of a stack of planes lies at base + p * plane_stride +
// r * ld + c; it must be below q[p % nq].
__global__ void range_u64_kernel(RangeCheckU64 a) {
    const int64_t total = a.planes * a.rows * a.cols;
    bool bad = false;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t c = i % a.cols;
        const int64_t t = i / a.cols;
        const int64_t r = t % a.rows;
        const int64_t p = t / a.rows;
        const uint64_t v = a.base[p * a.plane_stride + r * a.ld + c];
        bad |= v >= a.q[p % a.nq];
    }
    flag_range(a.status, bad);
}

// int32 plaintext entries must lie in [-128, 127].
__global__ void range_i32_kernel(const int32_t *U, int64_t rows, int64_t cols, int64_t ld,
                                 int *status) {
    const int64_t total = rows * cols;
    bool bad = false;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = U[(i / cols) * ld + i % cols];
        bad |= v < -128 || v > 127;
    }
    flag_range(status, bad);
}

unsigned grid_for(int64_t total) {
    const int64_t b = (total + 255) / 256;
    return static_cast<unsigned>(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
}

}  // namespace

bool debug_checks_on() { return g_debug_checks.load(std::memory_order_relaxed) != 0; }

cudaError_t launch_range_u64(const RangeCheckU64 &a, cudaStream_t s) {
    if (a.planes <= 0 || a.rows <= 0 || a.cols <= 0) return cudaSuccess;
    range_u64_kernel<<<grid_for(a.planes * a.rows * a.cols), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_range_i32(const int32_t *U, int64_t rows, int64_t cols, int64_t ld, int *status,
                             cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    range_i32_kernel<<<grid_for(rows * cols), 256, 0, s>>>(U, rows, cols, ld, status);
    return cudaGetLastError();
}

cudaError_t range_planes(const uint64_t *base, int64_t planes, int64_t rows, int64_t cols,
                         int64_t ld, int64_t plane_stride, const uint64_t *q, int nq, int *status,
                         cudaStream_t s) {
    if (nq < 1 || nq > kMaxRangeQ) return cudaErrorInvalidValue;
    RangeCheckU64 a{};
    a.base = base;
    a.planes = planes;
    a.rows = rows;
    a.cols = cols;
    a.ld = ld;
    a.plane_stride = plane_stride;
    a.nq = nq;
    for (int i = 0; i < nq; ++i) a.q[i] = q[i];
    a.status = status;
    return launch_range_u64(a, s);
}

}  // namespace modpp

extern "C" {

int modpp_set_debug_checks(int on) {
    if (on != 0 && on != 1) return MODPP_ERR_ARG;
    modpp::g_debug_checks.store(on);
    return MODPP_OK;
}

int modpp_get_debug_checks(void) { return modpp::g_debug_checks.load(); }

}  // extern "C"
