// qt_noalloc.cu -- qt_norm_static: the norm reduction for callers that may not
// allocate device memory.
//
// qt_norm keeps its partial sums in a buffer the circuit allocates with
// cudaMalloc.  Some callers cannot let a library call cudaMalloc: a process
// that hands all device memory to its own allocator or pool and forbids other
// allocations, or a latency-critical loop where an allocation (and the
// device-wide synchronisation cudaMalloc/cudaFree may imply) is not
// acceptable.  qt_norm_static runs the same two kernels on amplitudes the
// caller already holds in device memory and keeps the partial sums in the
// file-scope array below instead of allocating.
//
// The array's name is a host-side stand-in in host code, not a device
// address: passing it to a kernel from the host would fault or read the
// wrong memory.  So every call asks cudaGetSymbolAddress, with the caller's
// device current, for the array's device address on that device, and gives
// the kernels that address.  The lookup allocates nothing; doing it on every
// call (rather than caching it) keeps the address right across a context
// reset (cudaDeviceReset) between calls.
#include <cuda_runtime.h>

#include <string>

#include "qt_internal.h"

namespace qt {

// One partial sum per reduction block; launch_norm never uses more blocks
// than norm_partials_needed() returns, which is at most kMaxNormPartials.
constexpr int kNormStaticPartials = kMaxNormPartials;
static_assert(kNormStaticPartials * sizeof(double) == QT_NORM_STATIC_SCRATCH_BYTES, "documented scratch size");
static __device__ __align__(256) double g_norm_scratch[kNormStaticPartials];

}  // namespace qt

using namespace qt;

extern "C" qt_status qt_norm_static(const void* amps_device, uint64_t count, int32_t dtype, double* out_device,
                                    void* cuda_stream) {
    if (!amps_device || !out_device) {
        set_thread_error("qt_norm_static: amps_device and out_device must be device pointers, not NULL");
        return QT_ERR_ARG;
    }
    if (dtype != QT_C128 && dtype != QT_C64 && dtype != QT_C128_DF) {
        set_thread_error("qt_norm_static: unknown dtype");
        return QT_ERR_ARG;
    }
    if (count == 0 || count > QT_NORM_STATIC_MAX_AMPS) {
        set_thread_error("qt_norm_static: count must be in [1, QT_NORM_STATIC_MAX_AMPS = 2^34]");
        return QT_ERR_RANGE;
    }
    const int np = norm_partials_needed(count);
    if (np > kNormStaticPartials) {
        set_thread_error("qt_norm_static: more partial sums than the static scratch holds");
        return QT_ERR_RANGE;
    }
    void* scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&scratch, g_norm_scratch);
    if (e != cudaSuccess) {
        set_thread_error(std::string("qt_norm_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return QT_ERR_CUDA;
    }
    // Every call writes all np partial sums before the final kernel reads
    // them, so nothing in the scratch needs clearing between calls.
    const int rc = launch_norm(dtype, amps_device, count, static_cast<double*>(scratch), np, out_device, cuda_stream);
    if (rc) {
        set_thread_error(std::string("qt_norm_static: launch failed: ") + cudaGetErrorString(cudaError_t(rc)));
        return QT_ERR_CUDA;
    }
    return QT_OK;
}
