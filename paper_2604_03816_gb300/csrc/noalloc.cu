// sv_expect_noalloc: the Pauli-expectation reduction with no memory allocation at all.
//
// Who needs it: code that must not call cudaMalloc or cudaFree -- a host framework that
// owns the whole device-memory budget through its own pool and forbids side
// allocations, or a latency-critical loop where an allocation would synchronise the
// device and stall the other streams.  Such a caller cannot create an sv_state
// (sv_alloc allocates a workspace), so this entry point works on a raw device state
// vector that the caller owns.
//
// The kernel's scratch memory (one FP64 partial sum per block per batch of terms) lives
// in a file-scope __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.  Host code must not pass the array's name to a kernel
// (in host code it is only a stand-in symbol); its device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made on that device.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sv_internal.h"

namespace {

constexpr int kNoallocBlocks = 256;                 // fixed grid: 256 partials per batch
constexpr size_t kNoallocScratchDoubles = 16384;    // 128 KiB: at most 64 term batches

__device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
sv_status scratch_for_current_device(double **out) {
    int dev = 0;
    SV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return svi::set_error(SV_ERR_ARG, "sv_expect_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return svi::set_error(SV_ERR_CUDA, std::string("sv_expect_noalloc: cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return SV_OK;
}

}  // namespace

extern "C" sv_status sv_expect_noalloc(const void *psi, uint32_t n, sv_dtype dtype,
                                       const uint64_t *xmask, const uint64_t *zmask,
                                       const double *coef, size_t nterms, double *out_dev,
                                       void *stream) {
    svi::clear_error();
    if (!psi || !out_dev || (nterms && (!xmask || !zmask || !coef)))
        return svi::set_error(SV_ERR_ARG, "sv_expect_noalloc: null argument");
    if (n < 1 || n > SV_MAX_QUBITS) return svi::set_error(SV_ERR_ARG, "sv_expect_noalloc: n must be 1..34");
    if (dtype != SV_C64 && dtype != SV_C128)
        return svi::set_error(SV_ERR_ARG, "sv_expect_noalloc: bad dtype");
    if (reinterpret_cast<uintptr_t>(psi) & 15u)
        return svi::set_error(SV_ERR_ARG, "sv_expect_noalloc: state must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(out_dev) & 7u)
        return svi::set_error(SV_ERR_ARG, "sv_expect_noalloc: out_dev must be 8-byte aligned");
    // Both pointers must be device (or managed) memory that the current device can use: a
    // host pointer or another device's memory would reach the kernel and fault.
    int dev = 0;
    SV_CUDA(cudaGetDevice(&dev));
    const void *ptrs[2] = {psi, out_dev};
    const char *names[2] = {"psi", "out_dev"};
    for (int i = 0; i < 2; ++i) {
        cudaPointerAttributes pa;
        const cudaError_t e = cudaPointerGetAttributes(&pa, ptrs[i]);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return svi::set_error(SV_ERR_ARG, std::string("sv_expect_noalloc: ") + names[i] +
                                                  " is not a CUDA pointer (" + cudaGetErrorString(e) + ")");
        }
        const bool on_dev = (pa.type == cudaMemoryTypeDevice && pa.device == dev) ||
                            pa.type == cudaMemoryTypeManaged;
        if (!on_dev)
            return svi::set_error(SV_ERR_ARG, std::string("sv_expect_noalloc: ") + names[i] +
                                                  " must be device memory of the current device");
    }
    const uint64_t lim = (1ull << n) - 1;
    for (size_t t = 0; t < nterms; ++t)
        if ((xmask[t] & ~lim) || (zmask[t] & ~lim))
            return svi::set_error(SV_ERR_ARG, "sv_expect_noalloc: Pauli mask names a qubit >= n");
    double *scratch = nullptr;
    sv_status st = scratch_for_current_device(&scratch);
    if (st != SV_OK) return st;
    return svi::enqueue_expect_sum(psi, n, dtype, xmask, zmask, coef, nterms, scratch,
                                   kNoallocScratchDoubles, kNoallocBlocks, out_dev,
                                   static_cast<cudaStream_t>(stream));
}
