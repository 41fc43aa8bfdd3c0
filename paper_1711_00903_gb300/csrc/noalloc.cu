// fem_dot_noalloc: the deterministic FP64 dot product with its scratch in a
// file-scope device array instead of caller- or library-allocated memory.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// need a reduction -- a serving loop that must not allocate per request
// because an allocation can synchronise the device or fail under a fixed
// memory budget, and embedding applications whose device memory is owned by
// their own allocator.  They pass inputs and the output only.
//
// The scratch array is small (kNoallocParts doubles, 32 KiB) and every GPU
// that loads the library holds it until the process exits.  Each block of
// the first pass reduces one fixed chunk of kNoallocChunk entries, so the
// number of partial sums grows with n and n is capped at
// kNoallocParts * kNoallocChunk.
#include <mutex>

#include "fem_internal.h"
#include "kernels_common.cuh"

namespace fem {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocChunk = kNoallocThreads * 32;  // entries per partial sum
constexpr int kNoallocParts = 4096;                  // capacity of the scratch array

// The scratch: one partial sum per chunk.  Shared by every call in the
// process; each call overwrites the slots it reads, so nothing needs to be
// cleared between calls.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocParts];

__global__ void __launch_bounds__(kNoallocThreads)
noalloc_partial_kernel(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                       double *__restrict__ part) {
    __shared__ double sh[32];
    const int64_t base = (int64_t)blockIdx.x * kNoallocChunk;
    int64_t end = base + kNoallocChunk;
    if (end > n) end = n;
    double s = 0.0;
    for (int64_t i = base + threadIdx.x; i < end; i += kNoallocThreads) s = fma(x[i], y[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024)
noalloc_final_kernel(int nparts, const double *__restrict__ part, double *__restrict__ result) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *result = s;
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the symbol is only a host-side stand-in) and
// kept for the process: a cudaDeviceReset of the device after the first call
// would leave it stale, which the header states as unsupported.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace fem

extern "C" {

int64_t fem_dot_noalloc_max_n(void) { return (int64_t)fem::kNoallocParts * fem::kNoallocChunk; }

int fem_dot_noalloc(int64_t n, const double *x, const double *y, double *result, void *stream) {
    if (n < 0 || !result) return FEM_EINVAL;
    if (n > fem_dot_noalloc_max_n()) return FEM_ETOOBIG;
    if (n > 0 && (!x || !y)) return FEM_EINVAL;
    double *scratch = nullptr;
    cudaError_t e = fem::scratch_address(&scratch);
    if (e != cudaSuccess) return fem::record_cuda_error(e);
    const int parts = (int)((n + fem::kNoallocChunk - 1) / fem::kNoallocChunk);
    cudaStream_t s = (cudaStream_t)stream;
    if (parts > 0)
        fem::noalloc_partial_kernel<<<parts, fem::kNoallocThreads, 0, s>>>(n, x, y, scratch);
    fem::noalloc_final_kernel<<<1, 1024, 0, s>>>(parts, scratch, result);
    e = cudaGetLastError();
    return e == cudaSuccess ? FEM_OK : fem::record_cuda_error(e);
}

}  // extern "C"
