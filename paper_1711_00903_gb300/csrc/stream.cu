// Roofline calibration kernel: a stream with a chosen read:write ratio.
//
// Section 5 of the paper calibrates its bandwidth roofline with a plain
// device-to-device copy (one byte read per byte written).  The operators
// read several arrays for each one they write (BP3.5: eight planes of N_p
// values per plane written), so a second calibration point is a stream
// that reads k planes and writes their sum, dst[i] = sum_p src[p n + i],
// summed in plane order p = 0, 1, ..., k-1.
//
// GB300 design: 16-byte vector loads and stores (double2 / float4; the
// plane length is a multiple of the vector width, checked by the caller), a
// grid-stride loop over a grid of 152 SMs x 8 blocks, and the loads of an
// output vector issued in groups of eight before their adds, so that up to
// eight independent HBM requests are in flight per thread.
#include "fem_internal.h"
#include "kernels_common.cuh"

namespace fem {
namespace {

constexpr int kStreamThreads = 256;
constexpr int kStreamBlocks = 152 * 8;
constexpr int kMaxPlanes = 32;

template <typename V, typename T, int W>
__global__ void __launch_bounds__(kStreamThreads)
stream_sum_kernel(int planes, int64_t n, const T *__restrict__ src, T *__restrict__ dst) {
    constexpr int kChunk = 8;  // loads issued before their adds
    const int64_t nv = n / W;  // vectors per plane (n is a multiple of W)
    const V *s = reinterpret_cast<const V *>(src);
    V *d = reinterpret_cast<V *>(dst);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        V acc;
        for (int p0 = 0; p0 < planes; p0 += kChunk) {
            V v[kChunk];
#pragma unroll
            for (int c = 0; c < kChunk; c++)
                if (p0 + c < planes) v[c] = __ldcs(s + (int64_t)(p0 + c) * nv + i);
#pragma unroll
            for (int c = 0; c < kChunk; c++) {
                if (p0 + c >= planes) break;
                if (p0 + c == 0) {
                    acc = v[0];
                } else {
                    const T *pv = reinterpret_cast<const T *>(&v[c]);
                    T *pa = reinterpret_cast<T *>(&acc);
#pragma unroll
                    for (int w = 0; w < W; w++) pa[w] += pv[w];
                }
            }
        }
        __stcs(d + i, acc);
    }
}

}  // namespace

cudaError_t launch_stream_sum(int planes, int64_t n, const void *src, void *dst, int word, cudaStream_t s) {
    if (word == 8)
        stream_sum_kernel<double2, double, 2><<<kStreamBlocks, kStreamThreads, 0, s>>>(
            planes, n, (const double *)src, (double *)dst);
    else
        stream_sum_kernel<float4, float, 4><<<kStreamBlocks, kStreamThreads, 0, s>>>(
            planes, n, (const float *)src, (float *)dst);
    return cudaGetLastError();
}

int stream_max_planes() { return kMaxPlanes; }

// FP64 issue-rate probe: every thread runs eight independent FMA chains of
// `iters` steps (x <- x * b + c), so the FP64 pipe, not latency, sets the
// rate; one value per thread is stored so that nothing is optimised away.
// Flops = 2 * 8 * iters * threads.
namespace {
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, double b, double c, double *__restrict__ out) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int64_t k = 0; k < iters; k++) {
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = fma(x[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += x[i];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}
}  // namespace

// Self-test of the bounded mbarrier wait: one block waits on a barrier
// that expects two arrivals and gets one, so the phase never completes; every
// wait must give up after its iteration limit and count itself, the block
// must report the failure through a status word the way the stream kernels
// report it to the solver, and the kernel must return normally.
namespace {
__global__ void __launch_bounds__(64) wait_selftest_kernel(double *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&bar)) : "memory");
    }
    __syncthreads();
    const bool done = mbar_wait(&bar, 0);
    if (!done && (threadIdx.x & 31) == 0) atomicAdd(&g_wait_timeouts, 1ull);
    if (!__syncthreads_and(done) && threadIdx.x == 0) *status = 1.0;
}
__device__ double g_selftest_status;
}  // namespace

FEM_DEFINE_WAIT_COUNTER(wait_timeouts_selftest)

cudaError_t run_wait_selftest(unsigned long long *gave_up, bool *reported) {
    unsigned long long zero = 0;
    cudaError_t e = wait_timeouts_selftest(&zero, true);
    const double z = 0.0;
    double *st = nullptr;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_selftest_status, &z, sizeof z);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&st, g_selftest_status);
    if (e != cudaSuccess) return e;
    wait_selftest_kernel<<<1, 64>>>(st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = wait_timeouts_selftest(gave_up, true);
    double v = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_selftest_status, sizeof v);
    *reported = (v != 0.0);
    return e;
}

int64_t fma_probe_threads() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int64_t)(sms > 0 ? sms : 1) * 8 * 256;
}

cudaError_t launch_fma_probe(int64_t iters, double *out, cudaStream_t s) {
    const int64_t threads = fma_probe_threads();
    fma_probe_kernel<<<(unsigned)(threads / 256), 256, 0, s>>>(iters, 0.999999, 1e-6, out);
    return cudaGetLastError();
}

}  // namespace fem
