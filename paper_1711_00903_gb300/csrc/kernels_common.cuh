// Device helpers shared by the operator kernels.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fem_internal.h"

namespace fem {

// Elements per block for a slab of q x q threads per element: about
// `target` threads per block, bounded by the shared-memory budget (bytes per
// element given).
__host__ __device__ constexpr int pick_epb(int q, int smem_per_elem, int target = 256) {
    int t = target / (q * q);
    if (t < 1) t = 1;
    while (t > 1 && t * smem_per_elem > 96 * 1024) t--;
    return t;
}

// Rounds a count of doubles up to a multiple of 2 (16-byte alignment).
__host__ __device__ constexpr int pad2(int x) { return (x + 1) & ~1; }

// Asynchronous global -> shared copies (LDGSTS): the data lands in shared
// memory without passing through registers; cp_async_wait_all() blocks the
// issuing thread until its own copies have landed (a barrier then publishes
// them to the block).  Both addresses must be aligned to the copy size.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// TMA bulk prefetch of [p, p + bytes) into L2, rounded inward to 16-byte
// boundaries (a hint: nothing is prefetched outside the range).
__device__ __forceinline__ void prefetch_l2(const void *p, long long bytes) {
    const unsigned long long a = (unsigned long long)p, e = a + (unsigned long long)bytes;
    const unsigned long long a16 = (a + 15) & ~15ull, e16 = e & ~15ull;
    if (e16 <= a16) return;
    unsigned long long off = a16;
    while (off < e16) {  // a bulk prefetch moves at most 2^31 bytes; blocks use far less
        unsigned long long sz = e16 - off;
        if (sz > (1ull << 30)) sz = 1ull << 30;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(off), "r"((unsigned)sz) : "memory");
        off += sz;
    }
}

// ---- mbarrier and TMA bulk copies (global -> shared), CTA scope.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Initialises a shared-memory mbarrier expecting `count` arrivals and makes
// the initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous transfer.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// TMA bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Copies the byte range [src, src + bytes) of an array that ends at
// arr_end into shared memory at dst (16-byte aligned, with room for
// bytes + 32), for ranges that need not be 16-byte aligned: one TMA bulk
// copy of the enclosing 16-byte-aligned range, clipped to the last 16-byte
// boundary inside the array, and plain loads for the few bytes past that
// boundary.  The range's first byte lands at dst + (src & 15); the caller
// (one thread) adds the returned TMA byte count to the mbarrier's expected
// transaction count before this call's copy can complete -- so the expect
// is issued first, by the caller, with the total of all its copies.
struct RangeCopy {
    unsigned tma_bytes;  // bytes moved by the bulk copy (0: none)
    unsigned offset;     // where the range starts in dst
};
__device__ __forceinline__ RangeCopy range_copy_plan(const void *src, unsigned long long bytes, const void *arr_end) {
    const unsigned long long s = (unsigned long long)src, e = s + bytes, ae = (unsigned long long)arr_end;
    const unsigned long long a0 = s & ~15ull, a1 = (e + 15) & ~15ull, lim = ae & ~15ull;
    const unsigned long long t1 = a1 <= ae ? a1 : lim;
    RangeCopy r;
    r.tma_bytes = t1 > a0 ? (unsigned)(t1 - a0) : 0u;
    r.offset = (unsigned)(s - a0);
    return r;
}
__device__ __forceinline__ void range_copy_issue(unsigned char *dst, const void *src, unsigned long long bytes,
                                                 const RangeCopy &r, uint64_t *bar) {
    const unsigned long long s = (unsigned long long)src, a0 = s & ~15ull;
    if (r.tma_bytes) bulk_g2s(dst, (const void *)a0, r.tma_bytes, bar);
    // bytes past the bulk copy (only at the very end of the array): plain loads
    const unsigned long long done = a0 + r.tma_bytes, e = s + bytes;
    for (unsigned long long b = done; b < e; b++)
        dst[b - a0] = *(const unsigned char *)b;
}

// Bounded wait for the completion of phase `parity` of bar: at most
// kMbarWaitTries probes, each suspending the thread for up to about 1 us,
// so a wait gives up after about a second instead of hanging.  Returns
// whether the phase completed.
constexpr unsigned kMbarWaitTries = 1u << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    for (unsigned it = 0; it < kMbarWaitTries; it++) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Count of bounded waits that gave up, one per translation unit (no
// relocatable device code); fem_wait_timeouts adds them up.
static __device__ unsigned long long g_wait_timeouts;

// Host side: reads (and with reset, clears) this translation unit's count.
#define FEM_DEFINE_WAIT_COUNTER(fn)                                                          \
    cudaError_t fn(unsigned long long *count, bool reset) {                                  \
        cudaError_t e = cudaMemcpyFromSymbol(count, g_wait_timeouts, sizeof(*count));        \
        if (e == cudaSuccess && reset) {                                                     \
            const unsigned long long zero = 0;                                               \
            e = cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(zero));                    \
        }                                                                                    \
        return e;                                                                            \
    }

// A geometric factor read as the arithmetic type T: FP64 and FP32 factors
// as they are, FP16 factors (the half-precision inner operator) widened.
template <typename T>
__device__ __forceinline__ T factor_ldg(const T *p) { return __ldg(p); }
template <typename T>
__device__ __forceinline__ T factor_ldg(const __half *p) { return (T)__half2float(__ldg(p)); }
template <typename T>
__device__ __forceinline__ T factor_ld(const T *p) { return *p; }
template <typename T>
__device__ __forceinline__ T factor_ld(const __half *p) { return (T)__half2float(*p); }

// Scale that undoes the power-of-two scaling of FP16 factors: read from
// device memory when given (set by the solver on the device), else 1.
template <typename T>
__device__ __forceinline__ T factor_unscale(const double *ginv) { return ginv ? (T)(*ginv) : T(1); }

// Fused multiply-add in the precision of the operands.
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }

// A product rounded on its own, never contracted into a later addition: the
// kernels that must give bit-identical results (BP1.0 alone and inside the
// one-pass BP1.0 + BP3.0 kernel) round wJ q the same way whatever the
// compiler fuses around it.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// Copies `count` doubles from global to shared with all threads of the block.
__device__ __forceinline__ void block_copy(double *dst, const double *__restrict__ src, int count) {
    for (int t = threadIdx.x; t < count; t += blockDim.x) dst[t] = __ldg(src + t);
}

// Sum of v over the block (blockDim.x a multiple of 32), in a fixed order so
// that repeated runs give identical bits; the result is valid in thread 0.
// sh: at least 32 doubles of shared memory not in use by other threads.
// Every thread of the block must call it.
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Hooks around the factor phase of the operator cores (bp35_core,
// bp30_core), for kernels that stage the factors asynchronously: before()
// runs on every thread after the barrier that precedes the factor phase and
// returns whether the factors are there (the same value on every thread;
// false ends the core at once), after() runs on every thread once the
// factor phase's barrier has passed (the factors are no longer read).  The
// default does nothing.
struct NoFactorHooks {
    __device__ __forceinline__ bool before() const { return true; }
    __device__ __forceinline__ void after() const {}
};

// Dispatch of a functor templated on the degree N (1..15) at run time.
template <template <int> class F, typename... Args>
cudaError_t dispatch_degree(int N, Args &&...args) {
    switch (N) {
#define FEM_CASE(K) \
    case K:         \
        return F<K>::run(args...);
        FEM_CASE(1) FEM_CASE(2) FEM_CASE(3) FEM_CASE(4) FEM_CASE(5)
        FEM_CASE(6) FEM_CASE(7) FEM_CASE(8) FEM_CASE(9) FEM_CASE(10)
        FEM_CASE(11) FEM_CASE(12) FEM_CASE(13) FEM_CASE(14) FEM_CASE(15)
#undef FEM_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace fem
