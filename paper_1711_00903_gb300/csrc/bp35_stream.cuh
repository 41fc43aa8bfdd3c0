// The persistent, double-buffered TMA stream form of the FP32 BP3.5 operator
// (odd degree up to 9), shared by the FP32-factor kernels (bp35.cu) and the
// FP16-factor kernels of the half-precision inner operator (bp35_f16.cu).
#pragma once

#include <atomic>

#include "bp35_body.cuh"

namespace fem {
namespace {

// ---------------------------------------------------------------------------
// FP32 stream kernel.  In FP32 the operator is bound by HBM, and a kernel
// that loads each element's factors with per-thread loads in the middle of
// its phases leaves the memory system idle while its blocks compute.  Here a
// fixed grid of persistent blocks (two per SM) walks groups of EPS elements;
// for every group one thread issues TMA bulk copies of the group's factor
// planes and input field(s) (contiguous ranges) into one of two shared
// stages, completing on that stage's mbarrier, one group ahead of the
// compute, so each SM always has a group's bytes in flight while it
// computes the previous one.  Needs n even (every element's ranges then
// span multiples of 16 bytes): odd N, up to 9 (two stages must fit).
constexpr bool bp35_streamed(int N) { return (N % 2) == 1 && N <= 9; }
constexpr int kStreamThreads35 = 128;

template <int N, bool PCG, typename TG = float>
struct Bp35Stream {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    static constexpr int EPS = (kStreamThreads35 / nn) > 1 ? kStreamThreads35 / nn : 1;  // elements per group
    using L = Bp35Layout<float, N, EPS>;
    static constexpr int threads = L::threads;
    static constexpr int gElem = 7 * NP * (int)sizeof(TG);      // factor bytes per element
    static constexpr int vElem = NP * 4;                        // field bytes per element
    static constexpr int stage = EPS * (gElem + (PCG ? 2 : 1) * vElem);
    static constexpr int oStage = 16;                           // two mbarriers, then the stages
    static constexpr int oBox = oStage + 2 * stage;
    static constexpr int smem = oBox + (L::smem > 256 ? L::smem : 256);
    // as many resident blocks per SM as the shared memory holds (at most 8):
    // at low degree a group is small, and more blocks keep more bytes in
    // flight per SM
    static constexpr int per_sm_raw = (220 * 1024) / (smem + 1024);
    static constexpr int blocks_per_sm = per_sm_raw > 8 ? 8 : (per_sm_raw < 1 ? 1 : per_sm_raw);
    static_assert(gElem % 16 == 0 && vElem % 16 == 0, "bulk copies move multiples of 16 bytes");
};

template <int N, bool PCG, typename TG>
__global__ void __launch_bounds__(Bp35Stream<N, PCG, TG>::threads)
bp35_stream_kernel(int64_t E, const TG *__restrict__ G, double lambda, const float *__restrict__ q,
                   float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
                   const double *__restrict__ beta, double *__restrict__ partials, const double *__restrict__ ginv) {
    using S = Bp35Stream<N, PCG, TG>;
    using B = typename S::L::B;
    constexpr int n = S::n, nn = S::nn, NP = S::NP, EPS = S::EPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *boxes = reinterpret_cast<float *>(smem_raw + S::oBox);
    const int64_t groups = (E + EPS - 1) / EPS;
    const float bt = PCG ? (float)(*beta) : 0.0f;
    const float gscale = factor_unscale<float>(ginv);
    const bool read_p = PCG && bt != 0.0f;

    // stage k of group g: [factors | field (q or z) | p]
    auto issue = [&](int64_t g, int k) {
        const int64_t e0 = g * EPS;
        const int nel = (int)((E - e0) < EPS ? (E - e0) : EPS);
        unsigned char *st = smem_raw + S::oStage + k * S::stage;
        const unsigned gb = (unsigned)(nel * S::gElem), vb = (unsigned)(nel * S::vElem);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive_expect_tx(&bar[k], gb + vb + (read_p ? vb : 0u));
        bulk_g2s(st, G + e0 * 7 * NP, gb, &bar[k]);
        bulk_g2s(st + EPS * S::gElem, (PCG ? z : q) + e0 * NP, vb, &bar[k]);
        if (read_p) bulk_g2s(st + EPS * (S::gElem + S::vElem), p + e0 * NP, vb, &bar[k]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        if ((int64_t)blockIdx.x < groups) issue(blockIdx.x, 0);
    }
    __syncthreads();

    double dot = 0.0;  // the thread's p . Ap over its groups (FP32 per group)
    bool ok = true;
    int it = 0;
    for (int64_t g = blockIdx.x; g < groups; g += gridDim.x, it++) {
        const int k = it & 1;
        const unsigned parity = (unsigned)((it >> 1) & 1);
        if (threadIdx.x == 0 && g + gridDim.x < groups) issue(g + gridDim.x, k ^ 1);
        const bool done = mbar_wait(&bar[k], parity);
        if (!done && (threadIdx.x & 31) == 0) atomicAdd(&g_wait_timeouts, 1ull);
        ok = ok && done;

        const int64_t e0 = g * EPS;
        const int nel = (int)((E - e0) < EPS ? (E - e0) : EPS);
        const unsigned char *st = smem_raw + S::oStage + k * S::stage;
        const TG *sG = reinterpret_cast<const TG *>(st);
        const float *sV = reinterpret_cast<const float *>(st + EPS * S::gElem);
        const float *sP = reinterpret_cast<const float *>(st + EPS * (S::gElem + S::vElem));
        for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
            const int el = t / NP, s = t - el * NP;
            float v = sV[t];
            if (PCG) {
                if (read_p) v = fmx(bt, sP[t], v);
                p[e0 * NP + t] = v;
            }
            boxes[el * 3 * B::size + B::at(s % n, (s / n) % n, s / nn)] = v;
        }
        __syncthreads();
        dot += (double)bp35_core<float, N, EPS, PCG, true, TG>(boxes, e0, nel, sG, lambda, Aq, gscale);
        __syncthreads();  // the stage and the boxes are free again
    }
    if (PCG) {
        const double tot = block_sum(dot, reinterpret_cast<double *>(boxes));
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
    // a copy that did not complete in time may still be in flight: wait for
    // both stages once more (bounded) before the shared memory is released
    if (!ok) {
        mbar_wait(&bar[0], (unsigned)(((it + 1) >> 1) & 1));
        mbar_wait(&bar[1], (unsigned)((it >> 1) & 1));
    }
}

inline std::atomic<int> g_sm_count[64];

// Persistent grid of the stream kernel on the current device (SM count
// looked up once per device).
inline int64_t stream_grid35(int64_t groups, int blocks_per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) sms = g_sm_count[dev].load(std::memory_order_relaxed);
    if (sms <= 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (dev >= 0 && dev < 64) g_sm_count[dev].store(sms, std::memory_order_relaxed);
    }
    const int64_t full = (int64_t)sms * blocks_per_sm;
    return groups < full ? groups : full;
}

template <int N, bool PCG, typename TG = float>
cudaError_t launch_stream35(int64_t E, const TG *G, double lambda, const float *q, float *Aq, const float *z,
                            float *p, const double *beta, double *partials, cudaStream_t s,
                            const double *ginv = nullptr) {
    using S = Bp35Stream<N, PCG, TG>;
    const int64_t grid = stream_grid35((E + S::EPS - 1) / S::EPS, S::blocks_per_sm);
    bp35_stream_kernel<N, PCG, TG><<<(unsigned)grid, S::threads, S::smem, s>>>(E, G, lambda, q, Aq, z, p, beta,
                                                                               partials, ginv);
    return cudaGetLastError();
}

// Shared-memory attributes of the stream kernels of one degree and factor type.
template <int N, typename TG>
cudaError_t prepare_stream35() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bp35_stream_kernel<N, false, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Bp35Stream<N, false, TG>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bp35_stream_kernel<N, false, TG>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bp35_stream_kernel<N, true, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Bp35Stream<N, true, TG>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bp35_stream_kernel<N, true, TG>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

}  // namespace
}  // namespace fem
