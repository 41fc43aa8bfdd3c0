// The persistent TMA stream forms of the FP32 BP3.5 operator (two stages up
// to degree 9, one factor stage at any degree where it fits), shared by the
// FP32-factor kernels (bp35.cu) and the FP16-factor kernels of the
// half-precision inner operator (bp35_f16.cu); bp35_one_stage_pick chooses
// per degree, factor type and variant.
#pragma once

#include <atomic>

#include "bp35_body.cuh"

namespace fem {
namespace {

// ---------------------------------------------------------------------------
// FP32 stream kernel.  In FP32 the operator is bound by HBM, and a kernel
// that loads each element's factors with per-thread loads in the middle of
// its phases leaves the memory system idle while its blocks compute.  Here a
// fixed grid of persistent blocks (as many per SM as the shared memory
// holds) walks groups of EPS elements;
// for every group one thread issues TMA bulk copies of the group's factor
// planes and input field(s) (contiguous ranges) into one of two shared
// stages, completing on that stage's mbarrier, one group ahead of the
// compute, so each SM always has a group's bytes in flight while it
// computes the previous one.  For odd n (even N) an element's ranges are not
// multiples of 16 bytes; each range is then copied as its enclosing
// 16-byte-aligned range (range_copy_plan) and read at its offset.  Up to
// N = 9 (two stages must fit in shared memory).
constexpr bool bp35_two_stage_fits(int N) { return N <= 9; }
constexpr int kStreamThreads35 = 128;

template <int N, bool PCG, typename TG = float>
struct Bp35Stream {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    static constexpr int EPS = (kStreamThreads35 / nn) > 1 ? kStreamThreads35 / nn : 1;  // elements per group
    using L = Bp35Layout<float, N, EPS, true>;
    static constexpr int threads = L::threads;
    static constexpr int gElem = 7 * NP * (int)sizeof(TG);      // factor bytes per element
    static constexpr int vElem = NP * 4;                        // field bytes per element
    // element ranges on 16-byte boundaries (n even): plain bulk copies;
    // otherwise room for each range's aligned enclosing range
    static constexpr bool ALIGNED = gElem % 16 == 0 && vElem % 16 == 0;
    static constexpr int gRegion = ALIGNED ? EPS * gElem : ((EPS * gElem + 32 + 15) / 16) * 16;
    static constexpr int vRegion = ALIGNED ? EPS * vElem : ((EPS * vElem + 32 + 15) / 16) * 16;
    static constexpr int stage = gRegion + (PCG ? 2 : 1) * vRegion;
    static constexpr int oStage = 16;                           // two mbarriers, then the stages
    static constexpr int oBox = oStage + 2 * stage;
    static constexpr int smem = oBox + (L::smem > 256 ? L::smem : 256);
    // as many resident blocks per SM as the shared memory holds (at most 8):
    // at low degree a group is small, and more blocks keep more bytes in
    // flight per SM
    static constexpr int per_sm_raw = (220 * 1024) / (smem + 1024);
    static constexpr int blocks_per_sm = per_sm_raw > 8 ? 8 : (per_sm_raw < 1 ? 1 : per_sm_raw);
};

template <int N, bool PCG, typename TG>
__global__ void __launch_bounds__(Bp35Stream<N, PCG, TG>::threads)
bp35_stream_kernel(int64_t E, const TG *__restrict__ G, double lambda, const float *__restrict__ q,
                   float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
                   const double *__restrict__ beta, double *__restrict__ partials, const double *__restrict__ ginv,
                   double *__restrict__ status) {
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

    const float *fld = PCG ? z : q;
    const TG *G_end = G + E * 7 * NP;
    const float *fld_end = fld + E * NP;
    const float *p_end = PCG ? p + E * NP : nullptr;
    // the copy plans of group g: factors, field, and (PCG, beta != 0) p
    struct Plans {
        RangeCopy g, v, p;
    };
    auto plans = [&](int64_t g) {
        const int64_t e0 = g * EPS;
        const int nel = (int)((E - e0) < EPS ? (E - e0) : EPS);
        Plans pl;
        if constexpr (S::ALIGNED) {
            pl.g = RangeCopy{(unsigned)(nel * S::gElem), 0u};
            pl.v = RangeCopy{(unsigned)(nel * S::vElem), 0u};
            pl.p = RangeCopy{read_p ? (unsigned)(nel * S::vElem) : 0u, 0u};
        } else {
            pl.g = range_copy_plan(G + e0 * 7 * NP, (unsigned long long)nel * S::gElem, G_end);
            pl.v = range_copy_plan(fld + e0 * NP, (unsigned long long)nel * S::vElem, fld_end);
            pl.p = read_p ? range_copy_plan(p + e0 * NP, (unsigned long long)nel * S::vElem, p_end) : RangeCopy{0u, 0u};
        }
        return pl;
    };
    // stage k of group g: [factors | field (q or z) | p]
    auto issue = [&](int64_t g, int k) {
        const int64_t e0 = g * EPS;
        const int nel = (int)((E - e0) < EPS ? (E - e0) : EPS);
        unsigned char *st = smem_raw + S::oStage + k * S::stage;
        const Plans pl = plans(g);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive_expect_tx(&bar[k], pl.g.tma_bytes + pl.v.tma_bytes + (read_p ? pl.p.tma_bytes : 0u));
        if constexpr (S::ALIGNED) {
            bulk_g2s(st, G + e0 * 7 * NP, pl.g.tma_bytes, &bar[k]);
            bulk_g2s(st + S::gRegion, fld + e0 * NP, pl.v.tma_bytes, &bar[k]);
            if (read_p) bulk_g2s(st + S::gRegion + S::vRegion, p + e0 * NP, pl.p.tma_bytes, &bar[k]);
        } else {
            range_copy_issue(st, G + e0 * 7 * NP, (unsigned long long)nel * S::gElem, pl.g, &bar[k]);
            range_copy_issue(st + S::gRegion, fld + e0 * NP, (unsigned long long)nel * S::vElem, pl.v, &bar[k]);
            if (read_p)
                range_copy_issue(st + S::gRegion + S::vRegion, p + e0 * NP, (unsigned long long)nel * S::vElem, pl.p,
                                 &bar[k]);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        if ((int64_t)blockIdx.x < groups) issue(blockIdx.x, 0);
    }
    __syncthreads();

    double dot = 0.0;  // the thread's p . Ap over its groups (FP32 per group)
    bool failed = false, next_issued = false;
    int it = 0;
    for (int64_t g = blockIdx.x; g < groups; g += gridDim.x, it++) {
        const int k = it & 1;
        const unsigned parity = (unsigned)((it >> 1) & 1);
        next_issued = g + gridDim.x < groups;
        if (threadIdx.x == 0 && next_issued) issue(g + gridDim.x, k ^ 1);
        // the whole block leaves together when any of its threads gave up
        if (!__syncthreads_and(mbar_wait(&bar[k], parity))) {
            failed = true;
            break;
        }

        const int64_t e0 = g * EPS;
        const int nel = (int)((E - e0) < EPS ? (E - e0) : EPS);
        const Plans pl = plans(g);
        const unsigned char *st = smem_raw + S::oStage + k * S::stage;
        const TG *sG = reinterpret_cast<const TG *>(st + pl.g.offset);
        const float *sV = reinterpret_cast<const float *>(st + S::gRegion + pl.v.offset);
        const float *sP = reinterpret_cast<const float *>(st + S::gRegion + S::vRegion + pl.p.offset);
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
        dot += (double)bp35_core<float, N, EPS, PCG, true, TG, NoFactorHooks, true>(boxes, e0, nel, sG, lambda, Aq,
                                                                                      gscale);
        __syncthreads();  // the stage and the boxes are free again
    }
    if (failed) {
        // A stage did not land within the wait's limit: no more copies are
        // issued and nothing more is computed.  The block reports it (the
        // library-wide count, and the caller's status word when given),
        // then waits once more, bounded, for the copies that may still be
        // in flight (this iteration's stage and, if it was issued, the
        // next one) before its shared memory is released.
        if (threadIdx.x == 0) {
            atomicAdd(&g_wait_timeouts, 1ull);
            if (status) *status = 1.0;
        }
        const int k = it & 1;
        mbar_wait(&bar[k], (unsigned)((it >> 1) & 1));
        if (next_issued) mbar_wait(&bar[k ^ 1], (unsigned)(((it + 1) >> 1) & 1));
        if (PCG && threadIdx.x == 0) partials[blockIdx.x] = 0.0;
        return;
    }
    if (PCG) {
        const double tot = block_sum(dot, reinterpret_cast<double *>(boxes));
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
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
                            const double *ginv = nullptr, double *status = nullptr) {
    using S = Bp35Stream<N, PCG, TG>;
    const int64_t grid = stream_grid35((E + S::EPS - 1) / S::EPS, S::blocks_per_sm);
    bp35_stream_kernel<N, PCG, TG><<<(unsigned)grid, S::threads, S::smem, s>>>(E, G, lambda, q, Aq, z, p, beta,
                                                                               partials, ginv, status);
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

// ---------------------------------------------------------------------------
// Single-factor-stage stream kernel: above degree 9 two stages of an
// element's factors (37-115 KB in FP32) do not fit in shared memory, and
// at degrees 6-9 one element per block with one factor stage lets more
// blocks share an SM than the two-stage kernel.  One element per group;
// the input field is double-buffered (TMA
// bulk copies, one group ahead) and the factors have one stage: the copy of
// the next group's factors is issued as soon as this group's factor phase
// has passed its barrier (bp35_core's hooks), so it lands while this group
// finishes (transposes, output) and the next one stages its field and
// takes its derivatives.  The PCG variant reads the old p directly from
// global memory in the staging loop (a stage for it would not fit at
// N = 15).  Every wait is bounded; a block whose wait gives up stops
// issuing copies, waits once more (bounded) for those in flight, reports
// through the status word and leaves.
template <int N, bool PCG, typename TG = float>
struct Bp35Stream1 {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    using L = Bp35Layout<float, N, 1, true>;
    static constexpr int threads = L::threads;
    static constexpr int gElem = 7 * NP * (int)sizeof(TG);
    static constexpr int vElem = NP * 4;
    static constexpr bool ALIGNED = gElem % 16 == 0 && vElem % 16 == 0;
    static constexpr int gRegion = ALIGNED ? gElem : ((gElem + 32 + 15) / 16) * 16;
    static constexpr int vRegion = ALIGNED ? vElem : ((vElem + 32 + 15) / 16) * 16;
    static constexpr int oG = 32;  // three mbarriers, then the factor stage
    static constexpr int oV = oG + gRegion;
    static constexpr int oBox = oV + 2 * vRegion;
    static constexpr int smem = oBox + (L::smem > 256 ? L::smem : 256);
    static constexpr bool fits = smem <= 227 * 1024;
    static constexpr int per_sm_raw = (220 * 1024) / (smem + 1024);
    // up to 16 resident blocks: at middle degrees a block is small (one
    // element, 64-100 threads), and more of them keep more copies in flight
    static constexpr int blocks_per_sm = per_sm_raw > 16 ? 16 : (per_sm_raw < 1 ? 1 : per_sm_raw);
};

// The kernel form per degree and factor type, from the operator sweep on the
// 32^3 mesh (GB300, fraction of the copy rate at the operator's bytes):
//   - the one-factor-stage kernel from N = 6 where it fits and measured
//     faster: FP32 factors 0.87-0.91 at N = 6-9 against 0.80-0.85 for the
//     two-stage kernel, 0.78-0.97 at N = 10-12, 14, 15 against 0.57-0.70
//     for the block kernel; FP16 factors at N = 6-8 (0.60-0.82 against
//     0.56-0.73) and 10-14 (0.46-0.72 against 0.39-0.56);
//   - the two-stage kernel up to N = 5 (at N = 3-5 the one-stage kernel
//     measured 0.69-0.78 against 0.79-0.89), and with FP16 factors at N = 9;
//   - the block kernel at N = 13 with FP32 factors (one one-stage block per
//     SM fits; 0.62 against 0.65) and at N = 15 with FP16 factors (0.48
//     against 0.50);
//   - the PCG variants (p <- z + beta p fused in) keep the two-stage kernel
//     up to N = 9, which stages the old p by TMA: the mixed solves at N = 7
//     measured 207 us per inner iteration with it, 258 with the one-stage
//     kernel reading p in its staging loop, and 211 with a TMA stage for p
//     added to the one-stage kernel.
template <int N, bool PCG, typename TG>
constexpr bool bp35_one_stage_pick() {
    if (PCG && bp35_two_stage_fits(N)) return false;
    return sizeof(TG) == 4 ? (N >= 6 && N != 13) : ((N >= 6 && N <= 8) || (N >= 10 && N <= 14));
}
template <int N, bool PCG, typename TG>
constexpr bool bp35_streamed() {
    return bp35_two_stage_fits(N) && !bp35_one_stage_pick<N, PCG, TG>();
}
template <int N, bool PCG, typename TG>
constexpr bool bp35_streamed1() {
    return bp35_one_stage_pick<N, PCG, TG>() && Bp35Stream1<N, PCG, TG>::fits;
}

template <int N, bool PCG, typename TG>
__global__ void __launch_bounds__(Bp35Stream1<N, PCG, TG>::threads)
bp35_stream1_kernel(int64_t E, const TG *__restrict__ G, double lambda, const float *__restrict__ q,
                    float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
                    const double *__restrict__ beta, double *__restrict__ partials, const double *__restrict__ ginv,
                    double *__restrict__ status) {
    using S = Bp35Stream1<N, PCG, TG>;
    using B = typename S::L::B;
    constexpr int n = S::n, nn = S::nn, NP = S::NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);  // [0] factors, [1], [2] field stages
    float *boxes = reinterpret_cast<float *>(smem_raw + S::oBox);
    const float bt = PCG ? (float)(*beta) : 0.0f;
    const float gscale = factor_unscale<float>(ginv);
    const float *fld = PCG ? z : q;
    const TG *G_end = G + E * 7 * NP;
    const float *fld_end = fld + E * NP;

    auto gplan = [&](int64_t e) {
        return S::ALIGNED ? RangeCopy{(unsigned)S::gElem, 0u}
                          : range_copy_plan(G + e * 7 * NP, (unsigned long long)S::gElem, G_end);
    };
    auto vplan = [&](int64_t e) {
        return S::ALIGNED ? RangeCopy{(unsigned)S::vElem, 0u}
                          : range_copy_plan(fld + e * NP, (unsigned long long)S::vElem, fld_end);
    };
    auto issue_g = [&](int64_t e) {
        const RangeCopy pl = gplan(e);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive_expect_tx(&bar[0], pl.tma_bytes);
        range_copy_issue(smem_raw + S::oG, G + e * 7 * NP, (unsigned long long)S::gElem, pl, &bar[0]);
    };
    auto issue_v = [&](int64_t e, int k) {
        const RangeCopy pl = vplan(e);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive_expect_tx(&bar[1 + k], pl.tma_bytes);
        range_copy_issue(smem_raw + S::oV + k * S::vRegion, fld + e * NP, (unsigned long long)S::vElem, pl,
                         &bar[1 + k]);
    };

    // copies in flight, the same on every thread: the factors of the
    // current element, and each field stage with the use it belongs to
    bool pend_g = false, pend_v[2] = {false, false};
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        if ((int64_t)blockIdx.x < E) {
            issue_g(blockIdx.x);
            issue_v(blockIdx.x, 0);
        }
    }
    if ((int64_t)blockIdx.x < E) pend_g = pend_v[0] = true;
    __syncthreads();

    double dot = 0.0;
    bool failed = false;
    int it = 0;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x, it++) {
        const int k = it & 1;
        const bool has_next = e + gridDim.x < E;
        if (has_next) {
            if (threadIdx.x == 0) issue_v(e + gridDim.x, k ^ 1);
            pend_v[k ^ 1] = true;
        }
        if (!__syncthreads_and(mbar_wait(&bar[1 + k], (unsigned)((it >> 1) & 1)))) {
            failed = true;
            break;
        }
        pend_v[k] = false;

        const RangeCopy vp = vplan(e), gp = gplan(e);
        const float *sV = reinterpret_cast<const float *>(smem_raw + S::oV + k * S::vRegion + vp.offset);
        const TG *sG = reinterpret_cast<const TG *>(smem_raw + S::oG + gp.offset);
        for (int t = threadIdx.x; t < NP; t += blockDim.x) {
            float v = sV[t];
            if (PCG) {
                if (bt != 0.0f) v = fmx(bt, p[e * NP + t], v);
                p[e * NP + t] = v;
            }
            boxes[B::at(t % n, (t / n) % n, t / nn)] = v;
        }
        __syncthreads();

        struct Hooks {
            uint64_t *barg;
            unsigned parity;
            bool *failed, *pend_g;
            const bool next;
            decltype(issue_g) *iss;
            int64_t next_e;
            __device__ __forceinline__ bool before() const {
                const bool ok = __syncthreads_and(mbar_wait(barg, parity));
                if (!ok) *failed = true;
                return ok;
            }
            __device__ __forceinline__ void after() const {
                // the factor stage is free: the next element's factors go in now
                *pend_g = next;
                if (next && threadIdx.x == 0) (*iss)(next_e);
            }
        } hooks{&bar[0], (unsigned)(it & 1), &failed, &pend_g, has_next, &issue_g, e + gridDim.x};
        dot += (double)bp35_core<float, N, 1, PCG, true, TG, Hooks, true>(boxes, e, 1, sG, lambda, Aq, gscale,
                                                                           hooks);
        if (failed) break;
        __syncthreads();  // the boxes and the field stage are free again
    }
    if (failed) {
        // report, then wait once more (bounded) for every copy still in
        // flight before the shared memory is released
        if (threadIdx.x == 0) {
            atomicAdd(&g_wait_timeouts, 1ull);
            if (status) *status = 1.0;
        }
        if (pend_g) mbar_wait(&bar[0], (unsigned)(it & 1));
        for (int kk = 0; kk < 2; kk++)
            if (pend_v[kk]) {
                // stage kk's outstanding copy belongs to iteration it (kk == it & 1) or it + 1
                const int owner = (kk == (it & 1)) ? it : it + 1;
                mbar_wait(&bar[1 + kk], (unsigned)((owner >> 1) & 1));
            }
        if (PCG && threadIdx.x == 0) partials[blockIdx.x] = 0.0;
        return;
    }
    if (PCG) {
        const double tot = block_sum(dot, reinterpret_cast<double *>(boxes));
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

template <int N, bool PCG, typename TG = float>
cudaError_t launch_stream35_1(int64_t E, const TG *G, double lambda, const float *q, float *Aq, const float *z,
                              float *p, const double *beta, double *partials, cudaStream_t s,
                              const double *ginv = nullptr, double *status = nullptr) {
    using S = Bp35Stream1<N, PCG, TG>;
    const int64_t grid = stream_grid35(E, S::blocks_per_sm);
    bp35_stream1_kernel<N, PCG, TG><<<(unsigned)grid, S::threads, S::smem, s>>>(E, G, lambda, q, Aq, z, p, beta,
                                                                                partials, ginv, status);
    return cudaGetLastError();
}

template <int N, typename TG>
cudaError_t prepare_stream35_1() {
    cudaError_t e = cudaSuccess;
    if constexpr (Bp35Stream1<N, false, TG>::fits) {
        e = cudaFuncSetAttribute(bp35_stream1_kernel<N, false, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Bp35Stream1<N, false, TG>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp35_stream1_kernel<N, false, TG>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    if constexpr (Bp35Stream1<N, true, TG>::fits) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp35_stream1_kernel<N, true, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Bp35Stream1<N, true, TG>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp35_stream1_kernel<N, true, TG>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return e;
}

}  // namespace
}  // namespace fem
