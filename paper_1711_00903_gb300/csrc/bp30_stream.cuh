// FP32 BP3.0 (and its FP16-factor form) as a persistent TMA stream with one
// factor stage: the inner operator of the BP3.0 mixed-precision solves.
//
// The block kernel of bp30.cu reads each element's seven factor planes from
// global memory in its column phase, and its warps wait there (ncu: long
// scoreboard stalls first).  Here a fixed grid of persistent blocks walks
// groups of EPS elements.  For every group one thread issues TMA bulk
// copies of the group's input field (double-buffered, one group ahead) and
// of its factors (one stage) into shared memory; the next group's factors
// are issued as soon as this group's column phase has passed its barrier
// (bp30_core's hooks), so they land while this group runs its transposes
// and projections and the next one stages its field and interpolates.  The
// column phase then reads its factors from shared memory.  The PCG variant
// reads the old p directly from global memory in the staging loop.
//
// Every mbarrier wait is bounded (about a second); a block whose wait gives
// up stops issuing copies, waits once more (bounded) for those in flight,
// reports through the solve's status word and the library-wide count, and
// leaves.
#pragma once

#include "bp30_body.cuh"

namespace fem {
namespace {

template <int N, bool PCG, typename TG = float, int EPS_ = 1>
struct Bp30Stream {
    static constexpr int n = N + 1, m = N + 2, NP = n * n * n, MP = m * m * m;
    static constexpr int EPS = EPS_;
    using L = Bp30Layout<N, EPS, float>;
    static constexpr int threads = L::threads;
    static constexpr int gElem = 7 * MP * (int)sizeof(TG);
    static constexpr int vElem = NP * 4;
    static constexpr bool ALIGNED = gElem % 16 == 0 && vElem % 16 == 0;
    static constexpr int gRegion = ALIGNED ? EPS * gElem : ((EPS * gElem + 32 + 15) / 16) * 16;
    static constexpr int vRegion = ALIGNED ? EPS * vElem : ((EPS * vElem + 32 + 15) / 16) * 16;
    static constexpr int oG = 32;  // three mbarriers, then the factor stage
    static constexpr int oV = oG + gRegion;
    static constexpr int oBox = oV + 2 * vRegion;
    static constexpr int smem = oBox + (L::smem > 256 ? L::smem : 256);
    static constexpr bool fits = smem <= 227 * 1024;
    static constexpr int per_sm_raw = (224 * 1024) / (smem + 1024);
    static constexpr int blocks_per_sm = per_sm_raw > 16 ? 16 : (per_sm_raw < 1 ? 1 : per_sm_raw);
};

template <int N, bool PCG, typename TG, int EPS>
__global__ void __launch_bounds__(Bp30Stream<N, PCG, TG, EPS>::threads)
bp30_stream_kernel(int64_t E, const TG *__restrict__ G, double lambda, const float *__restrict__ q,
                   float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
                   const double *__restrict__ beta, double *__restrict__ partials, const double *__restrict__ ginv,
                   double *__restrict__ status) {
    using S = Bp30Stream<N, PCG, TG, EPS>;
    using B0 = typename S::L::B0;
    constexpr int n = S::n, NP = S::NP, MP = S::MP;
    constexpr int SZ = S::L::S, per = S::L::per;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);  // [0] factors, [1], [2] field stages
    float *boxes = reinterpret_cast<float *>(smem_raw + S::oBox);
    const int64_t groups = (E + EPS - 1) / EPS;
    const float bt = PCG ? (float)(*beta) : 0.0f;
    const float gscale = std::is_same<TG, float>::value ? 1.0f : factor_unscale<float>(ginv);
    const float *fld = PCG ? z : q;
    const TG *G_end = G + E * 7 * MP;
    const float *fld_end = fld + E * NP;

    auto nel_of = [&](int64_t g) { return (int)((E - g * EPS) < EPS ? (E - g * EPS) : EPS); };
    auto gplan = [&](int64_t g) {
        const unsigned long long bytes = (unsigned long long)nel_of(g) * S::gElem;
        return S::ALIGNED ? RangeCopy{(unsigned)bytes, 0u} : range_copy_plan(G + g * EPS * 7 * MP, bytes, G_end);
    };
    auto vplan = [&](int64_t g) {
        const unsigned long long bytes = (unsigned long long)nel_of(g) * S::vElem;
        return S::ALIGNED ? RangeCopy{(unsigned)bytes, 0u} : range_copy_plan(fld + g * EPS * NP, bytes, fld_end);
    };
    auto issue_g = [&](int64_t g) {
        const RangeCopy pl = gplan(g);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive_expect_tx(&bar[0], pl.tma_bytes);
        range_copy_issue(smem_raw + S::oG, G + g * EPS * 7 * MP, (unsigned long long)nel_of(g) * S::gElem, pl,
                         &bar[0]);
    };
    auto issue_v = [&](int64_t g, int k) {
        const RangeCopy pl = vplan(g);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive_expect_tx(&bar[1 + k], pl.tma_bytes);
        range_copy_issue(smem_raw + S::oV + k * S::vRegion, fld + g * EPS * NP,
                         (unsigned long long)nel_of(g) * S::vElem, pl, &bar[1 + k]);
    };

    // copies in flight, the same on every thread
    bool pend_g = false, pend_v[2] = {false, false};
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        if ((int64_t)blockIdx.x < groups) {
            issue_g(blockIdx.x);
            issue_v(blockIdx.x, 0);
        }
    }
    if ((int64_t)blockIdx.x < groups) pend_g = pend_v[0] = true;
    __syncthreads();

    struct Hooks {
        uint64_t *barg;
        unsigned parity;
        bool *failed, *pend_g;
        bool next;
        int64_t next_g;
        const decltype(issue_g) *iss;
        __device__ __forceinline__ bool before() const {
            const bool ok = __syncthreads_and(mbar_wait(barg, parity));
            if (!ok) *failed = true;
            return ok;
        }
        __device__ __forceinline__ void after() const {
            // the factor stage is free: the next group's factors go in now
            *pend_g = next;
            if (next && threadIdx.x == 0) (*iss)(next_g);
        }
    };

    double dot = 0.0;
    bool failed = false;
    int it = 0;
    for (int64_t g = blockIdx.x; g < groups; g += gridDim.x, it++) {
        const int k = it & 1;
        const bool has_next = g + gridDim.x < groups;
        if (has_next) {
            if (threadIdx.x == 0) issue_v(g + gridDim.x, k ^ 1);
            pend_v[k ^ 1] = true;
        }
        if (!__syncthreads_and(mbar_wait(&bar[1 + k], (unsigned)((it >> 1) & 1)))) {
            failed = true;
            break;
        }
        pend_v[k] = false;

        const int64_t e0 = g * EPS;
        const int nel = nel_of(g);
        const RangeCopy vp = vplan(g), gp = gplan(g);
        const float *sV = reinterpret_cast<const float *>(smem_raw + S::oV + k * S::vRegion + vp.offset);
        const TG *sG = reinterpret_cast<const TG *>(smem_raw + S::oG + gp.offset);
        for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
            const int el = t / NP, s = t - el * NP;
            float v = sV[t];
            if (PCG) {
                if (bt != 0.0f) v = fmx(bt, p[e0 * NP + t], v);
                p[e0 * NP + t] = v;
            }
            boxes[el * per + SZ + B0::at(s % n, (s / n) % n, s / (n * n))] = v;
        }
        __syncthreads();

        const Hooks hooks{&bar[0], (unsigned)(it & 1), &failed, &pend_g, has_next, g + gridDim.x, &issue_g};
        dot += (double)bp30_core<N, EPS, float, PCG, true, TG, false, Hooks>(boxes, e0, nel, sG, lambda, Aq, p,
                                                                             gscale, nullptr, hooks);
        if (failed) break;
        __syncthreads();  // the boxes and the field stage are free again
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicAdd(&g_wait_timeouts, 1ull);
            if (status) *status = 1.0;
        }
        if (pend_g) mbar_wait(&bar[0], (unsigned)(it & 1));
        for (int kk = 0; kk < 2; kk++)
            if (pend_v[kk]) {
                const int owner = (kk == (it & 1)) ? it : it + 1;
                mbar_wait(&bar[1 + kk], (unsigned)((owner >> 1) & 1));
            }
        if (PCG && threadIdx.x == 0) partials[blockIdx.x] = 0.0;
        return;
    }
    if (PCG) {
        __syncthreads();
        const double tot = block_sum(dot, reinterpret_cast<double *>(boxes));
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

// Persistent grid on the current device (SM count looked up once).
inline int64_t stream_grid30(int64_t groups, int blocks_per_sm) {
    static int sms[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int s = (dev >= 0 && dev < 64) ? sms[dev] : 0;
    if (s <= 0) {
        cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (s <= 0) s = 1;
        if (dev >= 0 && dev < 64) sms[dev] = s;
    }
    const int64_t full = (int64_t)s * blocks_per_sm;
    return groups < full ? groups : full;
}

template <int N, bool PCG, typename TG, int EPS>
cudaError_t launch_stream30(int64_t E, const TG *G, double lambda, const float *q, float *Aq, const float *z,
                            float *p, const double *beta, double *partials, cudaStream_t s, const double *ginv,
                            double *status) {
    using S = Bp30Stream<N, PCG, TG, EPS>;
    const int64_t grid = stream_grid30((E + EPS - 1) / EPS, S::blocks_per_sm);
    bp30_stream_kernel<N, PCG, TG, EPS><<<(unsigned)grid, S::threads, S::smem, s>>>(E, G, lambda, q, Aq, z, p, beta,
                                                                                    partials, ginv, status);
    return cudaGetLastError();
}

template <int N, typename TG, int EPS>
cudaError_t prepare_stream30() {
    cudaError_t e = cudaSuccess;
    if constexpr (Bp30Stream<N, false, TG, EPS>::fits) {
        e = cudaFuncSetAttribute(bp30_stream_kernel<N, false, TG, EPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Bp30Stream<N, false, TG, EPS>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp30_stream_kernel<N, false, TG, EPS>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    if constexpr (Bp30Stream<N, true, TG, EPS>::fits) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp30_stream_kernel<N, true, TG, EPS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, Bp30Stream<N, true, TG, EPS>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp30_stream_kernel<N, true, TG, EPS>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return e;
}

}  // namespace
}  // namespace fem
