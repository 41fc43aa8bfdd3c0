// BP3.5 collocated screened-Poisson matvec (Algorithm 4):
//   Aq = D_r^T Rr + D_s^T Rs + D_t^T Rt + lambda wJ q,
//   [Rr Rs Rt] = G [q_r q_s q_t],  q_r = (D x I x I) q, ...
// in IEEE FP64 (the operator of the paper) and in FP32 (the inner operator
// of the mixed-precision solver), plus a variant fused with the PCG
// direction update p <- z + beta p and the p . Ap reduction.
//
// GB300 design.  FP64 issues at 2 instructions per clock per SM on this
// part (1/64 of the FP32 rate), so the FP64 kernel is bound by its FP64
// instruction count, not by HBM or shared memory (ncu: FP64 pipe 83-96 %
// busy, DRAM 4-11 %); the same code in FP32 is bound by HBM.  The design
// minimises FP64 instructions and spends shared memory, registers and
// integer issue freely:
//   * every one-dimensional contraction is one thread applying the even-odd
//     folded D or D^T to a whole line (eo.cuh): about n/2 + 2 instructions
//     per node instead of n, operator entries as constant-bank operands;
//   * q^e and the r and s partial results of the element live in shared
//     memory (padded boxes), the t-direction work of a thread's (i, j)
//     column stays in registers, four barriers per element;
//   * several elements per block (n^2 threads each), coalesced loads of q
//     and of each geometric-factor plane, coalesced stores.
// FP32 at odd degree up to 9 (the mixed solver's hot kernel) runs as a
// persistent, double-buffered TMA stream instead (see bp35_stream_kernel).
#include <atomic>

#include "bp35_body.cuh"

namespace fem {
namespace {

// Minimum resident blocks per SM that the register allocation must allow
// (0: the compiler's own heuristic).  At high degree the fully unrolled line
// kernels take up to 255 registers and leave one block per SM; capping them
// trades a few spills for latency hiding.  Chosen per precision and degree
// from the operator sweep on GB300.
template <typename T, int N>
constexpr int bp35_min_blocks() {
    if (sizeof(T) == 8) return N >= 10 ? 3 : 0;
    return N == 15 ? 3 : 0;
}

template <typename T, int N, bool PCG>
__device__ __forceinline__ void bp35_entry(int64_t E, const T *__restrict__ G, double lambda, const T *__restrict__ q,
                                           T *__restrict__ Aq, const T *__restrict__ z, T *__restrict__ p,
                                           const double *__restrict__ beta, double *__restrict__ partials) {
    using C = Bp35Cfg<T, N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * C::EPB;
    const int nel = (int)((E - e0) < C::EPB ? (E - e0) : C::EPB);
    bp35_block<T, N, C::EPB, PCG>(smem_raw, e0, nel, G, lambda, q, Aq, z, p, beta,
                                  PCG ? partials + blockIdx.x : nullptr);
}

template <typename T, int N, bool PCG>
__global__ void __launch_bounds__(Bp35Cfg<T, N>::threads)
bp35_kernel(int64_t E, const T *__restrict__ G, double lambda, const T *__restrict__ q, T *__restrict__ Aq,
            const T *__restrict__ z, T *__restrict__ p, const double *__restrict__ beta,
            double *__restrict__ partials) {
    bp35_entry<T, N, PCG>(E, G, lambda, q, Aq, z, p, beta, partials);
}

template <typename T, int N, bool PCG>
__global__ void __launch_bounds__(Bp35Cfg<T, N>::threads, bp35_min_blocks<T, N>())
bp35_kernel_capped(int64_t E, const T *__restrict__ G, double lambda, const T *__restrict__ q, T *__restrict__ Aq,
                   const T *__restrict__ z, T *__restrict__ p, const double *__restrict__ beta,
                   double *__restrict__ partials) {
    bp35_entry<T, N, PCG>(E, G, lambda, q, Aq, z, p, beta, partials);
}

template <typename T, int N, bool PCG>
constexpr auto bp35_fn() {
    if constexpr (bp35_min_blocks<T, N>() > 0)
        return &bp35_kernel_capped<T, N, PCG>;
    else
        return &bp35_kernel<T, N, PCG>;
}

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

template <int N, bool PCG>
struct Bp35Stream {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    static constexpr int EPS = (kStreamThreads35 / nn) > 1 ? kStreamThreads35 / nn : 1;  // elements per group
    using L = Bp35Layout<float, N, EPS>;
    static constexpr int threads = L::threads;
    static constexpr int gElem = 7 * NP * 4;                    // factor bytes per element
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

template <int N, bool PCG>
__global__ void __launch_bounds__(Bp35Stream<N, PCG>::threads)
bp35_stream_kernel(int64_t E, const float *__restrict__ G, double lambda, const float *__restrict__ q,
                   float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
                   const double *__restrict__ beta, double *__restrict__ partials) {
    using S = Bp35Stream<N, PCG>;
    using B = typename S::L::B;
    constexpr int n = S::n, nn = S::nn, NP = S::NP, EPS = S::EPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *boxes = reinterpret_cast<float *>(smem_raw + S::oBox);
    const int64_t groups = (E + EPS - 1) / EPS;
    const float bt = PCG ? (float)(*beta) : 0.0f;
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
        const float *sG = reinterpret_cast<const float *>(st);
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
        dot += (double)bp35_core<float, N, EPS, PCG, true>(boxes, e0, nel, sG, lambda, Aq);
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

std::atomic<int> g_sm_count[64];

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

template <int N, bool PCG>
cudaError_t launch_stream35(int64_t E, const float *G, double lambda, const float *q, float *Aq, const float *z,
                            float *p, const double *beta, double *partials, cudaStream_t s) {
    using S = Bp35Stream<N, PCG>;
    const int64_t grid = stream_grid35((E + S::EPS - 1) / S::EPS, S::blocks_per_sm);
    bp35_stream_kernel<N, PCG><<<(unsigned)grid, S::threads, S::smem, s>>>(E, G, lambda, q, Aq, z, p, beta,
                                                                           partials);
    return cudaGetLastError();
}

template <int N>
struct Bp35Launch {
    static cudaError_t run(int64_t E, const double *G, double lambda, const double *q, double *Aq,
                           cudaStream_t s) {
        using C = Bp35Cfg<double, N>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp35_fn<double, N, false>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(
            E, G, lambda, q, Aq, nullptr, nullptr, nullptr, nullptr);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp35F32Launch {
    static cudaError_t run(int64_t E, const float *G, double lambda, const float *q, float *Aq,
                           cudaStream_t s) {
        if constexpr (bp35_streamed(N)) {
            return launch_stream35<N, false>(E, G, lambda, q, Aq, nullptr, nullptr, nullptr, nullptr, s);
        } else {
            using C = Bp35Cfg<float, N>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            bp35_fn<float, N, false>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(
                E, G, lambda, q, Aq, nullptr, nullptr, nullptr, nullptr);
            return cudaGetLastError();
        }
    }
};

template <typename T>
struct Bp35PcgLaunchT {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const T *G, double lambda, const T *z, T *p, const double *beta,
                               T *Ap, double *partials, cudaStream_t s) {
            if constexpr (sizeof(T) == 4 && bp35_streamed(N)) {
                return launch_stream35<N, true>(E, G, lambda, nullptr, Ap, z, p, beta, partials, s);
            } else {
                using C = Bp35Cfg<T, N>;
                const int64_t blocks = (E + C::EPB - 1) / C::EPB;
                bp35_fn<T, N, true>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, lambda, nullptr, Ap, z,
                                                                                   p, beta, partials);
                return cudaGetLastError();
            }
        }
    };
};

template <int N>
struct Bp35Blocks {
    static cudaError_t run(int64_t E, int which, int64_t *out) {
        using C = Bp35Cfg<double, N>;
        using F = Bp35Cfg<float, N>;
        const int64_t a = (E + C::EPB - 1) / C::EPB;
        int64_t b = (E + F::EPB - 1) / F::EPB;
        if constexpr (bp35_streamed(N)) {
            using S = Bp35Stream<N, true>;
            b = stream_grid35((E + S::EPS - 1) / S::EPS, S::blocks_per_sm);
        }
        *out = which == 0 ? a : which == 1 ? b : (a > b ? a : b);
        return cudaSuccess;
    }
};

template <int N>
struct Bp35Prepare {
    template <typename T, bool PCG>
    static cudaError_t one() {
        return cudaFuncSetAttribute(bp35_fn<T, N, PCG>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Bp35Cfg<T, N>::smem);
    }
    static cudaError_t run() {
        cudaError_t e = one<double, false>();
        if (e == cudaSuccess) e = one<double, true>();
        if constexpr (bp35_streamed(N)) {
            // all operands live in shared memory: ask for the largest carveout
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(bp35_stream_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Bp35Stream<N, false>::smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(bp35_stream_kernel<N, false>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(bp35_stream_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Bp35Stream<N, true>::smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(bp35_stream_kernel<N, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         100);
        } else {
            if (e == cudaSuccess) e = one<float, false>();
            if (e == cudaSuccess) e = one<float, true>();
        }
        return e;
    }
};

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp35_tu)

}  // namespace

FEM_DEFINE_WAIT_COUNTER(wait_timeouts_bp35)

cudaError_t launch_bp35(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                        double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp35Launch>(b->host.N, E, G, lambda, q, Aq, s);
}

cudaError_t launch_bp35_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q,
                            float *Aq, cudaStream_t s) {
    return dispatch_degree<Bp35F32Launch>(b->host.N, E, G, lambda, q, Aq, s);
}

cudaError_t launch_bp35_pcg(const fem_basis *b, int64_t E, const double *G, double lambda, const double *z,
                            double *p, const double *beta, double *Ap, double *partials, cudaStream_t s) {
    return dispatch_degree<Bp35PcgLaunchT<double>::L>(b->host.N, E, G, lambda, z, p, beta, Ap, partials, s);
}

cudaError_t launch_bp35_pcg_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                float *p, const double *beta, float *Ap, double *partials, cudaStream_t s) {
    return dispatch_degree<Bp35PcgLaunchT<float>::L>(b->host.N, E, G, lambda, z, p, beta, Ap, partials, s);
}

int64_t bp35_max_blocks(int N, int64_t E) {
    int64_t out = 0;
    dispatch_degree<Bp35Blocks>(N, E, 2, &out);
    return out;
}

int64_t bp35_blocks(int N, int64_t E, bool f32) {
    int64_t out = 0;
    dispatch_degree<Bp35Blocks>(N, E, f32 ? 1 : 0, &out);
    return out;
}

cudaError_t prepare_bp35(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp35_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<Bp35Prepare>(N);
}

}  // namespace fem
