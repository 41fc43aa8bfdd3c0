// BP3.5 with half-precision factors: the inner operator of the FP16-factor
// mixed-precision solver (FEM_PCG_MIXED16).  The seven factor planes are
// stored in IEEE binary16, scaled by a power of two s so that their largest
// magnitude sits just below 2^14 (no overflow, no underflow of the small
// off-diagonal factors); the kernels widen every factor to FP32, compute in
// FP32 exactly as the FP32 operator does, and multiply the output by 1/s,
// read from device memory.  Half the factor bytes of the FP32 operator: 22
// instead of 36 bytes per degree of freedom at every N.
//
// Same two kernel forms as FP32: the persistent TMA stream kernel up to
// N = 9 (bp35_stream.cuh) and the block-per-element-group kernel with an
// L2 prefetch above.
#include "bp35_stream.cuh"

namespace fem {
namespace {

template <int N, bool PCG>
__device__ __forceinline__ void f16g_entry(int64_t E, const __half *__restrict__ G, const double *__restrict__ ginv,
                                           double lambda, const float *__restrict__ q, float *__restrict__ Aq,
                                           const float *__restrict__ z, float *__restrict__ p,
                                           const double *__restrict__ beta, double *__restrict__ partials) {
    using C = Bp35Cfg<float, N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * C::EPB;
    const int nel = (int)((E - e0) < C::EPB ? (E - e0) : C::EPB);
    bp35_block<float, N, C::EPB, PCG, __half>(smem_raw, e0, nel, G, lambda, q, Aq, z, p, beta,
                                              PCG ? partials + blockIdx.x : nullptr, ginv);
}

// the FP32 operator's register caps apply (bp35_min_blocks)
template <int N, bool PCG>
__global__ void __launch_bounds__(Bp35Cfg<float, N>::threads)
bp35_f16g_kernel(int64_t E, const __half *__restrict__ G, const double *__restrict__ ginv, double lambda,
                 const float *__restrict__ q, float *__restrict__ Aq, const float *__restrict__ z,
                 float *__restrict__ p, const double *__restrict__ beta, double *__restrict__ partials) {
    f16g_entry<N, PCG>(E, G, ginv, lambda, q, Aq, z, p, beta, partials);
}
template <int N, bool PCG>
__global__ void __launch_bounds__(Bp35Cfg<float, N>::threads, bp35_min_blocks<float, N>())
bp35_f16g_kernel_capped(int64_t E, const __half *__restrict__ G, const double *__restrict__ ginv, double lambda,
                        const float *__restrict__ q, float *__restrict__ Aq, const float *__restrict__ z,
                        float *__restrict__ p, const double *__restrict__ beta, double *__restrict__ partials) {
    f16g_entry<N, PCG>(E, G, ginv, lambda, q, Aq, z, p, beta, partials);
}
template <int N, bool PCG>
constexpr auto f16g_fn() {
    if constexpr (bp35_min_blocks<float, N>() > 0)
        return &bp35_f16g_kernel_capped<N, PCG>;
    else
        return &bp35_f16g_kernel<N, PCG>;
}

template <bool PCG>
struct F16Launch {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const __half *G, const double *ginv, double lambda, const float *q,
                               float *Aq, const float *z, float *p, const double *beta, double *partials,
                               cudaStream_t s, double *status) {
            if constexpr (bp35_streamed<N, PCG, __half>()) {
                return launch_stream35<N, PCG, __half>(E, G, lambda, q, Aq, z, p, beta, partials, s, ginv, status);
            } else if constexpr (bp35_streamed1<N, PCG, __half>()) {
                return launch_stream35_1<N, PCG, __half>(E, G, lambda, q, Aq, z, p, beta, partials, s, ginv,
                                                         status);
            } else {
                using C = Bp35Cfg<float, N>;
                const int64_t blocks = (E + C::EPB - 1) / C::EPB;
                f16g_fn<N, PCG>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, ginv, lambda, q, Aq, z, p,
                                                                                beta, partials);
                return cudaGetLastError();
            }
        }
    };
};

template <int N>
struct F16Blocks {
    static cudaError_t run(int64_t E, int64_t *out) {
        if constexpr (bp35_streamed<N, true, __half>()) {
            using S = Bp35Stream<N, true, __half>;
            *out = stream_grid35((E + S::EPS - 1) / S::EPS, S::blocks_per_sm);
        } else if constexpr (bp35_streamed1<N, true, __half>()) {
            *out = stream_grid35(E, Bp35Stream1<N, true, __half>::blocks_per_sm);
        } else {
            using C = Bp35Cfg<float, N>;
            *out = (E + C::EPB - 1) / C::EPB;
        }
        return cudaSuccess;
    }
};

template <int N>
struct F16Prepare {
    static cudaError_t run() {
        cudaError_t e = cudaFuncSetAttribute(f16g_fn<N, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Bp35Cfg<float, N>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f16g_fn<N, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Bp35Cfg<float, N>::smem);
        if constexpr (bp35_two_stage_fits(N))
            if (e == cudaSuccess) e = prepare_stream35<N, __half>();
        if (e == cudaSuccess) e = prepare_stream35_1<N, __half>();
        return e;
    }
};

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp35_f16_tu)

}  // namespace

FEM_DEFINE_WAIT_COUNTER(wait_timeouts_bp35_f16)

cudaError_t launch_bp35_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                             const float *q, float *Aq, cudaStream_t s) {
    return dispatch_degree<F16Launch<false>::L>(b->host.N, E, G, ginv, lambda, q, Aq, (const float *)nullptr,
                                                (float *)nullptr, (const double *)nullptr, (double *)nullptr, s,
                                                (double *)nullptr);
}

cudaError_t launch_bp35_pcg_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                                 const float *z, float *p, const double *beta, float *Ap, double *partials,
                                 cudaStream_t s, double *status) {
    return dispatch_degree<F16Launch<true>::L>(b->host.N, E, G, ginv, lambda, (const float *)nullptr, Ap, z, p, beta,
                                               partials, s, status);
}

int64_t bp35_f16_blocks(int N, int64_t E) {
    int64_t out = 0;
    dispatch_degree<F16Blocks>(N, E, &out);
    return out;
}

cudaError_t prepare_bp35_f16(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp35_f16_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<F16Prepare>(N);
}

}  // namespace fem
