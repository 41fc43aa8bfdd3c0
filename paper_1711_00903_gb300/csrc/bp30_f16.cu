// BP3.0 with half-precision factors: the inner operator of the FP16-factor
// mixed-precision solver (FEM_PCG_MIXED16) for BP3.0 systems.  Factors in
// IEEE binary16 scaled by a power of two (see bp35_f16.cu), widened to FP32;
// FP32 data and arithmetic; the output multiplied by the inverse scale read
// from device memory.  The factors are 7 m^3 of the 2 n^3 + 7 m^3 values an
// element moves, so halving them cuts the operator's bytes by about 40 %.
#include "bp30_body.cuh"

namespace fem {
namespace {

template <int N, bool PCG>
__device__ __forceinline__ void f16g30_entry(int64_t E, const __half *__restrict__ G, const double *__restrict__ ginv,
                                             double lambda, const float *__restrict__ q, float *__restrict__ Aq,
                                             const float *__restrict__ z, float *__restrict__ p,
                                             const double *__restrict__ beta, double *__restrict__ partials) {
    using C = Bp30Cfg<N, float>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * C::EPB;
    const int nel = (int)((E - e0) < C::EPB ? (E - e0) : C::EPB);
    bp30_block<N, C::EPB, float, PCG, __half>(reinterpret_cast<float *>(smem_raw), e0, nel, G, lambda, q, Aq, z, p,
                                              beta, PCG ? partials + blockIdx.x : nullptr, ginv);
}

// The FP32 operator's register caps apply (bp30_min_blocks), except at
// N = 9, where six resident blocks per SM (40 registers) measured 7 % faster
// than the FP32 cap of four; the FP32 operator itself lost 6 % with six.
template <int N>
constexpr int bp30_f16_min_blocks() {
    return N == 9 ? 6 : bp30_min_blocks<float, N>();
}

template <int N, bool PCG>
__global__ void __launch_bounds__(Bp30Cfg<N, float>::threads)
bp30_f16g_kernel(int64_t E, const __half *__restrict__ G, const double *__restrict__ ginv, double lambda,
                 const float *__restrict__ q, float *__restrict__ Aq, const float *__restrict__ z,
                 float *__restrict__ p, const double *__restrict__ beta, double *__restrict__ partials) {
    f16g30_entry<N, PCG>(E, G, ginv, lambda, q, Aq, z, p, beta, partials);
}
template <int N, bool PCG>
__global__ void __launch_bounds__(Bp30Cfg<N, float>::threads, bp30_f16_min_blocks<N>())
bp30_f16g_kernel_capped(int64_t E, const __half *__restrict__ G, const double *__restrict__ ginv, double lambda,
                        const float *__restrict__ q, float *__restrict__ Aq, const float *__restrict__ z,
                        float *__restrict__ p, const double *__restrict__ beta, double *__restrict__ partials) {
    f16g30_entry<N, PCG>(E, G, ginv, lambda, q, Aq, z, p, beta, partials);
}
template <int N, bool PCG>
constexpr auto f16g30_fn() {
    if constexpr (bp30_f16_min_blocks<N>() > 0)
        return &bp30_f16g_kernel_capped<N, PCG>;
    else
        return &bp30_f16g_kernel<N, PCG>;
}

template <bool PCG>
struct F16Launch30 {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const __half *G, const double *ginv, double lambda, const float *q,
                               float *Aq, const float *z, float *p, const double *beta, double *partials,
                               cudaStream_t s, double *status) {
            if (bp30_stream_default(N, true, PCG))
                return launch_bp30_stream_f16g(N, PCG, E, G, ginv, lambda, q, Aq, z, p, beta, partials, s, status);
            using C = Bp30Cfg<N, float>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            f16g30_fn<N, PCG>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, ginv, lambda, q, Aq, z, p, beta,
                                                                             partials);
            return cudaGetLastError();
        }
    };
};

template <int N>
struct F16Prepare30 {
    static cudaError_t run() {
        cudaError_t e = cudaFuncSetAttribute(f16g30_fn<N, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Bp30Cfg<N, float>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f16g30_fn<N, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Bp30Cfg<N, float>::smem);
        return e;
    }
};

template <int N>
struct F16Blocks30 {
    static cudaError_t run(int64_t E, int64_t *out) {
        *out = bp30_stream_default(N, true, true) ? bp30_stream_grid(N, E, true)
                                            : (E + Bp30Cfg<N, float>::EPB - 1) / Bp30Cfg<N, float>::EPB;
        return cudaSuccess;
    }
};

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp30_f16_tu)

}  // namespace

cudaError_t launch_bp30_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                             const float *q, float *Aq, cudaStream_t s) {
    return dispatch_degree<F16Launch30<false>::L>(b->host.N, E, G, ginv, lambda, q, Aq, (const float *)nullptr,
                                                  (float *)nullptr, (const double *)nullptr, (double *)nullptr, s,
                                                  (double *)nullptr);
}

cudaError_t launch_bp30_pcg_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                                 const float *z, float *p, const double *beta, float *Ap, double *partials,
                                 cudaStream_t s, double *status) {
    return dispatch_degree<F16Launch30<true>::L>(b->host.N, E, G, ginv, lambda, (const float *)nullptr, Ap, z, p,
                                                 beta, partials, s, status);
}

int64_t bp30_f16_blocks(int N, int64_t E) {
    int64_t out = 0;
    dispatch_degree<F16Blocks30>(N, E, &out);
    return out;
}

cudaError_t prepare_bp30_f16(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp30_f16_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<F16Prepare30>(N);
}

}  // namespace fem
