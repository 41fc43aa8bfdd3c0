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
// FP32 at degree up to 9 (the mixed solver's hot kernel) runs as a
// persistent, double-buffered TMA stream instead (see bp35_stream_kernel),
// and above 9 as the stream kernel with one factor stage
// (bp35_stream1_kernel).
#include "bp35_stream.cuh"

namespace fem {
namespace {

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
        if constexpr (bp35_streamed<N, false, float>()) {
            return launch_stream35<N, false>(E, G, lambda, q, Aq, nullptr, nullptr, nullptr, nullptr, s);
        } else if constexpr (bp35_streamed1<N, false, float>()) {
            return launch_stream35_1<N, false>(E, G, lambda, q, Aq, nullptr, nullptr, nullptr, nullptr, s);
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
                               T *Ap, double *partials, cudaStream_t s, double *status) {
            if constexpr (sizeof(T) == 4 && bp35_streamed<N, true, float>()) {
                return launch_stream35<N, true>(E, G, lambda, nullptr, Ap, z, p, beta, partials, s, nullptr,
                                                status);
            } else if constexpr (sizeof(T) == 4 && bp35_streamed1<N, true, float>()) {
                return launch_stream35_1<N, true>(E, G, lambda, nullptr, Ap, z, p, beta, partials, s, nullptr,
                                                  status);
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
        if constexpr (bp35_streamed<N, true, float>()) {
            using S = Bp35Stream<N, true>;
            b = stream_grid35((E + S::EPS - 1) / S::EPS, S::blocks_per_sm);
        } else if constexpr (bp35_streamed1<N, true, float>()) {
            b = stream_grid35(E, Bp35Stream1<N, true, float>::blocks_per_sm);
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
        if (e == cudaSuccess) e = one<float, false>();
        if (e == cudaSuccess) e = one<float, true>();
        // the stream kernels keep all operands in shared memory: they ask
        // for the largest carveout
        if constexpr (bp35_two_stage_fits(N))
            if (e == cudaSuccess) e = prepare_stream35<N, float>();
        if (e == cudaSuccess) e = prepare_stream35_1<N, float>();
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
    return dispatch_degree<Bp35PcgLaunchT<double>::L>(b->host.N, E, G, lambda, z, p, beta, Ap, partials, s,
                                                       (double *)nullptr);
}

cudaError_t launch_bp35_pcg_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                float *p, const double *beta, float *Ap, double *partials, cudaStream_t s,
                                double *status) {
    return dispatch_degree<Bp35PcgLaunchT<float>::L>(b->host.N, E, G, lambda, z, p, beta, Ap, partials, s, status);
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

namespace {
// Layout check of degree N: the n^3 box of the FP32 stream kernels and of
// the FP64 and block kernels, each point mapped to a distinct word inside
// the box's share of the per-element buffer; the swizzled boxes (N = 7,
// 15) also serve every direction's warp line accesses without a bank
// conflict.
template <int N>
int bp35_layout_violations_of() {
    constexpr int n = N + 1;
    using T = typename Bp35Layout<float, N, 1, true>::B;
    using P = typename Bp35Layout<double, N, 1>::B;
    int bad = box_layout_violations<T, n, n, n>(T::size) + box_layout_violations<P, n, n, n>(P::size);
    if constexpr (N == 7 || N == 15) bad += box_line_conflicts<T, n>();
    return bad;
}
template <int... Ns>
int bp35_layout_violations_all(std::integer_sequence<int, Ns...>) {
    return (0 + ... + bp35_layout_violations_of<Ns + 1>());
}
}  // namespace

int layout_violations_bp35() { return bp35_layout_violations_all(std::make_integer_sequence<int, kMaxN>{}); }

}  // namespace fem
