// BP3.0 dealiased screened-Poisson matvec, IEEE FP64 (Algorithm 5):
//   Aq = (I^T x I^T x I^T) [ Dt_r^T Rr + Dt_s^T Rs + Dt_t^T Rt + lambda wJ qg ],
//   qg = (I x I x I) q,  [Rr Rs Rt] = G [Dt_r qg, Dt_s qg, Dt_t qg],
// twelve one-dimensional contractions per element in one kernel with no
// global intermediates (Section 8: a three-kernel split was no faster, and
// removing global intermediates was the largest gain).
//
// GB300 design.  Bound by FP64 instruction issue (2 per clock per SM), so
// every contraction is one thread applying an even-odd folded operator to
// a whole line with constant-bank operands (eo.cuh), and the element lives
// in three m^3 shared-memory boxes:
//   1. r-interpolation lines (j, k)               q      -> X1
//   2. s-interpolation lines (a, k)               X1     -> X2
//   3. t-interpolation columns (a, b)             X2     -> QG (m^3)
//   4. r- and s-derivative lines                  QG     -> UR, US
//   5. per column (a, b): t-derivative, chain rule with the 7 factors,
//      t-transpose and the lambda wJ qg term, in registers (kept to step 7)
//   6. r- and s-transpose lines, in place          UR, US
//   7. per column: sum, t-projection               -> X3 (m x m x n)
//   8. s-projection lines (a, k)                  X3     -> X4 (m x n x n)
//   9. r-projection lines (j, k)                  X4     -> Aq (global)
#include "bp30_body.cuh"

namespace fem {
namespace {

template <typename T, int N, bool PCG>
__device__ __forceinline__ void bp30_entry(int64_t E, const T *__restrict__ G, double lambda, const T *__restrict__ q,
                                           T *__restrict__ Aq, const T *__restrict__ z, T *__restrict__ p,
                                           const double *__restrict__ beta, double *__restrict__ partials) {
    using C = Bp30Cfg<N, T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t e0 = (int64_t)blockIdx.x * C::EPB;
    const int nel = (int)((E - e0) < C::EPB ? (E - e0) : C::EPB);
    bp30_block<N, C::EPB, T, PCG>(reinterpret_cast<T *>(smem_raw), e0, nel, G, lambda, q, Aq, z, p, beta,
                                  PCG ? partials + blockIdx.x : nullptr);
}

template <typename T, int N, bool PCG>
__global__ void __launch_bounds__(Bp30Cfg<N, T>::threads)
bp30_kernel(int64_t E, const T *__restrict__ G, double lambda, const T *__restrict__ q, T *__restrict__ Aq,
            const T *__restrict__ z, T *__restrict__ p, const double *__restrict__ beta,
            double *__restrict__ partials) {
    bp30_entry<T, N, PCG>(E, G, lambda, q, Aq, z, p, beta, partials);
}

template <typename T, int N, bool PCG>
__global__ void __launch_bounds__(Bp30Cfg<N, T>::threads, bp30_min_blocks<T, N>())
bp30_kernel_capped(int64_t E, const T *__restrict__ G, double lambda, const T *__restrict__ q, T *__restrict__ Aq,
                   const T *__restrict__ z, T *__restrict__ p, const double *__restrict__ beta,
                   double *__restrict__ partials) {
    bp30_entry<T, N, PCG>(E, G, lambda, q, Aq, z, p, beta, partials);
}

template <typename T, int N, bool PCG>
constexpr auto bp30_fn() {
    if constexpr (bp30_min_blocks<T, N>() > 0)
        return &bp30_kernel_capped<T, N, PCG>;
    else
        return &bp30_kernel<T, N, PCG>;
}

// BP1.0 and BP3.0 of one field in one pass (bp30_core with MASS): the
// interpolation to the Gauss points is done once for both, and BP1.0's wJ is
// the seventh BP3.0 factor.  Mq and Aq are bit for bit the outputs of the
// separate BP1.0 (with that wJ) and BP3.0 kernels.
template <int N>
struct Bp1Bp30Cfg
    : Bp30Layout<N, pick_epb(N + 2, 4 * Box<N + 2, N + 2, N + 2>::size * 8, 256), double, 4> {};

template <int N>
__device__ __forceinline__ void bp1_bp30_entry(int64_t E, const double *__restrict__ G, double lambda,
                                               const double *__restrict__ q, double *__restrict__ Mq,
                                               double *__restrict__ Aq) {
    using C = Bp1Bp30Cfg<N>;
    using B0 = typename C::B0;
    constexpr int n = C::n, NP = C::NP, MP = C::MP, S = C::S, per = C::per, EPB = C::EPB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *smem = reinterpret_cast<double *>(smem_raw);
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
        const int el = t / NP, s = t - el * NP;
        smem[el * per + S + B0::at(s % n, (s / n) % n, s / (n * n))] = __ldg(q + e0 * NP + t);
    }
    __syncthreads();
    bp30_core<N, EPB, double, false, false, double, true>(smem, e0, nel, G + e0 * 7 * MP, lambda, Aq, nullptr, 1.0,
                                                           Mq);
}

template <int N>
__global__ void __launch_bounds__(Bp1Bp30Cfg<N>::threads)
bp1_bp30_kernel(int64_t E, const double *__restrict__ G, double lambda, const double *__restrict__ q,
                double *__restrict__ Mq, double *__restrict__ Aq) {
    bp1_bp30_entry<N>(E, G, lambda, q, Mq, Aq);
}

template <int N>
__global__ void __launch_bounds__(Bp1Bp30Cfg<N>::threads, bp30_min_blocks<double, N>())
bp1_bp30_kernel_capped(int64_t E, const double *__restrict__ G, double lambda, const double *__restrict__ q,
                       double *__restrict__ Mq, double *__restrict__ Aq) {
    bp1_bp30_entry<N>(E, G, lambda, q, Mq, Aq);
}

template <int N>
constexpr auto bp1_bp30_fn() {
    if constexpr (bp30_min_blocks<double, N>() > 0)
        return &bp1_bp30_kernel_capped<N>;
    else
        return &bp1_bp30_kernel<N>;
}

template <int N>
struct Bp1Bp30Launch {
    static cudaError_t run(int64_t E, const double *G, double lambda, const double *q, double *Mq, double *Aq,
                           cudaStream_t s) {
        using C = Bp1Bp30Cfg<N>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp1_bp30_fn<N>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, lambda, q, Mq, Aq);
        return cudaGetLastError();
    }
};

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp30_tu)

// kernel selection of the FP32 entry points: 0 the default for the degree,
// 1 the block kernel, 2 the stream kernel
template <typename T, bool PCG>
struct Bp30LaunchT {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const T *G, double lambda, const T *q, T *Aq, const T *z, T *p,
                               const double *beta, double *partials, cudaStream_t s, double *status = nullptr,
                               int which = 0) {
            if constexpr (sizeof(T) == 4) {
                if (which == 2 || (which == 0 && bp30_stream_default(N, false, PCG)))
                    return launch_bp30_stream(N, PCG, E, G, lambda, q, Aq, z, p, beta, partials, s, status);
            }
            using C = Bp30Cfg<N, T>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            bp30_fn<T, N, PCG>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, lambda, q, Aq, z, p, beta,
                                                                              partials);
            return cudaGetLastError();
        }
    };
};

template <int N>
struct Bp30Blocks {
    static cudaError_t run(int64_t E, bool f32, int64_t *out) {
        const int epb = f32 ? Bp30Cfg<N, float>::EPB : Bp30Cfg<N, double>::EPB;
        *out = (E + epb - 1) / epb;
        if (f32 && bp30_stream_default(N, false, true)) *out = bp30_stream_grid(N, E);
        return cudaSuccess;
    }
};

template <int N>
struct Bp30Prepare {
    template <typename T, bool PCG>
    static cudaError_t one() {
        return cudaFuncSetAttribute(bp30_fn<T, N, PCG>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Bp30Cfg<N, T>::smem);
    }
    static cudaError_t run() {
        cudaError_t e = one<double, false>();
        if (e == cudaSuccess) e = one<double, true>();
        if (e == cudaSuccess) e = one<float, false>();
        if (e == cudaSuccess) e = one<float, true>();
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp1_bp30_fn<N>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Bp1Bp30Cfg<N>::smem);
        return e;
    }
};

}  // namespace

cudaError_t launch_bp30(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                        double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp30LaunchT<double, false>::L>(b->host.N, E, G, lambda, q, Aq, (const double *)nullptr,
                                                           (double *)nullptr, (const double *)nullptr,
                                                           (double *)nullptr, s);
}

cudaError_t launch_bp30_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q,
                            float *Aq, cudaStream_t s, int which) {
    return dispatch_degree<Bp30LaunchT<float, false>::L>(b->host.N, E, G, lambda, q, Aq, (const float *)nullptr,
                                                          (float *)nullptr, (const double *)nullptr,
                                                          (double *)nullptr, s, (double *)nullptr, which);
}

cudaError_t launch_bp30_pcg(const fem_basis *b, int64_t E, const double *G, double lambda, const double *z,
                            double *p, const double *beta, double *Ap, double *partials, cudaStream_t s) {
    return dispatch_degree<Bp30LaunchT<double, true>::L>(b->host.N, E, G, lambda, (const double *)nullptr, Ap, z, p,
                                                          beta, partials, s);
}

cudaError_t launch_bp30_pcg_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                float *p, const double *beta, float *Ap, double *partials, cudaStream_t s,
                                double *status) {
    return dispatch_degree<Bp30LaunchT<float, true>::L>(b->host.N, E, G, lambda, (const float *)nullptr, Ap, z, p,
                                                         beta, partials, s, status, 0);
}

cudaError_t launch_bp1_bp30(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                            double *Mq, double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp1Bp30Launch>(b->host.N, E, G, lambda, q, Mq, Aq, s);
}

int64_t bp30_blocks(int N, int64_t E, bool f32) {
    int64_t out = 0;
    dispatch_degree<Bp30Blocks>(N, E, f32, &out);
    return out;
}

cudaError_t prepare_bp30(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp30_tu(fold_table);
    if (e == cudaSuccess) e = dispatch_degree<Bp30Prepare>(N);
    if (e == cudaSuccess) e = prepare_bp30_stream(N, fold_table);
    return e;
}

namespace {
// Layout check of degree N: the four FP32 boxes (the stream and block
// kernels' layout) and the four FP64 boxes, each point of each box mapped
// to a distinct word inside the per-element buffer.
template <int N>
int bp30_layout_violations_of() {
    constexpr int n = N + 1, m = N + 2;
    using F = Bp30Layout<N, 1, float>;
    using D = Bp30Layout<N, 1, double>;
    return box_layout_violations<typename F::B0, n, n, n>(F::S) +
           box_layout_violations<typename F::B1, m, n, n>(F::S) +
           box_layout_violations<typename F::B2, m, m, n>(F::S) +
           box_layout_violations<typename F::B3, m, m, m>(F::S) +
           box_layout_violations<typename D::B0, n, n, n>(D::S) +
           box_layout_violations<typename D::B1, m, n, n>(D::S) +
           box_layout_violations<typename D::B2, m, m, n>(D::S) +
           box_layout_violations<typename D::B3, m, m, m>(D::S);
}
template <int... Ns>
int bp30_layout_violations_all(std::integer_sequence<int, Ns...>) {
    return (0 + ... + bp30_layout_violations_of<Ns + 1>());
}
}  // namespace

int layout_violations_bp30() { return bp30_layout_violations_all(std::make_integer_sequence<int, kMaxN>{}); }

}  // namespace fem
