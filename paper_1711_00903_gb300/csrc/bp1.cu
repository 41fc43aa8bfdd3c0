// BP1.0 mass matvec, IEEE FP64 (Algorithm 3):
//   Mq = (I^T x I^T x I^T) wJ (I x I x I) q   per element,
// interpolation GLL -> Gauss (Algorithm 1) and projection back (Algorithm 2)
// as three one-dimensional contractions each.
//
// GB300 design.  Bound by FP64 instruction issue (2 per clock per SM on this
// part), so every one-dimensional contraction is one thread applying the
// even-odd folded I or I^T (both centro-symmetric, the property the paper's
// Section 6 kernel 8 exploits for shared-memory loads) to a whole line, with
// the operator entries as constant-bank operands (eo.cuh):
//   1. r-interpolation lines (j, k)          q box    -> X1 (m x n x n)
//   2. s-interpolation lines (a, k)          X1       -> X2 (m x m x n)
//   3. per column (a, b): t-interpolation, wJ scaling and t-projection in
//      registers, back into X2 in place
//   4. s-projection lines (a, k)             X2       -> X4 (m x n x n)
//   5. r-projection lines (j, k)             X4       -> Mq (global)
// Five barriers; tasks are packed densely onto the block's threads.
#include "eo.cuh"

namespace fem {
namespace {

// TARGET: the block's thread target (256; 32 for meshes too small to give
// every SM two blocks, where one element per block spreads the work)
template <int N, int TARGET = 256>
struct Bp1Cfg {
    static constexpr int n = N + 1, m = N + 2;
    static constexpr int NP = n * n * n, MP = m * m * m;
    using B0 = Box<n, n, n>;  // q
    using B1 = Box<m, n, n>;  // r-interpolated / s-projected
    using B2 = Box<m, m, n>;  // s-interpolated / t-projected
    static constexpr int SA = (B0::size > B2::size) ? B0::size : B2::size;
    static constexpr int SB = B1::size;
    static constexpr int per = SA + SB;
    static constexpr int EPB = pick_epb(m, per * 8, TARGET);
    static constexpr int threads = ((m * m * EPB + 31) / 32) * 32;
    static constexpr int smem = EPB * per * 8;
    static constexpr int oI = fold_offset(N, kFoldI), oIT = fold_offset(N, kFoldIT);
    // three resident blocks per SM let one block's barriers overlap the
    // others' FP64 work; the register cap this implies costs a few spills
    // at high degree but was measured faster at every degree
    static constexpr int min_blocks = 3;
};

template <int N, int TARGET>
__global__ void __launch_bounds__(Bp1Cfg<N, TARGET>::threads, Bp1Cfg<N, TARGET>::min_blocks)
bp1_f64_kernel(int64_t E, const double *__restrict__ wJ, const double *__restrict__ q, double *__restrict__ Mq) {
    using C = Bp1Cfg<N, TARGET>;
    using B0 = typename C::B0;
    using B1 = typename C::B1;
    using B2 = typename C::B2;
    constexpr int n = C::n, m = C::m, NP = C::NP, MP = C::MP, EPB = C::EPB, per = C::per;
    extern __shared__ double smem[];

    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
        const int el = t / NP, p = t - el * NP;
        smem[el * per + B0::at(p % n, (p / n) % n, p / (n * n))] = __ldg(q + e0 * NP + t);
    }
    __syncthreads();

    // 1. r-interpolation: lines (j, k), n -> m
    for_tasks<n * n, EPB>(nel, [&](int el, int r) {
        const int j = r % n, k = r / n;
        const double *X0 = smem + el * per;
        double *X1 = smem + el * per + C::SA;
        double x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = X0[B0::at(l, j, k)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) X1[B1::at(l, j, k)] = y[l];
    });
    __syncthreads();

    // 2. s-interpolation: lines (a, k), n -> m
    for_tasks<m * n, EPB>(nel, [&](int el, int r) {
        const int a = r % m, k = r / m;
        const double *X1 = smem + el * per + C::SA;
        double *X2 = smem + el * per;
        double x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = X1[B1::at(a, l, k)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) X2[B2::at(a, l, k)] = y[l];
    });
    __syncthreads();

    // 3. column (a, b): t-interpolation, scaling by wJ, t-projection
    for_tasks<m * m, EPB>(nel, [&](int el, int r) {
        const int a = r % m, b = r / m;
        double *X2 = smem + el * per;
        const double *we = wJ + (e0 + el) * MP + r;
        double x[n], g[m], y[n];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = X2[B2::at(a, b, l)];
        eo_apply<m, n, 1, C::oI>(x, g);
#pragma unroll
        for (int c = 0; c < m; c++) g[c] = mul_rn(g[c], __ldg(we + c * m * m));
        eo_apply<n, m, 1, C::oIT>(g, y);
#pragma unroll
        for (int l = 0; l < n; l++) X2[B2::at(a, b, l)] = y[l];
    });
    __syncthreads();

    // 4. s-projection: lines (a, k), m -> n
    for_tasks<m * n, EPB>(nel, [&](int el, int r) {
        const int a = r % m, k = r / m;
        const double *X2 = smem + el * per;
        double *X4 = smem + el * per + C::SA;
        double x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = X2[B2::at(a, l, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) X4[B1::at(a, l, k)] = y[l];
    });
    __syncthreads();

    // 5. r-projection: lines (j, k), m -> n, to global
    for_tasks<n * n, EPB>(nel, [&](int el, int r) {
        const int j = r % n, k = r / n;
        const double *X4 = smem + el * per + C::SA;
        double x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = X4[B1::at(l, j, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
        double *o = Mq + (e0 + el) * NP + r * n;
#pragma unroll
        for (int l = 0; l < n; l++) o[l] = y[l];
    });
}

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp1_tu)

template <int N>
struct Bp1Launch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *wJ, const double *q, double *Mq,
                           cudaStream_t s) {
        using C = Bp1Cfg<N>;
        using Cs = Bp1Cfg<N, 32>;
        (void)b;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        if (blocks < 2 * 152) {  // small mesh: one element (or a few) per block
            bp1_f64_kernel<N, 32><<<(unsigned)((E + Cs::EPB - 1) / Cs::EPB), Cs::threads, Cs::smem, s>>>(E, wJ, q,
                                                                                                      Mq);
            return cudaGetLastError();
        }
        bp1_f64_kernel<N, 256><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, wJ, q, Mq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp1Prepare {
    static cudaError_t run() {
        cudaError_t e = cudaFuncSetAttribute(bp1_f64_kernel<N, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Bp1Cfg<N>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp1_f64_kernel<N, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Bp1Cfg<N, 32>::smem);
        return e;
    }
};

}  // namespace

cudaError_t launch_bp1(const fem_basis *b, int64_t E, const double *wJ, const double *q, double *Mq,
                       cudaStream_t s) {
    return dispatch_degree<Bp1Launch>(b->host.N, b, E, wJ, q, Mq, s);
}

cudaError_t prepare_bp1(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp1_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<Bp1Prepare>(N);
}

}  // namespace fem
