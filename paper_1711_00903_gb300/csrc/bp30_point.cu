// BP3.0 and BP3.5 in the point-per-thread ("3D") layouts of bp30_point.cuh
// and bp35_point.cuh as stand-alone kernels: one element per block, one
// thread per quadrature point or node (up to 1024; above that each thread
// takes several).
#include "bp30_point.cuh"
#include "bp35_point.cuh"

namespace fem {
namespace {

// Point-per-thread layout (bp30_point.cuh): one element per block.
template <int N>
__global__ void __launch_bounds__(Bp30Point<N>::threads)
bp30_point_kernel(int64_t E, const double *__restrict__ ops, const double *__restrict__ G, double lambda,
                  const double *__restrict__ q, double *__restrict__ Aq) {
    extern __shared__ __align__(16) double psm[];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        bp30_point_block<N, Bp30Point<N>::threads>(psm, ops, e, G, lambda, q, Aq);
        __syncthreads();
    }
}

template <int N>
struct Bp30PointLaunch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                           double *Aq, cudaStream_t s) {
        using P = Bp30Point<N>;
        const int64_t grid = E < (int64_t)1 << 30 ? E : (int64_t)1 << 30;
        bp30_point_kernel<N><<<(unsigned)grid, P::threads, P::smem, s>>>(E, b->d_ops, G, lambda, q, Aq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp30PointPrepare {
    static cudaError_t run() {
        return cudaFuncSetAttribute(bp30_point_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Bp30Point<N>::smem);
    }
};

template <int N>
__global__ void __launch_bounds__(Bp35Point<N>::threads)
bp35_point_kernel(int64_t E, const double *__restrict__ ops, const double *__restrict__ G, double lambda,
                  const double *__restrict__ q, double *__restrict__ Aq) {
    extern __shared__ __align__(16) double psm35[];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        bp35_point_block<N, Bp35Point<N>::threads>(psm35, ops, e, G, lambda, q, Aq);
        __syncthreads();
    }
}

template <int N>
struct Bp35PointLaunch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                           double *Aq, cudaStream_t s) {
        using P = Bp35Point<N>;
        const int64_t grid = E < (int64_t)1 << 30 ? E : (int64_t)1 << 30;
        bp35_point_kernel<N><<<(unsigned)grid, P::threads, P::smem, s>>>(E, b->d_ops, G, lambda, q, Aq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp35PointPrepare {
    static cudaError_t run() {
        return cudaFuncSetAttribute(bp35_point_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Bp35Point<N>::smem);
    }
};

}  // namespace

cudaError_t launch_bp35_point(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                              double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp35PointLaunch>(b->host.N, b, E, G, lambda, q, Aq, s);
}

cudaError_t launch_bp30_point(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                              double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp30PointLaunch>(b->host.N, b, E, G, lambda, q, Aq, s);
}

cudaError_t prepare_bp30_point(int N) {
    cudaError_t e = dispatch_degree<Bp30PointPrepare>(N);
    if (e == cudaSuccess) e = dispatch_degree<Bp35PointPrepare>(N);
    return e;
}

}  // namespace fem
