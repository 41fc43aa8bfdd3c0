// BP1.0 mass matvec, IEEE FP64 (Algorithm 3):
//   Mq = (I^T x I^T x I^T) wJ (I x I x I) q   per element,
// interpolation GLL -> Gauss (Algorithm 1) and projection back (Algorithm 2)
// as three one-dimensional contractions each.
//
// GB300 design.  The kernel is bound by FP64 instruction issue (FP64 runs at
// about 1/64 of the FP32 rate on this part), so it keeps the FP64 work at
// the sum-factorised count 2(m n^3 + m^2 n^2 + m^3 n) + m^3 per element and
// uses shared memory and registers to remove everything else:
//   * an m x m slab of threads per element (the 2D thread structure of
//     Section 6), several elements per block;
//   * the whole q^e in shared memory, so the six contractions need only
//     three barriers (the fewest-barriers idea of Section 6, kernel 7);
//   * the s-interpolation, t-interpolation, wJ scaling and t-projection of a
//     thread's (a, b) column are fused in registers;
//   * coalesced global loads of q and wJ and coalesced stores.
#include "kernels_common.cuh"

namespace fem {
namespace {

template <int n>
struct Bp1Cfg {
    static constexpr int m = n + 1;
    static constexpr int NP = n * n * n, MP = m * m * m;
    static constexpr int B0 = pad2(n * m * m);  // q (n^3), then the t-projected field (n m^2)
    static constexpr int B1 = pad2(n * n * m);  // r-interpolated, then s-projected field
    static constexpr int smem_elem = (B0 + B1) * 8;
    static constexpr int EPB = pick_epb(m, smem_elem);
    static constexpr int threads = m * m * EPB;
    static constexpr int smem = (pad2(m * n) + EPB * (B0 + B1)) * 8;
};

template <int n>
__global__ void __launch_bounds__(Bp1Cfg<n>::threads)
bp1_f64_kernel(int64_t E, const double *__restrict__ ops, const double *__restrict__ wJ,
               const double *__restrict__ q, double *__restrict__ Mq) {
    using C = Bp1Cfg<n>;
    constexpr int m = C::m, NP = C::NP, MP = C::MP, EPB = C::EPB, mm = m * m;
    extern __shared__ double smem[];
    double *sI = smem;  // I[a][i] at a*n + i
    double *buf = sI + pad2(m * n);
    const OpsLayout L{n, m};
    block_copy(sI, ops + L.offI(), m * n);

    // stage q of the block's elements (contiguous in memory) into shared
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int64_t nel = (E - e0) < EPB ? (E - e0) : EPB;
    for (int t = threadIdx.x; t < EPB * NP; t += blockDim.x) {
        const int el = t / NP, p = t % NP;
        buf[el * (C::B0 + C::B1) + p] = (el < nel) ? __ldg(q + (e0 + el) * NP + p) : 0.0;
    }

    const int el = threadIdx.x / mm, ab = threadIdx.x % mm;
    const int a = ab % m, b = ab / m;
    const int64_t e = e0 + el;
    const bool valid = el < nel;
    double *b0 = buf + el * (C::B0 + C::B1);  // q [k][j][i], later u [k][b][a]
    double *b1 = b0 + C::B0;                  // t1 [k][j][a], later v [k][j][a]
    __syncthreads();

    // r-interpolation: t1[k][j][a] = sum_i I[a][i] q[k][j][i]  (threads with b < n act as j)
    if (b < n) {
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < n; i++) s = fma(sI[a * n + i], b0[i + n * (b + n * k)], s);
            b1[a + m * (b + n * k)] = s;
        }
    }
    __syncthreads();

    // s- and t-interpolation, scaling and t-projection of column (a, b)
    {
        double t2[n];
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int jj = 0; jj < n; jj++) s = fma(sI[b * n + jj], b1[a + m * (jj + n * k)], s);
            t2[k] = s;
        }
        const double *we = wJ + (valid ? e : 0) * MP + ab;
        double u[n];
#pragma unroll
        for (int k = 0; k < n; k++) u[k] = 0.0;
#pragma unroll
        for (int c = 0; c < m; c++) {
            double g = 0.0;
#pragma unroll
            for (int k = 0; k < n; k++) g = fma(sI[c * n + k], t2[k], g);
            g *= valid ? __ldg(we + c * mm) : 0.0;
#pragma unroll
            for (int k = 0; k < n; k++) u[k] = fma(sI[c * n + k], g, u[k]);
        }
        // b0 (q) was last read before the previous barrier
#pragma unroll
        for (int k = 0; k < n; k++) b0[ab + mm * k] = u[k];
    }
    __syncthreads();

    // s-projection: v[k][j][a] = sum_b I[b][j] u[k][b][a]
    if (b < n) {
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int bb = 0; bb < m; bb++) s = fma(sI[bb * n + b], b0[a + m * (bb + m * k)], s);
            b1[a + m * (b + n * k)] = s;
        }
    }
    __syncthreads();

    // r-projection: out[k][j][i] = sum_a I[a][i] v[k][j][a]
    if (a < n && b < n && valid) {
        double *oe = Mq + e * NP + a + n * b;
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int aa = 0; aa < m; aa++) s = fma(sI[aa * n + a], b1[aa + m * (b + n * k)], s);
            oe[n * n * k] = s;
        }
    }
}

template <int N>
struct Bp1Launch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *wJ, const double *q,
                           double *Mq, cudaStream_t s) {
        using C = Bp1Cfg<N + 1>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp1_f64_kernel<N + 1><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, b->d_ops, wJ, q, Mq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp1Prepare {
    static cudaError_t run() {
        using C = Bp1Cfg<N + 1>;
        return cudaFuncSetAttribute(bp1_f64_kernel<N + 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    C::smem);
    }
};

}  // namespace

cudaError_t launch_bp1(const fem_basis *b, int64_t E, const double *wJ, const double *q,
                       double *Mq, cudaStream_t s) {
    return dispatch_degree<Bp1Launch>(b->host.N, b, E, wJ, q, Mq, s);
}

cudaError_t prepare_bp1(int N) { return dispatch_degree<Bp1Prepare>(N); }

}  // namespace fem
