// BP3.5 collocated screened-Poisson matvec, IEEE FP64 (Algorithm 4):
//   Aq = D_r^T Rr + D_s^T Rs + D_t^T Rt + lambda wJ q,
//   [Rr Rs Rt] = G [q_r q_s q_t],  q_r = (D x I x I) q, ...
//
// GB300 design.  FP64 arithmetic runs at about 1/64 of the FP32 rate on
// this part (a measured 1.0 TFLOP/s), so the kernel is bound by its FP64
// instruction count, not by HBM or shared-memory bandwidth.  The layout
// therefore spends registers and shared memory freely and keeps the FP64
// work at the sum-factorised minimum of 6n + 11 operations per node:
//   * one thread per (i, j) column of an element, looping over the k slabs
//     (the 2D thread structure of Section 6), several elements per block;
//   * q^e staged once in shared memory and the thread's own column in
//     registers, so the t-derivative and the t-transpose (a scatter into the
//     thread's register column) touch no shared memory;
//   * the r and s partial fluxes Rr, Rs kept for the whole element in shared
//     memory, so one barrier separates the two passes (the fewest-barriers
//     idea of Section 6, kernel 7, and Section 7, kernel 10);
//   * every global access is coalesced across the n*n threads of a slab.
#include "kernels_common.cuh"

namespace fem {
namespace {

template <int n>
struct Bp35Cfg {
    static constexpr int NP = n * n * n;
    static constexpr int smem_elem = 3 * NP * 8;
    static constexpr int EPB = pick_epb(n, smem_elem);
    static constexpr int threads = n * n * EPB;
    static constexpr int smem = (pad2(n * n) + 3 * EPB * NP) * 8;
};

template <int n>
__global__ void __launch_bounds__(Bp35Cfg<n>::threads)
bp35_f64_kernel(int64_t E, const double *__restrict__ ops, const double *__restrict__ G,
                double lambda, const double *__restrict__ q, double *__restrict__ Aq) {
    using C = Bp35Cfg<n>;
    constexpr int NP = C::NP, EPB = C::EPB, nn = n * n;
    extern __shared__ double smem[];
    double *sD = smem;                   // D[a][l] at a*n + l
    double *sq = sD + pad2(nn);          // EPB elements of q, [k][j][i]
    double *sRr = sq + EPB * NP;         // partial flux along r
    double *sRs = sRr + EPB * NP;        // partial flux along s

    const OpsLayout L{n, n + 1};
    block_copy(sD, ops + L.offD(), nn);

    const int el = threadIdx.x / nn, ij = threadIdx.x % nn;
    const int i = ij % n, j = ij / n;
    const int64_t e = (int64_t)blockIdx.x * EPB + el;
    const bool valid = e < E;
    double *eq = sq + el * NP, *eRr = sRr + el * NP, *eRs = sRs + el * NP;

    double qc[n], acc[n];
    const double *qe = q + (valid ? e : 0) * NP + ij;
#pragma unroll
    for (int k = 0; k < n; k++) {
        qc[k] = valid ? __ldg(qe + k * nn) : 0.0;
        eq[k * nn + ij] = qc[k];
        acc[k] = 0.0;
    }
    __syncthreads();

    const double *Ge = G + (valid ? e : 0) * 7 * NP + ij;
#pragma unroll
    for (int k = 0; k < n; k++) {
        const double *qk = eq + k * nn;
        double qr = 0.0, qs = 0.0, qt = 0.0;
#pragma unroll
        for (int l = 0; l < n; l++) {
            qr = fma(sD[i * n + l], qk[j * n + l], qr);
            qs = fma(sD[j * n + l], qk[l * n + i], qs);
            qt = fma(sD[k * n + l], qc[l], qt);
        }
        double g[7];
#pragma unroll
        for (int c = 0; c < 7; c++) g[c] = valid ? __ldg(Ge + c * NP + k * nn) : 0.0;
        const double Rr = g[0] * qr + g[1] * qs + g[2] * qt;
        const double Rs = g[1] * qr + g[3] * qs + g[4] * qt;
        const double Rt = g[2] * qr + g[4] * qs + g[5] * qt;
        eRr[k * nn + ij] = Rr;
        eRs[k * nn + ij] = Rs;
        // t-direction transpose: acc[l] += D[k][l] * Rt
#pragma unroll
        for (int l = 0; l < n; l++) acc[l] = fma(sD[k * n + l], Rt, acc[l]);
        if (lambda != 0.0) acc[k] = fma(lambda * g[6], qc[k], acc[k]);
    }
    __syncthreads();

    double *Ae = Aq + (valid ? e : 0) * NP + ij;
#pragma unroll
    for (int k = 0; k < n; k++) {
        const double *Rrk = eRr + k * nn, *Rsk = eRs + k * nn;
        double s = acc[k];
#pragma unroll
        for (int l = 0; l < n; l++) {
            s = fma(sD[l * n + i], Rrk[j * n + l], s);
            s = fma(sD[l * n + j], Rsk[l * n + i], s);
        }
        if (valid) Ae[k * nn] = s;
    }
}

template <int N>
struct Bp35Launch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda,
                           const double *q, double *Aq, cudaStream_t s) {
        using C = Bp35Cfg<N + 1>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp35_f64_kernel<N + 1><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, b->d_ops, G, lambda, q, Aq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp35Prepare {
    static cudaError_t run() {
        using C = Bp35Cfg<N + 1>;
        return cudaFuncSetAttribute(bp35_f64_kernel<N + 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    C::smem);
    }
};

}  // namespace

cudaError_t launch_bp35(const fem_basis *b, int64_t E, const double *G, double lambda,
                        const double *q, double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp35Launch>(b->host.N, b, E, G, lambda, q, Aq, s);
}

cudaError_t prepare_bp35(int N) { return dispatch_degree<Bp35Prepare>(N); }

}  // namespace fem
