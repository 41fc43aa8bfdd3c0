// BP3.5 with one thread per GLL node: the three-dimensional thread layout
// of the paper's Section 6 (Algorithm 7: per node, the three derivatives of
// q from the element's field in shared memory, the symmetric factor
// product, then the transposed derivatives), kept as a variant of the
// two-dimensional line layout of bp35_body.cuh and as a candidate of the
// batch autotuner.
//
// One element per block; each thread owns the nodes t, t + blockDim, ...:
//   1. q (n^3) and D (n x n)                          -> A, shared
//   2. per node: qr, qs, qt (three contractions of length n read from A),
//      [Rr Rs Rt] = G [qr qs qt] with the six factors  -> B, C, D
//      and lambda wJ q kept per thread
//   3. per node: Aq = Dr^T Rr + Ds^T Rs + Dt^T Rt + lambda wJ q
// Two barriers and no even-odd folding (the operator rows differ between
// the threads of a warp, so they are read from shared memory).
#pragma once

#include "kernels_common.cuh"

namespace fem {
namespace {

template <int N>
struct Bp35Point {
    static constexpr int n = N + 1, NP = n * n * n;
    static constexpr int oD = 0;              // D (n x n), row = node, derivative of basis l
    static constexpr int oA = pad2(n * n);    // four n^3 boxes
    static constexpr int oB = oA + NP, oC = oB + NP, oE = oC + NP;
    static constexpr int doubles = oE + NP;
    static constexpr int smem = doubles * 8;
    static constexpr int threads = NP < 1024 ? ((NP + 31) / 32) * 32 : 1024;
};

// BP3.5 of element e by the whole block (blockDim.x == THREADS), shared
// memory sm (Bp35Point<N>::doubles).  ops: the basis table (D at
// OpsLayout::offD(), n x n, row-major: D[i][l] = l_l'(r_i)).
template <int N, int THREADS>
__device__ __forceinline__ void bp35_point_block(double *sm, const double *__restrict__ ops, int64_t e,
                                                 const double *__restrict__ G, double lambda,
                                                 const double *__restrict__ q, double *__restrict__ Aq) {
    using P = Bp35Point<N>;
    constexpr int n = P::n, NP = P::NP, nn = n * n;
    constexpr int PPT = (NP + THREADS - 1) / THREADS;
    const int tid = threadIdx.x, bd = blockDim.x;
    double *sD = sm + P::oD, *A = sm + P::oA, *B = sm + P::oB, *Cb = sm + P::oC, *Db = sm + P::oE;
    const OpsLayout L{n, n + 1};
    for (int t = tid; t < nn; t += bd) sD[t] = __ldg(ops + L.offD() + t);
    for (int t = tid; t < NP; t += bd) A[t] = __ldg(q + e * NP + t);
    __syncthreads();

    double mass[PPT];
    const double *Ge = G + e * 7 * NP;
#pragma unroll
    for (int j = 0; j < PPT; j++) {
        const int t = tid + j * bd;
        if (t < NP) {
            const int i = t % n, jj = (t / n) % n, k = t / nn;
            double qr = 0.0, qs = 0.0, qt = 0.0;
#pragma unroll
            for (int l = 0; l < n; l++) {
                qr = fma(sD[i * n + l], A[l + n * jj + nn * k], qr);
                qs = fma(sD[jj * n + l], A[i + n * l + nn * k], qs);
                qt = fma(sD[k * n + l], A[i + n * jj + nn * l], qt);
            }
            double g[7];
#pragma unroll
            for (int h = 0; h < 7; h++) g[h] = __ldg(Ge + h * NP + t);
            B[t] = g[0] * qr + g[1] * qs + g[2] * qt;
            Cb[t] = g[1] * qr + g[3] * qs + g[4] * qt;
            Db[t] = g[2] * qr + g[4] * qs + g[5] * qt;
            mass[j] = (lambda != 0.0) ? (lambda * g[6]) * A[t] : 0.0;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PPT; j++) {
        const int t = tid + j * bd;
        if (t < NP) {
            const int i = t % n, jj = (t / n) % n, k = t / nn;
            double w = mass[j];
#pragma unroll
            for (int l = 0; l < n; l++) {
                w = fma(sD[l * n + i], B[l + n * jj + nn * k], w);
                w = fma(sD[l * n + jj], Cb[i + n * l + nn * k], w);
                w = fma(sD[l * n + k], Db[i + n * jj + nn * l], w);
            }
            Aq[e * NP + t] = w;
        }
    }
}

}  // namespace
}  // namespace fem
