// BP3.0 with one thread per quadrature point: the three-dimensional thread
// layout of the paper's Section 6 (its 3D kernels), kept as a variant to
// compare against the two-dimensional line layout of bp30_body.cuh.
//
// One element per block.  Each thread owns the points t, t + blockDim, ...
// of every phase, and every output is a full contraction of length n or m
// read from shared memory with the 1D operators I (m x n) and Dt (m x m)
// also in shared memory (the threads of a warp need different operator
// rows, so constant-bank operands would serialise):
//   1. q (n^3)                                  -> A
//   2. r-interpolation      X1 (m n n)          A -> B
//   3. s-interpolation      X2 (m m n)          B -> A
//   4. t-interpolation      QG (m^3)            A -> B
//   5. Gauss-point gradient, chain rule with the seven factors
//                           Rr, Rs, Rt          B -> A, C, D (mass term kept per thread)
//   6. transposed derivatives summed, plus lambda wJ qg
//                           W (m^3)             A, C, D -> B
//   7. t-projection         Y1 (m m n)          B -> A
//   8. s-projection         Y2 (m n n)          A -> C
//   9. r-projection         Aq (n^3)            C -> global
// Eight barriers and no even-odd folding: at N = 7 this executes about 1.4
// times the FP64 instructions of the line layout, the quantity that bounds
// FP64 on GB300, so the line layout is the default and this one is measured
// against it (the paper found its 3D kernels slower too, and limited them to
// N < 9 for lack of threads).
#pragma once

#include "kernels_common.cuh"

namespace fem {
namespace {

template <int N>
struct Bp30Point {
    static constexpr int n = N + 1, m = N + 2, NP = n * n * n, MP = m * m * m;
    static constexpr int oI = 0, oDt = m * n;                  // operators
    static constexpr int oA = pad2(m * n + m * m);             // four m^3 work boxes
    static constexpr int oB = oA + MP, oC = oB + MP, oD = oC + MP;
    static constexpr int doubles = oD + MP;
    static constexpr int smem = doubles * 8;
    // threads of the stand-alone kernel: one per point, up to 1024
    static constexpr int threads = MP < 1024 ? ((MP + 31) / 32) * 32 : 1024;
};

// BP3.0 of element e by the whole block (blockDim.x == THREADS), shared
// memory sm (Bp30Point<N>::doubles).
// ops: the basis table (I at offset 0, m x n; Dt at OpsLayout::offDt(),
// m x m; both row-major, row = Gauss point).
template <int N, int THREADS>
__device__ __forceinline__ void bp30_point_block(double *sm, const double *__restrict__ ops, int64_t e,
                                                 const double *__restrict__ G, double lambda,
                                                 const double *__restrict__ q, double *__restrict__ Aq) {
    using P = Bp30Point<N>;
    constexpr int n = P::n, m = P::m, NP = P::NP, MP = P::MP;
    constexpr int PPT = (MP + THREADS - 1) / THREADS;  // points per thread in the point phases
    const int tid = threadIdx.x, bd = blockDim.x;
    double *sI = sm + P::oI, *sDt = sm + P::oDt;
    double *A = sm + P::oA, *B = sm + P::oB, *Cb = sm + P::oC, *D = sm + P::oD;
    const OpsLayout L{n, m};
    for (int t = tid; t < m * n; t += bd) sI[t] = __ldg(ops + L.offI() + t);
    for (int t = tid; t < m * m; t += bd) sDt[t] = __ldg(ops + L.offDt() + t);
    for (int t = tid; t < NP; t += bd) A[t] = __ldg(q + e * NP + t);
    __syncthreads();

    // 2. X1[a, j, k] = sum_i I[a][i] q[i, j, k]
    for (int t = tid; t < m * n * n; t += bd) {
        const int a = t % m, jk = t / m;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < n; i++) s = fma(sI[a * n + i], A[i + n * jk], s);
        B[t] = s;
    }
    __syncthreads();
    // 3. X2[a, b, k] = sum_j I[b][j] X1[a, j, k]
    for (int t = tid; t < m * m * n; t += bd) {
        const int a = t % m, r = t / m, b = r % m, k = r / m;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < n; j++) s = fma(sI[b * n + j], B[a + m * (j + n * k)], s);
        A[t] = s;
    }
    __syncthreads();
    // 4. QG[a, b, c] = sum_k I[c][k] X2[a, b, k]
    for (int t = tid; t < MP; t += bd) {
        const int ab = t % (m * m), c = t / (m * m);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < n; k++) s = fma(sI[c * n + k], A[ab + m * m * k], s);
        B[t] = s;
    }
    __syncthreads();
    // 5. gradient at the Gauss point, chain rule with the factors
    double mass[PPT];
    const double *Ge = G + e * 7 * MP;
#pragma unroll
    for (int j = 0; j < PPT; j++) {
        const int t = tid + j * bd;
        if (t < MP) {
            const int a = t % m, b = (t / m) % m, c = t / (m * m);
            double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
            for (int l = 0; l < m; l++) {
                ur = fma(sDt[a * m + l], B[l + m * (b + m * c)], ur);
                us = fma(sDt[b * m + l], B[a + m * (l + m * c)], us);
                ut = fma(sDt[c * m + l], B[a + m * (b + m * l)], ut);
            }
            double g[7];
#pragma unroll
            for (int h = 0; h < 7; h++) g[h] = __ldg(Ge + h * MP + t);
            A[t] = g[0] * ur + g[1] * us + g[2] * ut;
            Cb[t] = g[1] * ur + g[3] * us + g[4] * ut;
            D[t] = g[2] * ur + g[4] * us + g[5] * ut;
            mass[j] = (lambda != 0.0) ? (lambda * g[6]) * B[t] : 0.0;
        }
    }
    __syncthreads();
    // 6. W = Dt_r^T Rr + Dt_s^T Rs + Dt_t^T Rt + lambda wJ qg
#pragma unroll
    for (int j = 0; j < PPT; j++) {
        const int t = tid + j * bd;
        if (t < MP) {
            const int a = t % m, b = (t / m) % m, c = t / (m * m);
            double w = mass[j];
#pragma unroll
            for (int l = 0; l < m; l++) {
                w = fma(sDt[l * m + a], A[l + m * (b + m * c)], w);
                w = fma(sDt[l * m + b], Cb[a + m * (l + m * c)], w);
                w = fma(sDt[l * m + c], D[a + m * (b + m * l)], w);
            }
            B[t] = w;
        }
    }
    __syncthreads();
    // 7. Y1[a, b, k] = sum_c I[c][k] W[a, b, c]
    for (int t = tid; t < m * m * n; t += bd) {
        const int ab = t % (m * m), k = t / (m * m);
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < m; c++) s = fma(sI[c * n + k], B[ab + m * m * c], s);
        A[t] = s;
    }
    __syncthreads();
    // 8. Y2[a, j, k] = sum_b I[b][j] Y1[a, b, k]
    for (int t = tid; t < m * n * n; t += bd) {
        const int a = t % m, r = t / m, jj = r % n, k = r / n;
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < m; b++) s = fma(sI[b * n + jj], A[a + m * (b + m * k)], s);
        Cb[t] = s;
    }
    __syncthreads();
    // 9. Aq[i, j, k] = sum_a I[a][i] Y2[a, j, k]
    for (int t = tid; t < NP; t += bd) {
        const int i = t % n, jk = t / n;
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < m; a++) s = fma(sI[a * n + i], Cb[a + m * jk], s);
        Aq[e * NP + t] = s;
    }
}

}  // namespace
}  // namespace fem
