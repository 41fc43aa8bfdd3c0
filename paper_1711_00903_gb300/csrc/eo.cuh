// Even-odd folded one-dimensional contractions and padded element boxes.
//
// Every 1D operator of the method is centro-symmetric (I and its transpose:
// A[P-1-a][Q-1-i] = A[a][i], Section 6 kernel 8 uses the same symmetry) or
// anti-centro-symmetric (D, Dt and their transposes: A[P-1-a][Q-1-i] =
// -A[a][i]).  With e_i = x_i + x_{Q-1-i} and o_i = x_i - x_{Q-1-i} (i < Q/2),
//   E_a = sum_i S[a][i] e_i (+ A[a][Q/2] x_mid),  O_a = sum_i T[a][i] o_i,
//   S = (A[a][i] + A[a][Q-1-i]) / 2,  T = (A[a][i] - A[a][Q-1-i]) / 2,
//   y_a = E_a + O_a,  y_{P-1-a} = sigma (E_a - O_a),
// and a middle output row (P odd) uses e (sigma = +1) or o (sigma = -1)
// only (Solomonoff 1992; Kopriva, "Implementing Spectral Methods for PDEs",
// 2009).  A line of Q inputs and P outputs then costs about P Q / 2 FMAs
// plus P + Q adds instead of P Q FMAs.  On GB300, where FP64 issues at
// 2 instructions per clock per SM, that is the quantity that bounds the
// FP64 operators.
//
// The folded matrices of every degree live in one __constant__ table; each
// kernel reads them at compile-time offsets, so every operator entry is a
// uniform constant-bank operand of the FMA (no load instruction).
#pragma once

#include "fold_layout.h"
#include "kernels_common.cuh"

namespace fem {

// ------------------------------------------------------------ device side

// One constant table per translation unit and precision (no relocatable
// device code); every TU that uses them uploads the same contents at basis
// setup.
static __constant__ double c_fold[kFoldTotal];
static __constant__ float c_fold32[kFoldTotal];

template <typename T>
__device__ __forceinline__ T fold_at(int i);
template <>
__device__ __forceinline__ double fold_at<double>(int i) { return c_fold[i]; }
template <>
__device__ __forceinline__ float fold_at<float>(int i) { return c_fold32[i]; }


// y (P) = A x (Q) along one line, A folded at table offset OFF, parity SIG,
// in the precision T of the data.
template <int P, int Q, int SIG, int OFF, typename T>
__device__ __forceinline__ void eo_apply(const T (&x)[Q], T (&y)[P]) {
    constexpr int hp = P / 2, hq = Q / 2;
    constexpr int oS = OFF, oT = OFF + hp * hq, oC = OFF + 2 * hp * hq;
    constexpr int oR = oC + ((Q % 2) ? hp : 0);
    T e[hq > 0 ? hq : 1], o[hq > 0 ? hq : 1];
#pragma unroll
    for (int i = 0; i < hq; i++) {
        e[i] = x[i] + x[Q - 1 - i];
        o[i] = x[i] - x[Q - 1 - i];
    }
#pragma unroll
    for (int a = 0; a < hp; a++) {
        T E = T(0), O = T(0);
#pragma unroll
        for (int i = 0; i < hq; i++) {
            E = fmx(fold_at<T>(oS + a * hq + i), e[i], E);
            O = fmx(fold_at<T>(oT + a * hq + i), o[i], O);
        }
        if (Q % 2) E = fmx(fold_at<T>(oC + a), x[hq], E);
        y[a] = E + O;
        y[P - 1 - a] = (SIG > 0) ? (E - O) : (O - E);
    }
    if (P % 2) {
        T M = T(0);
#pragma unroll
        for (int i = 0; i < hq; i++) M = fmx(fold_at<T>(oR + i), (SIG > 0) ? e[i] : o[i], M);
        if ((Q % 2) && SIG > 0) M = fmx(fold_at<T>(oR + hq), x[hq], M);
        y[hp] = M;
    }
}

// Padded element box q1 x q2 x q3 (i fastest); an odd row stride keeps the
// per-thread lines along i free of shared-memory bank conflicts.
template <int q1, int q2, int q3>
struct Box {
    static constexpr int sj = (q1 % 2) ? q1 : q1 + 1;
    static constexpr int sk = sj * q2;
    static constexpr int size = pad2(sk * q3);
    __device__ __forceinline__ static int at(int i, int j, int k) { return i + sj * j + sk * k; }
};

// Runs f(el, r) for every task r < COUNT of every element el < EPB of the
// block, densely over the block's threads (whole warps stay busy).
template <int COUNT, int EPB, class F>
__device__ __forceinline__ void for_tasks(int nel, F &&f) {
    for (int t = threadIdx.x; t < COUNT * EPB; t += blockDim.x) {
        const int el = t / COUNT, r = t - el * COUNT;
        if (el < nel) f(el, r);
    }
}

// Host: uploads the folded table (kFoldTotal doubles) to this TU's copies
// (the FP32 copy rounded from it).
#define FEM_DEFINE_FOLD_UPLOAD(NAME)                                                     \
    cudaError_t NAME(const double *table) {                                              \
        static float t32[kFoldTotal];                                                    \
        for (int i = 0; i < kFoldTotal; i++) t32[i] = (float)table[i];                   \
        cudaError_t e = cudaMemcpyToSymbol(c_fold, table, sizeof(double) * kFoldTotal, 0, \
                                           cudaMemcpyHostToDevice);                      \
        if (e != cudaSuccess) return e;                                                  \
        return cudaMemcpyToSymbol(c_fold32, t32, sizeof(float) * kFoldTotal, 0,         \
                                  cudaMemcpyHostToDevice);                               \
    }

}  // namespace fem
