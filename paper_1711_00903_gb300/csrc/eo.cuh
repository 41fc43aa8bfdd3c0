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
//
// FP32: the FP32 kernels are bound by instruction issue, not by the FMA
// lanes, so their contractions pair the two sums of each output row,
// (E_a, O_a) += (S[a][i], T[a][i]) * (e_i, o_i), in one packed two-lane FMA
// (__ffma2_rn, sm_100 and later) whose 64-bit coefficient is again a
// constant-bank operand: half the FMA instructions.  Each lane rounds like
// fmaf and the summation order is unchanged, so the results are the bits
// of the scalar form.
#pragma once

#include <type_traits>
#include <utility>
#include <vector>

#include "fold_layout.h"
#include "kernels_common.cuh"

namespace fem {

// ------------------------------------------------------------ device side

// One constant table per translation unit and precision (no relocatable
// device code); every TU that uses them uploads the same contents at basis
// setup.
static __constant__ double c_fold[kFoldTotal];
static __constant__ float2 c_fold32p[kFoldPairTotal];

// FP32 form of eo_apply below (the pair table, OFF its folded offset).
template <int P, int Q, int SIG, int OFF>
__device__ __forceinline__ void eo_apply_f32(const float (&x)[Q], float (&y)[P]) {
    constexpr int hp = P / 2, hq = Q / 2;
    constexpr int oP = fold_pair_offset_of(OFF);
    static_assert(oP >= 0, "no folded operator block starts at this offset");
    constexpr int oC = oP + hp * hq, oR = oC + ((Q % 2) ? hp : 0);
    float2 eo[hq > 0 ? hq : 1];
#pragma unroll
    for (int i = 0; i < hq; i++) eo[i] = make_float2(x[i] + x[Q - 1 - i], x[i] - x[Q - 1 - i]);
#pragma unroll
    for (int a = 0; a < hp; a++) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < hq; i++) acc = __ffma2_rn(c_fold32p[oP + a * hq + i], eo[i], acc);
        float E = acc.x;
        const float O = acc.y;
        if (Q % 2) E = fmaf(c_fold32p[oC + a].x, x[hq], E);
        y[a] = E + O;
        y[P - 1 - a] = (SIG > 0) ? (E - O) : (O - E);
    }
    if (P % 2) {
        float M = 0.0f;
#pragma unroll
        for (int i = 0; i < hq; i++) M = fmaf(c_fold32p[oR + i].x, (SIG > 0) ? eo[i].x : eo[i].y, M);
        if ((Q % 2) && SIG > 0) M = fmaf(c_fold32p[oR + hq].x, x[hq], M);
        y[hp] = M;
    }
}


// FP64 form of eo_apply below.
template <int P, int Q, int SIG, int OFF, typename T>
__device__ __forceinline__ void eo_apply_f64(const T (&x)[Q], T (&y)[P]) {
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
            E = fmx(c_fold[oS + a * hq + i], e[i], E);
            O = fmx(c_fold[oT + a * hq + i], o[i], O);
        }
        if (Q % 2) E = fmx(c_fold[oC + a], x[hq], E);
        y[a] = E + O;
        y[P - 1 - a] = (SIG > 0) ? (E - O) : (O - E);
    }
    if (P % 2) {
        T M = T(0);
#pragma unroll
        for (int i = 0; i < hq; i++) M = fmx(c_fold[oR + i], (SIG > 0) ? e[i] : o[i], M);
        if ((Q % 2) && SIG > 0) M = fmx(c_fold[oR + hq], x[hq], M);
        y[hp] = M;
    }
}

// y (P) = A x (Q) along one line, A folded at table offset OFF, parity SIG,
// in the precision T of the data.
template <int P, int Q, int SIG, int OFF, typename T>
__device__ __forceinline__ void eo_apply(const T (&x)[Q], T (&y)[P]) {
    static_assert(std::is_same<T, float>::value || std::is_same<T, double>::value, "FP32 or FP64 lines");
    if constexpr (std::is_same<T, float>::value)
        eo_apply_f32<P, Q, SIG, OFF>(x, y);
    else
        eo_apply_f64<P, Q, SIG, OFF>(x, y);
}

// Padded element box q1 x q2 x q3 (i fastest); an odd row stride keeps the
// per-thread lines along i free of shared-memory bank conflicts.
template <int q1, int q2, int q3>
struct Box {
    static constexpr int sj = (q1 % 2) ? q1 : q1 + 1;
    static constexpr int sk = sj * q2;
    static constexpr int size = pad2(sk * q3);
    __host__ __device__ __forceinline__ static int at(int i, int j, int k) { return i + sj * j + sk * k; }
};

// Box with explicit strides (1, SJ, SK) (the FP32 operators choose theirs
// against shared-memory bank conflicts).
template <int q1, int q2, int q3, int SJ, int SK>
struct StridedBox {
    static_assert(SJ >= q1 && SK >= SJ * q2, "strides too small for the box");
    static constexpr int sj = SJ, sk = SK;
    static constexpr int size = pad2(SK * (q3 - 1) + SJ * (q2 - 1) + q1);
    __host__ __device__ __forceinline__ static int at(int i, int j, int k) { return i + SJ * j + SK * k; }
};

// n^3 box (n = 8 or 16, a power of two dividing 32 with n >= 8) whose lines
// along every direction are free of bank conflicts on 32 banks of 4 bytes
// when the lanes of a warp take consecutive lines: rows of n words, planes
// n^2 + n words apart, and the row's words permuted by
//   (i, j, k) -> n^2 k + n k + n j + (i XOR g),  g = j / R + (n / R) (k mod R),
// R = 32 / n the rows a warp covers.  A warp's lanes on lines along i
// (fixed i, lanes over (j, k)) land in n-word groups indexed by j + k mod R
// and, inside a group, at distinct i XOR g; along j (lanes over (i, k)) and
// along k (lanes over (i, j)) the groups differ by k or j and i XOR g is a
// permutation of i.  A linear layout cannot serve all three at n = 8 or 16.
template <int n>
struct SwizzledBox {
    static_assert(n == 8 || n == 16, "swizzled boxes are for n = 8 and 16");
    static constexpr int R = 32 / n;
    static constexpr int sj = n, sk = n * n + n;
    static constexpr int size = pad2(sk * (n - 1) + sj * (n - 1) + n);
    __host__ __device__ __forceinline__ static int at(int i, int j, int k) {
        return sk * k + sj * j + (i ^ (j / R + (n / R) * (k % R)));
    }
};

// Host checks of a box layout (the library's layout self-check): the
// number of points (i, j, k) of the q1 x q2 x q3 box B that map outside
// [0, size) or onto a word that another point maps to.
template <class B, int q1, int q2, int q3>
int box_layout_violations(int size) {
    std::vector<unsigned char> seen((size_t)(size > 0 ? size : 0), 0);
    int bad = 0;
    for (int k = 0; k < q3; k++)
        for (int j = 0; j < q2; j++)
            for (int i = 0; i < q1; i++) {
                const int a = B::at(i, j, k);
                if (a < 0 || a >= size || seen[(size_t)a]++) bad++;
            }
    return bad;
}

// The bank conflicts (extra words served by one of 32 banks of 4 bytes) of
// the lines of an n^3 box B along each direction, the lanes of a warp
// taking 32 consecutive lines (line r at the other two indices (r mod n,
// r / n)), summed over every position along the line.
template <class B, int n>
int box_line_conflicts() {
    int extra = 0;
    for (int dir = 0; dir < 3; dir++)
        for (int l = 0; l < n; l++)
            for (int w = 0; w * 32 < n * n; w++) {
                int words[32][32];
                int count[32] = {0};
                for (int lane = 0; lane < 32 && w * 32 + lane < n * n; lane++) {
                    const int r = w * 32 + lane, u = r % n, v = r / n;
                    const int a = dir == 0 ? B::at(l, u, v) : dir == 1 ? B::at(u, l, v) : B::at(u, v, l);
                    const int bank = a % 32;
                    bool dup = false;
                    for (int c = 0; c < count[bank]; c++) dup = dup || words[bank][c] == a;
                    if (!dup) words[bank][count[bank]++] = a;
                }
                int most = 0;
                for (int b = 0; b < 32; b++) most = count[b] > most ? count[b] : most;
                extra += most > 1 ? most - 1 : 0;
            }
    return extra;
}

// Runs f(el, r) for every task r < COUNT of every element el < EPB of the
// block, densely over the block's threads (whole warps stay busy).
template <int COUNT, int EPB, class F>
__device__ __forceinline__ void for_tasks(int nel, F &&f) {
    for (int t = threadIdx.x; t < COUNT * EPB; t += blockDim.x) {
        const int el = t / COUNT, r = t - el * COUNT;
        if (el < nel) f(el, r);
    }
}

// Host: uploads the folded table (kFoldTotal doubles) to this TU's copies:
// the FP64 table as it is, the FP32 pair table rounded from it.
#define FEM_DEFINE_FOLD_UPLOAD(NAME)                                                      \
    cudaError_t NAME(const double *table) {                                               \
        static float2 tp[kFoldPairTotal];                                                 \
        for (int N = 1; N <= kMaxN; N++)                                                  \
            for (int op = 0; op < kFoldCount; op++) {                                     \
                const int P = fold_rows(op, N + 1, N + 2), Q = fold_cols(op, N + 1, N + 2);  \
                const int hh = (P / 2) * (Q / 2), rest = fold_size(P, Q) - 2 * hh;        \
                const double *f = table + fold_offset(N, op);                             \
                float2 *o = tp + fold_pair_offset(N, op);                                 \
                for (int k = 0; k < hh; k++) o[k] = make_float2((float)f[k], (float)f[hh + k]); \
                for (int k = 0; k < rest; k++) o[hh + k] = make_float2((float)f[2 * hh + k], 0.0f); \
            }                                                                             \
        cudaError_t e = cudaMemcpyToSymbol(c_fold, table, sizeof(double) * kFoldTotal, 0,  \
                                           cudaMemcpyHostToDevice);                       \
        if (e != cudaSuccess) return e;                                                   \
        return cudaMemcpyToSymbol(c_fold32p, tp, sizeof(float2) * kFoldPairTotal, 0,     \
                                  cudaMemcpyHostToDevice);                                \
    }

}  // namespace fem
