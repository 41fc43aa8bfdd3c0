// Layout of the folded (even-odd) operator table shared by the host, which
// builds it at basis setup, and the kernels, which read it (eo.cuh).
#pragma once

#include "fem_internal.h"

namespace fem {

__host__ __device__ constexpr int fold_size(int P, int Q) {
    return 2 * (P / 2) * (Q / 2) + (P / 2) * (Q % 2) + (Q / 2) * (P % 2) + (P % 2) * (Q % 2);
}

// Operators of one degree, in table order.
enum FoldOp { kFoldI = 0, kFoldIT, kFoldD, kFoldDT, kFoldDt, kFoldDtT, kFoldCount };

__host__ __device__ constexpr int fold_rows(int op, int n, int m) {
    return (op == kFoldI || op == kFoldDt || op == kFoldDtT) ? m : n;
}
__host__ __device__ constexpr int fold_cols(int op, int n, int m) {
    return (op == kFoldIT || op == kFoldDt || op == kFoldDtT) ? m : n;
}
__host__ __device__ constexpr int fold_degree_size(int N) {
    int s = 0;
    for (int op = 0; op < kFoldCount; op++) s += fold_size(fold_rows(op, N + 1, N + 2), fold_cols(op, N + 1, N + 2));
    return s;
}
// Offset of degree N's block (N = 1..15) in the table.
__host__ __device__ constexpr int fold_degree_offset(int N) {
    int s = 0;
    for (int k = 1; k < N; k++) s += fold_degree_size(k);
    return s;
}
__host__ __device__ constexpr int fold_offset(int N, int op) {
    int s = fold_degree_offset(N);
    for (int k = 0; k < op; k++) s += fold_size(fold_rows(k, N + 1, N + 2), fold_cols(k, N + 1, N + 2));
    return s;
}
constexpr int kFoldTotal = fold_degree_offset(kMaxN + 1);

// The same table in pairs for the FP32 kernels, whose contractions issue one
// packed two-lane FMA per (S, T) entry: per operator, the hp x hq pairs
// (S[a][i], T[a][i]), then every remaining folded entry (middle column,
// middle row, centre) as (value, 0), in the order of the folded block.
__host__ __device__ constexpr int fold_pair_size(int P, int Q) { return fold_size(P, Q) - (P / 2) * (Q / 2); }
__host__ __device__ constexpr int fold_pair_offset(int N, int op) {
    int s = 0;
    for (int k = 1; k < N; k++)
        for (int o = 0; o < kFoldCount; o++) s += fold_pair_size(fold_rows(o, k + 1, k + 2), fold_cols(o, k + 1, k + 2));
    for (int o = 0; o < op; o++) s += fold_pair_size(fold_rows(o, N + 1, N + 2), fold_cols(o, N + 1, N + 2));
    return s;
}
constexpr int kFoldPairTotal = fold_pair_offset(kMaxN + 1, 0);
// Pair offset of the operator block that starts at folded offset off (-1 if
// no block starts there).
__host__ __device__ constexpr int fold_pair_offset_of(int off) {
    for (int N = 1; N <= kMaxN; N++)
        for (int op = 0; op < kFoldCount; op++)
            if (fold_offset(N, op) == off) return fold_pair_offset(N, op);
    return -1;
}

// Host: writes the folded form of A (P x Q row-major, parity sigma) to out
// (fold_size(P, Q) doubles): S, T (P/2 x Q/2 each), the middle column
// A[a][Q/2] (Q odd), the middle row A[P/2][i] (P odd), the centre entry.
inline void fold_matrix(int P, int Q, const double *A, double *out) {
    const int hp = P / 2, hq = Q / 2;
    double *S = out, *T = out + hp * hq, *cm = T + hp * hq, *rm = cm + (Q % 2 ? hp : 0);
    for (int a = 0; a < hp; a++)
        for (int i = 0; i < hq; i++) {
            S[a * hq + i] = 0.5 * (A[a * Q + i] + A[a * Q + (Q - 1 - i)]);
            T[a * hq + i] = 0.5 * (A[a * Q + i] - A[a * Q + (Q - 1 - i)]);
        }
    if (Q % 2)
        for (int a = 0; a < hp; a++) cm[a] = A[a * Q + hq];
    if (P % 2) {
        for (int i = 0; i < hq; i++) rm[i] = A[hp * Q + i];
        if (Q % 2) rm[hq] = A[hp * Q + hq];
    }
}

// Host: the whole folded block of one degree from its I, D, Dt.
void build_fold_block(int N, const double *I, const double *D, const double *Dt, double *out);

}  // namespace fem
