// Operand layout of the tensor-core operators (bp30_tc.cu, bp35_tc.cu): the
// 1D operators of Algorithms 4 and 5 as B fragments of mma.sync m16n8k16
// (f16 operands, FP32 accumulate), and the position map of the split K axis.
//
// Each contraction y[o] = sum_k Op[o][k] x[k] (k < Q, o < P) runs in one
// pass over a K axis of 3Q positions that carries three products,
//   x_hi Op_hi  +  x_lo' (Op_hi 2^-11)  +  x_hi Op_lo,
// with x_hi = f16(x), x_lo' = f16((x - x_hi) 2^11), Op_hi = f16(Op),
// Op_lo = f16(Op - Op_hi): the dropped x_lo Op_lo term and the roundings of
// the two parts leave about 2^-22 of relative error, against 2^-11 for one
// f16 product.  The positions come in blocks of 8 raw indices (segments hi,
// lo', hi of the same 8 indices), then a tail of the Q mod 8 remaining
// indices in the same three segments; in a block the 8-wide segments line
// up with the fragment columns, so a lane needs the same two raw values for
// all three segments.
//
// Shared by the host table builder and the kernel (both in the library).
#pragma once

#include <cstdint>

namespace fem {

// BP3.0: interpolation I (m x n), Gauss-point derivative Dt (m x m), its
// transpose, projection I^T (n x m); BP3.5: GLL derivative D (n x n) and its
// transpose.
enum { TC_I = 0, TC_DT = 1, TC_DTT = 2, TC_IT = 3, TC_D = 4, TC_DTR = 5, TC_OPS = 6 };

__host__ __device__ constexpr int tc_nt(int P) { return (P + 7) / 8; }         // 8-wide output tiles
__host__ __device__ constexpr int tc_ks(int Q) { return (3 * Q + 15) / 16; }   // 16-wide K steps
__host__ __device__ constexpr int tc_P(int N, int op) { return (op == TC_IT || op >= TC_D) ? N + 1 : N + 2; }
__host__ __device__ constexpr int tc_Q(int N, int op) { return (op == TC_I || op >= TC_D) ? N + 1 : N + 2; }
__host__ __device__ constexpr int tc_tiles(int N, int op) { return tc_nt(tc_P(N, op)) * tc_ks(tc_Q(N, op)); }
// Offset of an operator's tiles in the degree's table (in tiles of 32 lanes x 2 words).
__host__ __device__ constexpr int tc_offset(int N, int op) {
    int o = 0;
    for (int k = 0; k < op; k++) o += tc_tiles(N, k);
    return o;
}
__host__ __device__ constexpr int tc_total_tiles(int N) { return tc_offset(N, TC_OPS); }

// Segment (0: x_hi Op_hi, 1: x_lo' Op_hi 2^-11, 2: x_hi Op_lo) and raw
// index k of position p on the K axis of a contraction of length Q; raw -1
// marks padding.
__host__ __device__ constexpr int tc_seg(int Q, int p) {
    const int nb = Q / 8, r = Q % 8;
    if (p < 24 * nb) return (p % 24) / 8;
    const int w = p - 24 * nb;
    return (r > 0 && w < 3 * r) ? w / r : 0;
}
__host__ __device__ constexpr int tc_raw(int Q, int p) {
    const int nb = Q / 8, r = Q % 8;
    if (p < 24 * nb) return 8 * (p / 24) + (p % 8);
    const int w = p - 24 * nb;
    return (r > 0 && w < 3 * r) ? 8 * nb + w % r : -1;
}

// Shared-memory box strides (1, sj, sk) of the degree: chosen by counting
// bank conflicts of every fragment load and store of the kernel's phases
// over candidate strides (sj >= m, sk >= sj m).
__host__ __device__ constexpr int tc_sj(int N) {
    constexpr int t[16] = {0, 3, 5, 6, 6, 7, 12, 9, 10, 11, 12, 13, 19, 20, 20, 20};
    return t[N];
}
__host__ __device__ constexpr int tc_sk(int N) {
    constexpr int t[16] = {0, 9, 26, 37, 38, 76, 116, 92, 108, 140, 164, 180, 268, 300, 332, 340};
    return t[N];
}
// The same for the n x n x n boxes of the BP3.5 operator (sj >= n,
// sk >= sj n), counted over its own phases.
__host__ __device__ constexpr int tc35_sj(int N) {
    constexpr int t[16] = {0, 2, 3, 5, 6, 6, 7, 12, 9, 10, 11, 12, 13, 19, 23, 20};
    return t[N];
}
__host__ __device__ constexpr int tc35_sk(int N) {
    constexpr int t[16] = {0, 4, 9, 26, 37, 38, 52, 100, 92, 108, 140, 148, 180, 268, 348, 324};
    return t[N];
}

}  // namespace fem
