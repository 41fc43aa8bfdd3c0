// Warp-level machinery of the tensor-core operators (bp30_tc.cu,
// bp35_tc.cu): mma.sync m16n8k16 with f16 operands and FP32 accumulation,
// the hi/lo split of each value on one K axis (tc_layout.h), the
// power-of-two scaling of every contraction line, and the tile of 16 lines
// that loads, converts, multiplies and hands its outputs to an epilogue.
#pragma once

#include <cuda_fp16.h>

#include "kernels_common.cuh"
#include "tc_layout.h"

namespace fem {
namespace {

// ---------------------------------------------------------------- fragments

__device__ __forceinline__ void mma16816(float (&c)[4], const unsigned (&a)[4], uint2 b) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ unsigned h2bits(__half2 h) { return *reinterpret_cast<unsigned *>(&h); }

// hi = f16(x), lo' = f16((x - hi) 2^11) of a pair (first in the low half).
__device__ __forceinline__ void split2(float x0, float x1, unsigned &hi, unsigned &lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 f = __half22float2(h);
    hi = h2bits(h);
    lo = h2bits(__floats2half2_rn((x0 - f.x) * 2048.f, (x1 - f.y) * 2048.f));
}

// The part of segment seg (1: lo', else hi) of one value, as an f16.
__device__ __forceinline__ __half part1(float x, int seg) {
    const __half h = __float2half_rn(x);
    return seg == 1 ? __float2half_rn((x - __half2float(h)) * 2048.f) : h;
}

// Power-of-two scale of a line (largest |x| of the quad of lanes that holds
// it, brought into [2^14, 2^15)) and its inverse.  Every lane of the warp
// takes part (shuffles).
__device__ __forceinline__ void line_scale(float mx, float &s, float &inv) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    unsigned e = (__float_as_uint(mx) >> 23) & 0xffu;
    e = e < 15u ? 15u : (e > 254u ? 254u : e);
    s = __uint_as_float((268u - e) << 23);
    inv = __uint_as_float((e - 14u) << 23);
}

// ---------------------------------------------------------------- one tile

// B fragments of one operator for a phase: NT x KS pairs of words per lane.
template <int NT, int KS>
struct OpFrag {
    uint2 b[NT][KS];
    __device__ __forceinline__ void load(const uint2 *__restrict__ tab, int lane) {
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int ks = 0; ks < KS; ks++) b[nt][ks] = __ldg(tab + (nt * KS + ks) * 32 + lane);
    }
};

// One 16-line tile of a contraction of length Q into P outputs.
// src.base(row) -> offset of a line, src.at(base, k) -> its k-th input;
// epi(nt, c, row, out, valid, v) receives each output (c: accumulator
// register 0..3; rows r0 = 16 mt + g for c < 2, r0 + 8 for c >= 2).
template <int Q, int P, class Src, class Epi>
__device__ __forceinline__ void tc_tile(int mt, int lines, const OpFrag<tc_nt(P), tc_ks(Q)> &op, Src &src,
                                        Epi &&epi) {
    constexpr int NT = tc_nt(P), KS = tc_ks(Q), nb = Q / 8, r = Q % 8, NB1 = nb > 0 ? nb : 1;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int rows[2] = {16 * mt + g, 16 * mt + g + 8};
    float xf[2][NB1][2];       // raw values 8 blk + 2t, + 1 of each row
    float xt[2][KS][2][2];     // tail values of each (k-step, half, element)
    float mx[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const bool ok = rows[h] < lines;
        const int base = ok ? src.base(rows[h]) : 0;
#pragma unroll
        for (int blk = 0; blk < nb; blk++) {
            const int k = 8 * blk + 2 * t;
            xf[h][blk][0] = ok ? src.at(base, k) : 0.f;
            xf[h][blk][1] = ok ? src.at(base, k + 1) : 0.f;
            mx[h] = fmaxf(mx[h], fmaxf(fabsf(xf[h][blk][0]), fabsf(xf[h][blk][1])));
        }
#pragma unroll
        for (int ks = 0; ks < KS; ks++)
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                const int c0 = 16 * ks + 8 * hh;
                if (c0 >= 24 * nb) {  // tail or padding
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int w = c0 - 24 * nb + 2 * t + e;
                        float v = 0.f;
                        if (r > 0 && w < 3 * r && ok) v = src.at(base, 8 * nb + w % (r > 0 ? r : 1));
                        xt[h][ks][hh][e] = v;
                        mx[h] = fmaxf(mx[h], fabsf(v));
                    }
                }
            }
    }
    float sc[2], inv[2];
    line_scale(mx[0], sc[0], inv[0]);
    line_scale(mx[1], sc[1], inv[1]);

    unsigned hiF[2][NB1], loF[2][NB1];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int blk = 0; blk < nb; blk++)
            split2(xf[h][blk][0] * sc[h], xf[h][blk][1] * sc[h], hiF[h][blk], loF[h][blk]);

    unsigned a[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ks++)
#pragma unroll
        for (int hh = 0; hh < 2; hh++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int c0 = 16 * ks + 8 * hh;
                unsigned word;
                if (c0 + 8 <= 24 * nb) {  // inside a block: segment and block known here
                    const int blk = c0 / 24, seg = (c0 % 24) / 8;
                    word = seg == 1 ? loF[h][blk < NB1 ? blk : 0] : hiF[h][blk < NB1 ? blk : 0];
                } else {
                    __half p[2];
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int w = c0 - 24 * nb + 2 * t + e;
                        const int seg = (r > 0 && w < 3 * r) ? w / (r > 0 ? r : 1) : 0;
                        p[e] = part1(xt[h][ks][hh][e] * sc[h], seg);
                    }
                    word = h2bits(__halves2half2(p[0], p[1]));
                }
                a[ks][2 * hh + h] = word;
            }

#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < KS; ks++) mma16816(acc, a[ks], op.b[nt][ks]);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int h = c >> 1, out = 8 * nt + 2 * t + (c & 1);
            epi(nt, c, rows[h], out, rows[h] < lines && out < P, acc[c] * inv[h]);
        }
    }
}

// ---------------------------------------------------------------- sources

// Line decomposition along direction DIR of a box with extents (d0, d1, d2)
// and strides (1, sj, sk): lines enumerate the other two directions, first
// one fastest.
template <int DIR, int D0, int D1, int SJ, int SK>
__device__ __forceinline__ int line_base(int row) {
    if (DIR == 0) return (row % D1) * SJ + (row / D1) * SK;  // (j, k)
    if (DIR == 1) return (row % D0) + (row / D0) * SK;       // (i, k)
    return (row % D0) + (row / D0) * SJ;                     // (i, j)
}
template <int DIR, int SJ, int SK>
struct KStride {
    static constexpr int v = DIR == 0 ? 1 : (DIR == 1 ? SJ : SK);
};

template <int DIR, int D0, int D1, int SJ, int SK>
struct BoxSrc {
    const float *p;
    __device__ __forceinline__ int base(int row) const { return line_base<DIR, D0, D1, SJ, SK>(row); }
    __device__ __forceinline__ float at(int b, int k) const { return p[b + k * KStride<DIR, SJ, SK>::v]; }
};

// Sum of three boxes with the same strides (phase 7).
template <int DIR, int D0, int D1, int SJ, int SK>
struct Sum3Src {
    const float *p0, *p1, *p2;
    __device__ __forceinline__ int base(int row) const { return line_base<DIR, D0, D1, SJ, SK>(row); }
    __device__ __forceinline__ float at(int b, int k) const {
        const int o = b + k * KStride<DIR, SJ, SK>::v;
        return p0[o] + p1[o] + p2[o];
    }
};

// The element's input field in global memory (i fastest), r-direction
// lines (j, k) at offset n * line; read-only (__ldg) unless written earlier
// in the same launch (PCG: p).
template <int n, bool RO>
struct GlobalSrc {
    const float *p;
    __device__ __forceinline__ int base(int row) const { return n * row; }
    __device__ __forceinline__ float at(int b, int k) const { return RO ? __ldg(p + b + k) : p[b + k]; }
};

__device__ __forceinline__ void phase_sync(int W) {
    if (W == 1)
        __syncwarp();
    else
        __syncthreads();
}

}  // namespace
}  // namespace fem
