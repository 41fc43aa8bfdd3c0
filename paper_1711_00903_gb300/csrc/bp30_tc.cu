// BP3.0 dealiased screened-Poisson matvec (Algorithm 5) with its twelve 1D
// contractions on the tensor cores: mma.sync m16n8k16, f16 operands, FP32
// accumulate, FP32 vectors and geometric factors.  It is the inner operator
// of the FP64 defect-correction solver (FEM_PCG_MIXED_TC), where it stands
// in for the FP32 CUDA-core operator of FEM_PCG_MIXED.
//
// Accuracy.  One f16 product keeps 11 bits, and the inner solver needs
// about single precision: with element condition numbers near 10^6 a
// rounding noise of 2^-11 in the stages after the factors does not let the
// correction equation converge.  So every contraction carries three
// products on one K axis (tc_layout.h): x_hi Op_hi + x_lo' Op_hi 2^-11 +
// x_hi Op_lo, about 2^-22 of relative error.  To keep x inside the f16
// range whatever the field's magnitude, every line of every contraction is
// scaled by a power of two before the split (its largest entry into
// [2^14, 2^15)) and its results unscaled after the MMA: exact in both
// directions, so the operator stays linear.
//
// GB300 design.
//   - One warp per element and no block barrier for degrees up to 9
//     (two and four warps per element above, for the shared-memory size of
//     an element): each phase is a loop over 16-line tiles of the element
//     owned by the warp, so a warp waiting on its factors does not hold
//     others at a barrier.
//   - Lines are the MMA's M rows (16 per tile), the operator is the B
//     operand (held in registers for the phase, read once from a per-degree
//     table in L1), outputs are the N columns (8 per tile).
//   - Three shared boxes per element with strides chosen against bank
//     conflicts of the fragment loads and stores (tc_layout.h).
//   - The factors of an element are prefetched into L2 when the element
//     starts; the seven planes are read once, at the Gauss points of the
//     t-derivative tile that uses them.
// Phases (boxes A, B, C):
//   1. r-interpolation, q (global) -> X1 (B)         [m n n]
//   2. s-interpolation, B -> X2 (C)                   [m m n]
//   3. t-interpolation, C -> QG (A)                   [m m m]
//   4. r- and s-derivatives, A -> UR (B), US (C)
//   5. per t-line tile: t-derivative of A, chain rule with the 7 factors
//      (Wr -> B, Ws -> C, Wt -> A, lambda wJ qg kept in registers), then
//      the t-transpose of Wt plus the mass term -> A
//   6. r- and s-transposes in place (B, C)
//   7. t-projection of A + B + C -> X3 (A)           [m m n]
//   8. s-projection, A -> X4 (B)                     [m n n]
//   9. r-projection, B -> Aq (global)
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

// ---------------------------------------------------------------- layout

template <int N>
struct Tc30 {
    static constexpr int n = N + 1, m = N + 2, NP = n * n * n, MP = m * m * m, mm = m * m;
    static constexpr int SJ = tc_sj(N), SK = tc_sk(N);
    static_assert(SJ >= m && SK >= SJ * m, "box strides too small");
    static constexpr int BOX = ((SK * m + 3) / 4) * 4;  // floats per box (16-byte multiple)
    static constexpr int W = N <= 9 ? 1 : (N <= 12 ? 2 : 4);  // warps per element
    static constexpr int threads = 32 * W;
    static constexpr int smem = 3 * BOX * (int)sizeof(float) + 8 * W;
    // resident blocks per SM the register allocation must allow: as many as
    // the shared memory admits (about 200 KB of it), at most 24
    static constexpr int by_smem = (200 * 1024) / smem;
    static constexpr int min_blocks = by_smem < 1 ? 1 : (by_smem > 24 ? 24 : by_smem);
};

__device__ __forceinline__ void phase_sync(int W) {
    if (W == 1)
        __syncwarp();
    else
        __syncthreads();
}

// ---------------------------------------------------------------- kernel

template <int N, bool PCG>
__global__ void __launch_bounds__(Tc30<N>::threads, Tc30<N>::min_blocks)
bp30_tc_kernel(int64_t E, const float *__restrict__ G, double lambda, const float *__restrict__ q,
               float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
               const double *__restrict__ beta, double *__restrict__ part, const uint2 *__restrict__ tab) {
    using C = Tc30<N>;
    constexpr int n = C::n, m = C::m, NP = C::NP, MP = C::MP, mm = C::mm, SJ = C::SJ, SK = C::SK, W = C::W;
    extern __shared__ __align__(16) float tc_smem[];
    float *bA = tc_smem, *bB = tc_smem + C::BOX, *bC = tc_smem + 2 * C::BOX;
    const int64_t e = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float *Ge = G + e * 7 * MP;
    if (threadIdx.x == 0) prefetch_l2(Ge, 7ll * MP * (long long)sizeof(float));
    (void)g;
    (void)t;

    const float *qe;
    if (PCG) {  // p <- z + beta p of the element (beta = 0: p = z)
        const float bt = (float)(*beta);
        float *pe = p + e * NP;
        const float *ze = z + e * NP;
        for (int i = threadIdx.x; i < NP; i += blockDim.x) pe[i] = (bt == 0.f) ? ze[i] : fmaf(bt, pe[i], ze[i]);
        __syncthreads();
        qe = pe;
    } else {
        qe = q + e * NP;
    }

    // 1. r-interpolation: q -> X1 (B), extents (m, n, n)
    {
        OpFrag<tc_nt(m), tc_ks(n)> op;
        op.load(tab + 32 * tc_offset(N, TC_I), lane);
        GlobalSrc<n, !PCG> src{qe};
        constexpr int lines = n * n;
        for (int mt = warp; mt < (lines + 15) / 16; mt += W)
            tc_tile<n, m>(mt, lines, op, src, [&](int, int, int row, int o, bool ok, float v) {
                if (ok) bB[o + line_base<0, m, n, SJ, SK>(row)] = v;
            });
    }
    phase_sync(W);
    // 2. s-interpolation: X1 (B) -> X2 (C), extents (m, m, n)
    {
        OpFrag<tc_nt(m), tc_ks(n)> op;
        op.load(tab + 32 * tc_offset(N, TC_I), lane);
        BoxSrc<1, m, n, SJ, SK> src{bB};
        constexpr int lines = m * n;
        for (int mt = warp; mt < (lines + 15) / 16; mt += W)
            tc_tile<n, m>(mt, lines, op, src, [&](int, int, int row, int o, bool ok, float v) {
                if (ok) bC[o * SJ + line_base<1, m, m, SJ, SK>(row)] = v;
            });
    }
    phase_sync(W);
    // 3. t-interpolation: X2 (C) -> QG (A), extents (m, m, m)
    {
        OpFrag<tc_nt(m), tc_ks(n)> op;
        op.load(tab + 32 * tc_offset(N, TC_I), lane);
        BoxSrc<2, m, m, SJ, SK> src{bC};
        constexpr int lines = mm;
        for (int mt = warp; mt < (lines + 15) / 16; mt += W)
            tc_tile<n, m>(mt, lines, op, src, [&](int, int, int row, int o, bool ok, float v) {
                if (ok) bA[o * SK + line_base<2, m, m, SJ, SK>(row)] = v;
            });
    }
    phase_sync(W);
    // 4. r- and s-derivatives of QG: A -> UR (B), US (C)
    {
        OpFrag<tc_nt(m), tc_ks(m)> op;
        op.load(tab + 32 * tc_offset(N, TC_DT), lane);
        constexpr int lines = mm, MT = (lines + 15) / 16;
        BoxSrc<0, m, m, SJ, SK> sr{bA};
        BoxSrc<1, m, m, SJ, SK> ss{bA};
        for (int it = warp; it < 2 * MT; it += W) {
            if (it < MT)
                tc_tile<m, m>(it, lines, op, sr, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bB[o + line_base<0, m, m, SJ, SK>(row)] = v;
                });
            else
                tc_tile<m, m>(it - MT, lines, op, ss, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bC[o * SJ + line_base<1, m, m, SJ, SK>(row)] = v;
                });
        }
    }
    phase_sync(W);
    // 5. t-lines: derivative, chain rule with the factors, t-transpose
    {
        OpFrag<tc_nt(m), tc_ks(m)> opd, opt;
        opd.load(tab + 32 * tc_offset(N, TC_DT), lane);
        opt.load(tab + 32 * tc_offset(N, TC_DTT), lane);
        const float lam = (float)lambda;
        constexpr int lines = mm, NT = tc_nt(m);
        BoxSrc<2, m, m, SJ, SK> src{bA};
        for (int mt = warp; mt < (lines + 15) / 16; mt += W) {
            float mass[NT][4];
            tc_tile<m, m>(mt, lines, opd, src, [&](int nt, int c, int row, int o, bool ok, float ut) {
                float mv = 0.f;
                if (ok) {
                    const int s = o * SK + line_base<2, m, m, SJ, SK>(row);  // point (a, b, c = o)
                    const float *gp = Ge + row + o * mm;                       // a + m b + m^2 c
                    float gg[7];
#pragma unroll
                    for (int hh = 0; hh < 7; hh++) gg[hh] = __ldg(gp + hh * MP);
                    const float ur = bB[s], us = bC[s], qg = bA[s];
                    bB[s] = gg[0] * ur + gg[1] * us + gg[2] * ut;
                    bC[s] = gg[1] * ur + gg[3] * us + gg[4] * ut;
                    bA[s] = gg[2] * ur + gg[4] * us + gg[5] * ut;
                    mv = lam * gg[6] * qg;
                }
                mass[nt][c] = mv;
            });
            __syncwarp();
            tc_tile<m, m>(mt, lines, opt, src, [&](int nt, int c, int row, int o, bool ok, float v) {
                if (ok) bA[o * SK + line_base<2, m, m, SJ, SK>(row)] = v + mass[nt][c];
            });
        }
    }
    phase_sync(W);
    // 6. r- and s-transposes in place (B, C)
    {
        OpFrag<tc_nt(m), tc_ks(m)> op;
        op.load(tab + 32 * tc_offset(N, TC_DTT), lane);
        constexpr int lines = mm, MT = (lines + 15) / 16;
        BoxSrc<0, m, m, SJ, SK> sr{bB};
        BoxSrc<1, m, m, SJ, SK> ss{bC};
        for (int it = warp; it < 2 * MT; it += W) {
            if (it < MT)
                tc_tile<m, m>(it, lines, op, sr, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bB[o + line_base<0, m, m, SJ, SK>(row)] = v;
                });
            else
                tc_tile<m, m>(it - MT, lines, op, ss, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bC[o * SJ + line_base<1, m, m, SJ, SK>(row)] = v;
                });
        }
    }
    phase_sync(W);
    // 7. t-projection of the sum: A + B + C -> X3 (A), extents (m, m, n)
    {
        OpFrag<tc_nt(n), tc_ks(m)> op;
        op.load(tab + 32 * tc_offset(N, TC_IT), lane);
        Sum3Src<2, m, m, SJ, SK> src{bA, bB, bC};
        constexpr int lines = mm;
        for (int mt = warp; mt < (lines + 15) / 16; mt += W)
            tc_tile<m, n>(mt, lines, op, src, [&](int, int, int row, int o, bool ok, float v) {
                if (ok) bA[o * SK + line_base<2, m, m, SJ, SK>(row)] = v;
            });
    }
    phase_sync(W);
    // 8. s-projection: X3 (A) -> X4 (B), extents (m, n, n)
    {
        OpFrag<tc_nt(n), tc_ks(m)> op;
        op.load(tab + 32 * tc_offset(N, TC_IT), lane);
        BoxSrc<1, m, m, SJ, SK> src{bA};
        constexpr int lines = m * n;
        for (int mt = warp; mt < (lines + 15) / 16; mt += W)
            tc_tile<m, n>(mt, lines, op, src, [&](int, int, int row, int o, bool ok, float v) {
                if (ok) bB[o * SJ + line_base<1, m, n, SJ, SK>(row)] = v;
            });
    }
    phase_sync(W);
    // 9. r-projection: X4 (B) -> Aq (global, i fastest)
    float dot = 0.f;
    {
        OpFrag<tc_nt(n), tc_ks(m)> op;
        op.load(tab + 32 * tc_offset(N, TC_IT), lane);
        BoxSrc<0, m, n, SJ, SK> src{bB};
        float *oe = Aq + e * NP;
        const float *pe = PCG ? p + e * NP : nullptr;
        constexpr int lines = n * n;
        for (int mt = warp; mt < (lines + 15) / 16; mt += W)
            tc_tile<m, n>(mt, lines, op, src, [&](int, int, int row, int o, bool ok, float v) {
                if (ok) {
                    oe[n * row + o] = v;
                    if (PCG) dot = fmaf(pe[n * row + o], v, dot);
                }
            });
    }
    if (PCG) {  // the block's p . Ap, in a fixed order
        double d = (double)dot;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        double *red = reinterpret_cast<double *>(tc_smem + 3 * C::BOX);
        if (W > 1) {
            __syncthreads();
            if (lane == 0) red[warp] = d;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s = 0.0;
                for (int w = 0; w < W; w++) s += red[w];
                part[e] = s;
            }
        } else if (lane == 0) {
            part[e] = d;
        }
    }
}

template <bool PCG>
struct Tc30Launch {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const float *G, double lambda, const float *q, float *Aq, const float *z,
                               float *p, const double *beta, double *part, const uint2 *tab, cudaStream_t s) {
            using C = Tc30<N>;
            bp30_tc_kernel<N, PCG><<<(unsigned)E, C::threads, C::smem, s>>>(E, G, lambda, q, Aq, z, p, beta, part,
                                                                            tab);
            return cudaGetLastError();
        }
    };
};

template <int N>
struct Tc30Prepare {
    static cudaError_t run() {
        cudaError_t e = cudaFuncSetAttribute(bp30_tc_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Tc30<N>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp30_tc_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Tc30<N>::smem);
        return e;
    }
};

}  // namespace

cudaError_t launch_bp30_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                           cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<Tc30Launch<false>::L>(b->host.N, E, G, lambda, q, Aq, (const float *)nullptr,
                                                 (float *)nullptr, (const double *)nullptr, (double *)nullptr,
                                                 (const uint2 *)b->d_tc, s);
}

cudaError_t launch_bp30_pcg_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                               float *p, const double *beta, float *Ap, double *partials, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<Tc30Launch<true>::L>(b->host.N, E, G, lambda, (const float *)nullptr, Ap, z, p, beta,
                                                partials, (const uint2 *)b->d_tc, s);
}

int64_t bp30_tc_blocks(int64_t E) { return E; }

cudaError_t prepare_bp30_tc(int N) { return dispatch_degree<Tc30Prepare>(N); }

}  // namespace fem
