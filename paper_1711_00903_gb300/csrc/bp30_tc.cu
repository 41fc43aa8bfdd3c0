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
#include "tc_tile.cuh"

namespace fem {
namespace {

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

cudaError_t prepare_bp30_tc(int N) { return dispatch_degree<Tc30Prepare>(N); }

}  // namespace fem
