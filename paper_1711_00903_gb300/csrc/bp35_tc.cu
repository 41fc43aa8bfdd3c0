// BP3.5 collocated screened-Poisson matvec (Algorithm 4) with its six 1D
// derivative contractions on the tensor cores: the split-f16 mma.sync
// scheme of bp30_tc.cu (tc_tile.cuh) applied to D and D^T at the GLL nodes,
// FP32 vectors and factors, the chain rule and the lambda term in FP32 on
// the CUDA cores.  The inner operator of FEM_PCG_MIXED_TC for BP3.5.
//
// One warp per element up to N = 11 (two and four above), three shared
// n^3 boxes per element with strides chosen against the bank conflicts of
// this kernel's fragment loads and stores (tc_layout.h):
//   0. q (or p <- z + beta p)                            -> A
//   1. r- and s-derivatives, A -> B, C
//   2. per t-line tile: t-derivative of A, chain rule with the 7 factors
//      (Wr -> B, Ws -> C, Wt -> A, lambda wJ q kept in registers), then the
//      t-transpose of Wt plus the mass term -> A
//   3. r- and s-transposes in place (B, C)
//   4. Aq = A + B + C (global), and for PCG the block's p . Ap
#include "tc_tile.cuh"

namespace fem {
namespace {

template <int N>
struct Tc35 {
    static constexpr int n = N + 1, NP = n * n * n, nn = n * n;
    static constexpr int SJ = tc35_sj(N), SK = tc35_sk(N);
    static_assert(SJ >= n && SK >= SJ * n, "box strides too small");
    static constexpr int BOX = ((SK * n + 3) / 4) * 4;
    static constexpr int W = N <= 11 ? 1 : (N <= 13 ? 2 : 4);
    static constexpr int threads = 32 * W;
    static constexpr int smem = 3 * BOX * (int)sizeof(float) + 8 * W;
    static constexpr int by_smem = (200 * 1024) / smem;
    static constexpr int min_blocks = by_smem < 1 ? 1 : (by_smem > 24 ? 24 : by_smem);
};

template <int N, bool PCG>
__global__ void __launch_bounds__(Tc35<N>::threads, Tc35<N>::min_blocks)
bp35_tc_kernel(int64_t E, const float *__restrict__ G, double lambda, const float *__restrict__ q,
               float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
               const double *__restrict__ beta, double *__restrict__ part, const uint2 *__restrict__ tab) {
    using C = Tc35<N>;
    constexpr int n = C::n, NP = C::NP, nn = C::nn, SJ = C::SJ, SK = C::SK, W = C::W;
    extern __shared__ __align__(16) float tc35_smem[];
    float *bA = tc35_smem, *bB = tc35_smem + C::BOX, *bC = tc35_smem + 2 * C::BOX;
    const int64_t e = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float *Ge = G + e * 7 * NP;
    if (threadIdx.x == 0) prefetch_l2(Ge, 7ll * NP * (long long)sizeof(float));

    // 0. the input field into A
    if (PCG) {
        const float bt = (float)(*beta);
        float *pe = p + e * NP;
        const float *ze = z + e * NP;
        for (int i = threadIdx.x; i < NP; i += blockDim.x) {
            const float v = (bt == 0.f) ? ze[i] : fmaf(bt, pe[i], ze[i]);
            pe[i] = v;
            bA[i % n + SJ * ((i / n) % n) + SK * (i / nn)] = v;
        }
    } else {
        const float *qe = q + e * NP;
        for (int i = threadIdx.x; i < NP; i += blockDim.x) bA[i % n + SJ * ((i / n) % n) + SK * (i / nn)] = __ldg(qe + i);
    }
    phase_sync(W);

    constexpr int lines = nn, MT = (lines + 15) / 16;
    // 1. r- and s-derivatives: A -> B, C
    {
        OpFrag<tc_nt(n), tc_ks(n)> op;
        op.load(tab + 32 * tc_offset(N, TC_D), lane);
        BoxSrc<0, n, n, SJ, SK> sr{bA};
        BoxSrc<1, n, n, SJ, SK> ss{bA};
        for (int it = warp; it < 2 * MT; it += W) {
            if (it < MT)
                tc_tile<n, n>(it, lines, op, sr, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bB[o + line_base<0, n, n, SJ, SK>(row)] = v;
                });
            else
                tc_tile<n, n>(it - MT, lines, op, ss, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bC[o * SJ + line_base<1, n, n, SJ, SK>(row)] = v;
                });
        }
    }
    phase_sync(W);
    // 2. t-lines: derivative, chain rule with the factors, t-transpose
    {
        OpFrag<tc_nt(n), tc_ks(n)> opd, opt;
        opd.load(tab + 32 * tc_offset(N, TC_D), lane);
        opt.load(tab + 32 * tc_offset(N, TC_DTR), lane);
        const float lam = (float)lambda;
        constexpr int NT = tc_nt(n);
        BoxSrc<2, n, n, SJ, SK> src{bA};
        for (int mt = warp; mt < MT; mt += W) {
            float mass[NT][4];
            tc_tile<n, n>(mt, lines, opd, src, [&](int nt, int c, int row, int o, bool ok, float ut) {
                float mv = 0.f;
                if (ok) {
                    const int s = o * SK + line_base<2, n, n, SJ, SK>(row);  // node (i, j, k = o)
                    const float *gp = Ge + row + o * nn;                       // i + n j + n^2 k
                    float gg[7];
#pragma unroll
                    for (int hh = 0; hh < 7; hh++) gg[hh] = __ldg(gp + hh * NP);
                    const float ur = bB[s], us = bC[s], qv = bA[s];
                    bB[s] = gg[0] * ur + gg[1] * us + gg[2] * ut;
                    bC[s] = gg[1] * ur + gg[3] * us + gg[4] * ut;
                    bA[s] = gg[2] * ur + gg[4] * us + gg[5] * ut;
                    mv = lam * gg[6] * qv;
                }
                mass[nt][c] = mv;
            });
            __syncwarp();
            tc_tile<n, n>(mt, lines, opt, src, [&](int nt, int c, int row, int o, bool ok, float v) {
                if (ok) bA[o * SK + line_base<2, n, n, SJ, SK>(row)] = v + mass[nt][c];
            });
        }
    }
    phase_sync(W);
    // 3. r- and s-transposes in place
    {
        OpFrag<tc_nt(n), tc_ks(n)> op;
        op.load(tab + 32 * tc_offset(N, TC_DTR), lane);
        BoxSrc<0, n, n, SJ, SK> sr{bB};
        BoxSrc<1, n, n, SJ, SK> ss{bC};
        for (int it = warp; it < 2 * MT; it += W) {
            if (it < MT)
                tc_tile<n, n>(it, lines, op, sr, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bB[o + line_base<0, n, n, SJ, SK>(row)] = v;
                });
            else
                tc_tile<n, n>(it - MT, lines, op, ss, [&](int, int, int row, int o, bool ok, float v) {
                    if (ok) bC[o * SJ + line_base<1, n, n, SJ, SK>(row)] = v;
                });
        }
    }
    phase_sync(W);
    // 4. the sum of the three directions, coalesced to global memory
    float dot = 0.f;
    {
        float *oe = Aq + e * NP;
        const float *pe = PCG ? p + e * NP : nullptr;
        for (int i = threadIdx.x; i < NP; i += blockDim.x) {
            const int s = i % n + SJ * ((i / n) % n) + SK * (i / nn);
            const float v = bA[s] + bB[s] + bC[s];
            oe[i] = v;
            if (PCG) dot = fmaf(pe[i], v, dot);
        }
    }
    if (PCG) {  // the block's p . Ap, in a fixed order
        double d = (double)dot;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (W > 1) {
            double *red = reinterpret_cast<double *>(tc35_smem + 3 * C::BOX);
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
struct Tc35Launch {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const float *G, double lambda, const float *q, float *Aq, const float *z,
                               float *p, const double *beta, double *part, const uint2 *tab, cudaStream_t s) {
            using C = Tc35<N>;
            bp35_tc_kernel<N, PCG><<<(unsigned)E, C::threads, C::smem, s>>>(E, G, lambda, q, Aq, z, p, beta, part,
                                                                            tab);
            return cudaGetLastError();
        }
    };
};

template <int N>
struct Tc35Prepare {
    static cudaError_t run() {
        cudaError_t e = cudaFuncSetAttribute(bp35_tc_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Tc35<N>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp35_tc_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Tc35<N>::smem);
        return e;
    }
};

}  // namespace

cudaError_t launch_bp35_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                           cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<Tc35Launch<false>::L>(b->host.N, E, G, lambda, q, Aq, (const float *)nullptr,
                                                 (float *)nullptr, (const double *)nullptr, (double *)nullptr,
                                                 (const uint2 *)b->d_tc, s);
}

cudaError_t launch_bp35_pcg_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                               float *p, const double *beta, float *Ap, double *partials, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<Tc35Launch<true>::L>(b->host.N, E, G, lambda, (const float *)nullptr, Ap, z, p, beta,
                                                partials, (const uint2 *)b->d_tc, s);
}

cudaError_t prepare_bp35_tc(int N) { return dispatch_degree<Tc35Prepare>(N); }

}  // namespace fem
