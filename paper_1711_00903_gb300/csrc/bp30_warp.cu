// FP32 BP3.0 matvec (Algorithm 5) with one warp per element: the inner
// operator of the FP32 defect-correction solver for BP3.0, and the FP32
// BP3.0 entry point, at the degrees where it is faster than the block
// kernel of bp30.cu.
//
// Why a second FP32 kernel.  The block kernel packs several elements into a
// block and separates its nine phases with block barriers; in FP32 it is
// neither ALU- nor bandwidth-bound but waits: on the seven factor planes of
// the column phase and on the barriers around it.  Here a warp owns an
// element from start to end and its phases are separated by __syncwarp
// only (two or four warps per element above N = 9, where an element's
// boxes would otherwise limit a SM to a few warps), so twenty-odd
// independent warps per SM each overlap their own factor loads with the
// other warps' contractions.  The lines are the block kernel's: one lane
// applies an even-odd folded 1D operator (eo.cuh) to a whole line in
// registers; the boxes and their padding are the same.
// Phases (boxes A, B, C of m^3 floats):
//   0. q (or p <- z + beta p) -> B                       [n n n]
//   1. r-interpolation lines (j, k)    B -> C             [m n n]
//   2. s-interpolation lines (a, k)    C -> B             [m m n]
//   3. t-interpolation columns (a, b)  B -> A             [m m m]
//   4. r- and s-derivative lines       A -> B, C
//   5. columns (a, b): t-derivative, chain rule with the 7 factors, the
//      t-transpose and the lambda wJ qg term -> A; Wr, Ws -> B, C in place
//   6. r- and s-transposes in place    B, C
//   7. columns: A + B + C, t-projection -> A (first n planes)
//   8. s-projection lines (a, k)       A -> B             [m n n]
//   9. r-projection lines (j, k)       B -> Aq (global)
#include "eo.cuh"

namespace fem {
namespace {

template <int N>
struct W30 {
    static constexpr int n = N + 1, m = N + 2, NP = n * n * n, MP = m * m * m, mm = m * m;
    using B0 = Box<n, n, n>;
    using B1 = Box<m, n, n>;
    using B2 = Box<m, m, n>;
    using B3 = Box<m, m, m>;
    static constexpr int S = ((B3::size + 3) / 4) * 4;  // floats per box
    static constexpr int W = N <= 9 ? 1 : (N <= 12 ? 2 : 4);
    static constexpr int threads = 32 * W;
    static constexpr int smem = 3 * S * (int)sizeof(float) + 8 * W;
    static constexpr int by_smem = (200 * 1024) / smem;
    static constexpr int min_blocks = by_smem < 1 ? 1 : (by_smem > 24 ? 24 : by_smem);
    static constexpr int oI = fold_offset(N, kFoldI), oIT = fold_offset(N, kFoldIT);
    static constexpr int oDt = fold_offset(N, kFoldDt), oDtT = fold_offset(N, kFoldDtT);
};

template <int W>
__device__ __forceinline__ void wsync() {
    if (W == 1)
        __syncwarp();
    else
        __syncthreads();
}

template <int N, bool PCG>
__global__ void __launch_bounds__(W30<N>::threads, W30<N>::min_blocks)
bp30w_kernel(int64_t E, const float *__restrict__ G, double lambda, const float *__restrict__ q,
             float *__restrict__ Aq, const float *__restrict__ z, float *__restrict__ p,
             const double *__restrict__ beta, double *__restrict__ part) {
    using C = W30<N>;
    using B0 = typename C::B0;
    using B1 = typename C::B1;
    using B2 = typename C::B2;
    using B3 = typename C::B3;
    constexpr int n = C::n, m = C::m, NP = C::NP, MP = C::MP, mm = C::mm, W = C::W, T = C::threads;
    extern __shared__ __align__(16) float w30_smem[];
    float *bA = w30_smem, *bB = w30_smem + C::S, *bC = w30_smem + 2 * C::S;
    const int64_t e = blockIdx.x;
    const int tid = threadIdx.x;
    const float *Ge = G + e * 7 * MP;
    if (tid == 0) prefetch_l2(Ge, 7ll * MP * (long long)sizeof(float));

    // 0. the input field into B
    if (PCG) {
        const float bt = (float)(*beta);
        float *pe = p + e * NP;
        const float *ze = z + e * NP;
        for (int i = tid; i < NP; i += T) {
            const float v = (bt == 0.f) ? ze[i] : fmaf(bt, pe[i], ze[i]);
            pe[i] = v;
            bB[B0::at(i % n, (i / n) % n, i / (n * n))] = v;
        }
    } else {
        const float *qe = q + e * NP;
        for (int i = tid; i < NP; i += T) bB[B0::at(i % n, (i / n) % n, i / (n * n))] = __ldg(qe + i);
    }
    wsync<W>();

    // 1. r-interpolation (j, k): B -> C
    for (int r = tid; r < n * n; r += T) {
        const int j = r % n, k = r / n;
        float x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = bB[B0::at(l, j, k)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) bC[B1::at(l, j, k)] = y[l];
    }
    wsync<W>();
    // 2. s-interpolation (a, k): C -> B
    for (int r = tid; r < m * n; r += T) {
        const int a = r % m, k = r / m;
        float x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = bC[B1::at(a, l, k)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) bB[B2::at(a, l, k)] = y[l];
    }
    wsync<W>();
    // 3. t-interpolation (a, b): B -> A
    for (int r = tid; r < mm; r += T) {
        const int a = r % m, b = r / m;
        float x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = bB[B2::at(a, b, l)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) bA[B3::at(a, b, l)] = y[l];
    }
    wsync<W>();
    // 4. r-derivative lines (b, c) -> B and s-derivative lines (a, c) -> C
    for (int r = tid; r < 2 * mm; r += T) {
        const bool sdir = r >= mm;
        const int rr = sdir ? r - mm : r, u = rr % m, v = rr / m;
        float x[m], y[m];
        if (!sdir) {
#pragma unroll
            for (int l = 0; l < m; l++) x[l] = bA[B3::at(l, u, v)];
            eo_apply<m, m, -1, C::oDt>(x, y);
#pragma unroll
            for (int l = 0; l < m; l++) bB[B3::at(l, u, v)] = y[l];
        } else {
#pragma unroll
            for (int l = 0; l < m; l++) x[l] = bA[B3::at(u, l, v)];
            eo_apply<m, m, -1, C::oDt>(x, y);
#pragma unroll
            for (int l = 0; l < m; l++) bC[B3::at(u, l, v)] = y[l];
        }
    }
    wsync<W>();
    // 5. columns (a, b): t-derivative, chain rule, t-transpose, mass term
    {
        const float lam = (float)lambda;
        for (int r = tid; r < mm; r += T) {
            const int a = r % m, b = r / m;
            float x[m], ut[m], Rt[m], ms[m], y[m];
#pragma unroll
            for (int l = 0; l < m; l++) x[l] = bA[B3::at(a, b, l)];
            eo_apply<m, m, -1, C::oDt>(x, ut);
            const float *gp = Ge + r;
#pragma unroll
            for (int c = 0; c < m; c++) {
                float g[7];
#pragma unroll
                for (int h = 0; h < 7; h++) g[h] = __ldg(gp + h * MP + c * mm);
                const int s = B3::at(a, b, c);
                const float ur = bB[s], us = bC[s];
                bB[s] = g[0] * ur + g[1] * us + g[2] * ut[c];
                bC[s] = g[1] * ur + g[3] * us + g[4] * ut[c];
                Rt[c] = g[2] * ur + g[4] * us + g[5] * ut[c];
                ms[c] = lam * g[6] * x[c];
            }
            eo_apply<m, m, -1, C::oDtT>(Rt, y);
#pragma unroll
            for (int c = 0; c < m; c++) bA[B3::at(a, b, c)] = y[c] + ms[c];
        }
    }
    wsync<W>();
    // 6. r- and s-transposes in place
    for (int r = tid; r < 2 * mm; r += T) {
        const bool sdir = r >= mm;
        const int rr = sdir ? r - mm : r, u = rr % m, v = rr / m;
        float x[m], y[m];
        if (!sdir) {
#pragma unroll
            for (int l = 0; l < m; l++) x[l] = bB[B3::at(l, u, v)];
            eo_apply<m, m, -1, C::oDtT>(x, y);
#pragma unroll
            for (int l = 0; l < m; l++) bB[B3::at(l, u, v)] = y[l];
        } else {
#pragma unroll
            for (int l = 0; l < m; l++) x[l] = bC[B3::at(u, l, v)];
            eo_apply<m, m, -1, C::oDtT>(x, y);
#pragma unroll
            for (int l = 0; l < m; l++) bC[B3::at(u, l, v)] = y[l];
        }
    }
    wsync<W>();
    // 7. columns: sum of the three directions, t-projection -> A (k < n)
    for (int r = tid; r < mm; r += T) {
        const int a = r % m, b = r / m;
        float x[m], y[n];
#pragma unroll
        for (int c = 0; c < m; c++) {
            const int s = B3::at(a, b, c);
            x[c] = bA[s] + bB[s] + bC[s];
        }
        eo_apply<n, m, 1, C::oIT>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) bA[B3::at(a, b, l)] = y[l];
    }
    wsync<W>();
    // 8. s-projection (a, k): A -> B
    for (int r = tid; r < m * n; r += T) {
        const int a = r % m, k = r / m;
        float x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = bA[B3::at(a, l, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) bB[B1::at(a, l, k)] = y[l];
    }
    wsync<W>();
    // 9. r-projection (j, k): B -> Aq
    float dot = 0.f;
    for (int r = tid; r < n * n; r += T) {
        const int j = r % n, k = r / n;
        float x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = bB[B1::at(l, j, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
        float *o = Aq + e * NP + r * n;
#pragma unroll
        for (int l = 0; l < n; l++) o[l] = y[l];
        if (PCG) {
            const float *pp = p + e * NP + r * n;  // written in phase 0 by this block
#pragma unroll
            for (int l = 0; l < n; l++) dot = fmaf(pp[l], y[l], dot);
        }
    }
    if (PCG) {  // the block's p . Ap in a fixed order
        double d = (double)dot;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (W == 1) {
            if (tid == 0) part[e] = d;
        } else {
            double *red = reinterpret_cast<double *>(w30_smem + 3 * C::S);
            if ((tid & 31) == 0) red[tid >> 5] = d;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < W; w++) s += red[w];
                part[e] = s;
            }
        }
    }
}

template <bool PCG>
struct W30Launch {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const float *G, double lambda, const float *q, float *Aq, const float *z,
                               float *p, const double *beta, double *part, cudaStream_t s) {
            using C = W30<N>;
            bp30w_kernel<N, PCG><<<(unsigned)E, C::threads, C::smem, s>>>(E, G, lambda, q, Aq, z, p, beta, part);
            return cudaGetLastError();
        }
    };
};

template <int N>
struct W30Prepare {
    static cudaError_t run() {
        cudaError_t e = cudaFuncSetAttribute(bp30w_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             W30<N>::smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bp30w_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     W30<N>::smem);
        return e;
    }
};

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp30w_tu)

}  // namespace

cudaError_t launch_bp30_warp(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                             cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<W30Launch<false>::L>(b->host.N, E, G, lambda, q, Aq, (const float *)nullptr,
                                                (float *)nullptr, (const double *)nullptr, (double *)nullptr, s);
}

cudaError_t launch_bp30_pcg_warp(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                 float *p, const double *beta, float *Ap, double *partials, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<W30Launch<true>::L>(b->host.N, E, G, lambda, (const float *)nullptr, Ap, z, p, beta,
                                               partials, s);
}

cudaError_t prepare_bp30_warp(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp30w_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<W30Prepare>(N);
}

}  // namespace fem
