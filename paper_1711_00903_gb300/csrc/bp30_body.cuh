// Body of the FP64 BP3.0 kernel as a device function, shared by the
// stand-alone kernel (bp30.cu) and the batched persistent kernel (batch.cu).
// See bp30.cu for the algorithm and the GB300 design.
#pragma once

#include <type_traits>

#include "eo.cuh"

namespace fem {
namespace {


// Strides (sj, sk) of the four FP32 boxes n^3, m n^2, m^2 n, m^3 of degree
// N (box b = 0..3), chosen by counting the shared-memory bank conflicts of
// every access of bp30_core, in the stream launch (one element per group)
// and the block launch (EPB elements per block), a conflicting store
// weighted twice (as measured), among the strides whose box fits in the
// m^3 box of the FP64 layout (shared memory per element unchanged).  On a
// 32-bank memory no linear m^3 layout serves the r-, s- and t-direction
// lines all without conflicts; the FP64 layout's odd row stride leaves
// conflicts in the other boxes and, for even m, in the columns.
__host__ __device__ constexpr int bp30f_stride(int N, int b, int which) {
    constexpr short t[16][4][2] = {{{0, 0}, {0, 0}, {0, 0}, {0, 0}},
                                   {{2, 16}, {3, 6}, {3, 9}, {3, 9}},
                                   {{3, 9}, {4, 21}, {4, 20}, {4, 19}},
                                   {{4, 16}, {5, 20}, {5, 25}, {5, 25}},
                                   {{5, 25}, {9, 45}, {6, 38}, {6, 41}},
                                   {{6, 36}, {7, 42}, {7, 52}, {7, 49}},
                                   {{7, 49}, {9, 72}, {8, 72}, {9, 72}},
                                   {{8, 65}, {9, 88}, {9, 85}, {9, 81}},
                                   {{9, 81}, {13, 117}, {10, 106}, {10, 101}},
                                   {{10, 100}, {11, 110}, {11, 121}, {11, 121}},
                                   {{11, 121}, {13, 143}, {12, 172}, {12, 145}},
                                   {{12, 145}, {14, 173}, {13, 173}, {13, 169}},
                                   {{13, 169}, {15, 206}, {14, 206}, {14, 199}},
                                   {{14, 196}, {15, 210}, {15, 239}, {15, 225}},
                                   {{15, 225}, {17, 255}, {16, 272}, {17, 272}},
                                   {{17, 272}, {18, 305}, {17, 305}, {17, 289}}};
    return t[N][b][which];
}

template <int N, typename T, int b, int q1, int q2, int q3>
struct Bp30Box {
    using type = Box<q1, q2, q3>;
};
template <int N, int b, int q1, int q2, int q3>
struct Bp30Box<N, float, b, q1, q2, q3> {
    using type = StridedBox<q1, q2, q3, bp30f_stride(N, b, 0), bp30f_stride(N, b, 1)>;
};

constexpr int max4(int a, int b, int c, int d) {
    return (a > b ? a : b) > (c > d ? c : d) ? (a > b ? a : b) : (c > d ? c : d);
}

// Layout of one block of EPB elements (three m^3 shared boxes each), data
// type T (double for the paper's FP64 operator, float for the inner operator
// of the mixed-precision solver).
template <int N, int EPB_, typename T = double, int BOXES = 3>
struct Bp30Layout {
    static constexpr int n = N + 1, m = N + 2;
    static constexpr int NP = n * n * n, MP = m * m * m, mm = m * m;
    using B0 = typename Bp30Box<N, T, 0, n, n, n>::type;
    using B1 = typename Bp30Box<N, T, 1, m, n, n>::type;
    using B2 = typename Bp30Box<N, T, 2, m, m, n>::type;
    using B3 = typename Bp30Box<N, T, 3, m, m, m>::type;
    // every buffer holds any box; the FP64 m^3 box size, so that elements
    // sit as far apart as the strides above were chosen for
    static constexpr int S = Box<m, m, m>::size;
    static_assert(max4(B0::size, B1::size, B2::size, B3::size) <= S, "an FP32 box outgrows the m^3 box");
    static constexpr int per = BOXES * S;
    static constexpr int EPB = EPB_;
    static constexpr int threads = ((mm * EPB + 31) / 32) * 32;  // the block needs at least this many
    static constexpr int bytes = EPB * per * (int)sizeof(T);
    static constexpr int smem = bytes > threads * 8 ? bytes : threads * 8;
    static constexpr bool PREFETCH = sizeof(T) == 4;  // see bp35_body.cuh
    static constexpr int oI = fold_offset(N, kFoldI), oIT = fold_offset(N, kFoldIT);
    static constexpr int oDt = fold_offset(N, kFoldDt), oDtT = fold_offset(N, kFoldDtT);
};

// Elements per block of the stand-alone kernel: as many as fit the target
// threads under the shared-memory budget: 256, and for the FP32 kernels 128
// at N = 3-6 and 8, where the smaller blocks measured 2-12 % faster.
constexpr int bp30_f32_threads(int N) { return (N >= 3 && N <= 6) || N == 8 ? 128 : 256; }
template <int N, typename T = double>
struct Bp30Cfg : Bp30Layout<N,
                            pick_epb(N + 2, 3 * Box<N + 2, N + 2, N + 2>::size * (int)sizeof(T),
                                     sizeof(T) == 4 ? bp30_f32_threads(N) : 256),
                            T> {};

// BP3.0 of elements [e0, e0 + nel) (nel <= EPB) by the whole block
// (blockDim.x >= Layout::threads), shared memory at smem (Layout::smem
// bytes).  PCG = true: the input field is p <- z + beta p (stored back to p;
// beta read from *beta, p not read when beta is 0), and thread 0 writes the
// block's p . Ap to *part_out.
// The operator on elements [e0, e0 + nel) whose input field is already in
// buffer B of each element (filled before a barrier): phases 1-9 below.
// Gsrc points at the factors of element e0, in global memory or (G_SMEM) in
// shared memory, 7 planes of m^3 values per element, of type TG (T, or FP16
// scaled by a power of two that gscale undoes on the output).  PCG: p holds
// the input field in global memory (the staging wrote it) for the thread's
// share of p . Ap, which is returned.  Ends without a barrier.
// MASS = true: also BP1.0 of the same field, Mq = I^T wJ I q with wJ the
// seventh factor, from the interpolated field the operator computes anyway
// (four boxes per element, the fourth, D, for BP1.0's t-projection); its
// projections run in phases 5, 6 and 8 beside the operator's.
template <int N, int EPB_, typename T, bool PCG, bool G_SMEM, typename TG, bool MASS = false,
          typename H = NoFactorHooks>
__device__ __forceinline__ T bp30_core(T *smem, int64_t e0, int nel, const TG *__restrict__ Gsrc, double lambda,
                                       T *__restrict__ Aq, const T *__restrict__ p, T gscale,
                                       T *__restrict__ Mq = nullptr, const H &hooks = H()) {
    using C = Bp30Layout<N, EPB_, T, MASS ? 4 : 3>;
    using B0 = typename C::B0;
    using B1 = typename C::B1;
    using B2 = typename C::B2;
    using B3 = typename C::B3;
    constexpr int n = C::n, m = C::m, NP = C::NP, MP = C::MP, mm = C::mm, EPB = C::EPB;
    constexpr int S = C::S, per = C::per;

    // 1. r-interpolation (j, k): q (buffer B) -> X1 (buffer C)
    for_tasks<n * n, EPB>(nel, [&](int el, int r) {
        const int j = r % n, k = r / n;
        const T *X0 = smem + el * per + S;
        T *X1 = smem + el * per + 2 * S;
        T x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = X0[B0::at(l, j, k)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) X1[B1::at(l, j, k)] = y[l];
    });
    __syncthreads();

    // 2. s-interpolation (a, k): X1 (C) -> X2 (B)
    for_tasks<m * n, EPB>(nel, [&](int el, int r) {
        const int a = r % m, k = r / m;
        const T *X1 = smem + el * per + 2 * S;
        T *X2 = smem + el * per + S;
        T x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = X1[B1::at(a, l, k)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) X2[B2::at(a, l, k)] = y[l];
    });
    __syncthreads();

    // 3. t-interpolation (a, b): X2 (B) -> QG (A)
    for_tasks<mm, EPB>(nel, [&](int el, int r) {
        const int a = r % m, b = r / m;
        const T *X2 = smem + el * per + S;
        T *QG = smem + el * per;
        T x[n], y[m];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = X2[B2::at(a, b, l)];
        eo_apply<m, n, 1, C::oI>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) QG[B3::at(a, b, l)] = y[l];
    });
    __syncthreads();

    // 4. r-derivative lines (b=u, c=v) -> UR (B), s-derivative lines (a=u, c=v) -> US (C)
    for_tasks<mm, EPB>(nel, [&](int el, int r) {
        const int u = r % m, v = r / m;
        const T *QG = smem + el * per;
        T *UR = smem + el * per + S, *US = smem + el * per + 2 * S;
        T x[m], y[m];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = QG[B3::at(l, u, v)];
        eo_apply<m, m, -1, C::oDt>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) UR[B3::at(l, u, v)] = y[l];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = QG[B3::at(u, l, v)];
        eo_apply<m, m, -1, C::oDt>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) US[B3::at(u, l, v)] = y[l];
    });
    __syncthreads();
    if (!hooks.before()) return T(0);

    // 5. column (a, b): t-derivative, chain rule, t-transpose, mass term.
    // Each thread has at most one column task (threads >= m*m*EPB), so acc
    // stays in its registers until step 7.
    const int cel = threadIdx.x / mm, cr = threadIdx.x - cel * mm;
    const int ca = cr % m, cb = cr / m;
    const bool cact = cel < nel;
    T acc[m];
    if (cact) {
        const T *QG = smem + cel * per;
        T *UR = smem + cel * per + S, *US = smem + cel * per + 2 * S;
        T x[m], ut[m], Rt[m];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = QG[B3::at(ca, cb, l)];
        eo_apply<m, m, -1, C::oDt>(x, ut);
        const TG *Ge = Gsrc + cel * 7 * MP + cr;
        T w1[m];  // MASS: wJ qg of the column (BP1.0's field)
#pragma unroll
        for (int c = 0; c < m; c++) {
            const int s = B3::at(ca, cb, c);
            const T ur = UR[s], us = US[s];
            T g[7];
#pragma unroll
            for (int h = 0; h < 7; h++) g[h] = G_SMEM ? factor_ld<T>(Ge + h * MP + c * mm) : factor_ldg<T>(Ge + h * MP + c * mm);
            UR[s] = g[0] * ur + g[1] * us + g[2] * ut[c];
            US[s] = g[1] * ur + g[3] * us + g[4] * ut[c];
            Rt[c] = g[2] * ur + g[4] * us + g[5] * ut[c];
            acc[c] = (T)lambda * g[6];  // lambda wJ, applied below
            if (MASS) w1[c] = mul_rn(g[6], x[c]);
        }
        T y[m];
        eo_apply<m, m, -1, C::oDtT>(Rt, y);
        // t-transpose plus the lambda wJ qg term (qg re-read from the box)
#pragma unroll
        for (int c = 0; c < m; c++)
            acc[c] = (lambda != 0.0) ? fmx(acc[c], QG[B3::at(ca, cb, c)], y[c]) : y[c];
        if constexpr (MASS) {  // BP1.0: t-projection of wJ qg -> D
            T y1[n];
            eo_apply<n, m, 1, C::oIT>(w1, y1);
            T *D = smem + cel * per + 3 * S;
#pragma unroll
            for (int l = 0; l < n; l++) D[B2::at(ca, cb, l)] = y1[l];
        }
    }
    __syncthreads();
    hooks.after();

    // 6. r- and s-transposes in place
    for_tasks<mm, EPB>(nel, [&](int el, int r) {
        const int u = r % m, v = r / m;
        T *UR = smem + el * per + S, *US = smem + el * per + 2 * S;
        T x[m], y[m];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = UR[B3::at(l, u, v)];
        eo_apply<m, m, -1, C::oDtT>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) UR[B3::at(l, u, v)] = y[l];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = US[B3::at(u, l, v)];
        eo_apply<m, m, -1, C::oDtT>(x, y);
#pragma unroll
        for (int l = 0; l < m; l++) US[B3::at(u, l, v)] = y[l];
    });
    if constexpr (MASS) {  // BP1.0: s-projection (a, k), D -> A (the interpolated field is no longer read)
        for_tasks<m * n, EPB>(nel, [&](int el, int r) {
            const int a = r % m, k = r / m;
            const T *D = smem + el * per + 3 * S;
            T *X = smem + el * per;
            T x[m], y[n];
#pragma unroll
            for (int l = 0; l < m; l++) x[l] = D[B2::at(a, l, k)];
            eo_apply<n, m, 1, C::oIT>(x, y);
#pragma unroll
            for (int l = 0; l < n; l++) X[B1::at(a, l, k)] = y[l];
        });
    }
    __syncthreads();

    // 7. column (a, b): sum of the three directions, t-projection -> X3 (A;
    // D when MASS, where A holds BP1.0's field)
    if (cact) {
        const T *UR = smem + cel * per + S, *US = smem + cel * per + 2 * S;
        T *X3 = smem + cel * per + (MASS ? 3 * S : 0);
        T y[n];
#pragma unroll
        for (int c = 0; c < m; c++) {
            const int s = B3::at(ca, cb, c);
            acc[c] += UR[s] + US[s];
        }
        eo_apply<n, m, 1, C::oIT>(acc, y);
#pragma unroll
        for (int l = 0; l < n; l++) X3[B2::at(ca, cb, l)] = y[l];
    }
    __syncthreads();

    // 8. s-projection (a, k): X3 (A, or D) -> X4 (B); MASS: BP1.0's
    // r-projection (j, k), A -> Mq
    if constexpr (MASS) {
        for_tasks<n * n, EPB>(nel, [&](int el, int r) {
            const T *X = smem + el * per;
            const int j = r % n, k = r / n;
            T x[m], y[n];
#pragma unroll
            for (int l = 0; l < m; l++) x[l] = X[B1::at(l, j, k)];
            eo_apply<n, m, 1, C::oIT>(x, y);
            T *o = Mq + (e0 + el) * NP + r * n;
#pragma unroll
            for (int l = 0; l < n; l++) o[l] = y[l];
        });
    }
    for_tasks<m * n, EPB>(nel, [&](int el, int r) {
        const int a = r % m, k = r / m;
        const T *X3 = smem + el * per + (MASS ? 3 * S : 0);
        T *X4 = smem + el * per + S;
        T x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = X3[B2::at(a, l, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) X4[B1::at(a, l, k)] = y[l];
    });
    __syncthreads();

    // 9. r-projection (j, k): X4 (B) -> Aq
    T dot = T(0);  // p . Ap of the thread's lines (PCG), in the data's precision
    for_tasks<n * n, EPB>(nel, [&](int el, int r) {
        const T *X4 = smem + el * per + S;
        const int j = r % n, k = r / n;
        T x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = X4[B1::at(l, j, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
        if (!std::is_same<TG, T>::value) {
#pragma unroll
            for (int l = 0; l < n; l++) y[l] *= gscale;
        }
        T *o = Aq + (e0 + el) * NP + r * n;
#pragma unroll
        for (int l = 0; l < n; l++) o[l] = y[l];
        if (PCG) {
            const T *pp = p + (e0 + el) * NP + r * n;  // written by this block's staging
#pragma unroll
            for (int l = 0; l < n; l++) dot = fmx(pp[l], y[l], dot);
        }
    });
    return dot;
}

// TG: type of the factors (T, or FP16 scaled by a power of two that the
// value at ginv undoes on the output).
template <int N, int EPB_, typename T = double, bool PCG = false, typename TG = T>
__device__ __forceinline__ void bp30_block(T *smem, int64_t e0, int nel, const TG *__restrict__ G, double lambda,
                                           const T *__restrict__ q, T *__restrict__ Aq,
                                           const T *__restrict__ z = nullptr, T *__restrict__ p = nullptr,
                                           const double *__restrict__ beta = nullptr,
                                           double *__restrict__ part_out = nullptr,
                                           const double *__restrict__ ginv = nullptr) {
    using C = Bp30Layout<N, EPB_, T>;
    using B0 = typename C::B0;
    constexpr int n = C::n, NP = C::NP, MP = C::MP;
    constexpr int S = C::S, per = C::per;
    // per element: buffer A = smem + el*per, B = A + S, C = A + 2S
    if (C::PREFETCH && threadIdx.x == 0)
        prefetch_l2(G + e0 * 7 * MP, (long long)nel * 7 * MP * (long long)sizeof(TG));
    if (PCG) {
        const T bt = (T)(*beta);
        for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
            const int el = t / NP, s = t - el * NP;
            const int64_t g = e0 * NP + t;
            const T v = (bt == T(0)) ? z[g] : fmx(bt, p[g], z[g]);
            p[g] = v;
            smem[el * per + S + B0::at(s % n, (s / n) % n, s / (n * n))] = v;
        }
    } else {
        for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
            const int el = t / NP, s = t - el * NP;
            smem[el * per + S + B0::at(s % n, (s / n) % n, s / (n * n))] = __ldg(q + e0 * NP + t);
        }
    }
    __syncthreads();
    const T gscale = std::is_same<TG, T>::value ? T(1) : factor_unscale<T>(ginv);
    const T dot = bp30_core<N, EPB_, T, PCG, false, TG>(smem, e0, nel, G + e0 * 7 * MP, lambda, Aq, p, gscale);
    if (PCG) {
        __syncthreads();  // the shared boxes are reused for the reduction
        const double tot = block_sum((double)dot, reinterpret_cast<double *>(smem));
        if (threadIdx.x == 0) *part_out = tot;
    }
}

// Minimum resident blocks per SM that the register allocation must allow
// (0: the compiler's own heuristic); see bp35_min_blocks.  Chosen per precision and
// degree from the operator sweep on GB300.
template <typename T, int N>
constexpr int bp30_min_blocks() {
    if (sizeof(T) == 8) return (N >= 9 && N <= 14) ? 2 : 0;
    if (N >= 9 && N <= 12) return 4;
    if (N == 13) return 3;
    if (N == 15) return 2;
    return 0;
}

}  // namespace
}  // namespace fem
