// BP3.0 dealiased screened-Poisson matvec, IEEE FP64 (Algorithm 5):
//   Aq = (I^T x I^T x I^T) [ Dt_r^T Rr + Dt_s^T Rs + Dt_t^T Rt + lambda wJ qg ],
//   qg = (I x I x I) q,  [Rr Rs Rt] = G [Dt_r qg, Dt_s qg, Dt_t qg],
// twelve one-dimensional contractions per element in one kernel with no
// global intermediates (Section 8: a three-kernel split was no faster, and
// removing global intermediates was the largest gain).
//
// GB300 design.  Bound by FP64 instruction issue (2 per clock per SM), so
// every contraction is one thread applying an even-odd folded operator to
// a whole line with constant-bank operands (eo.cuh), and the element lives
// in three m^3 shared-memory boxes:
//   1. r-interpolation lines (j, k)               q      -> X1
//   2. s-interpolation lines (a, k)               X1     -> X2
//   3. t-interpolation columns (a, b)             X2     -> QG (m^3)
//   4. r- and s-derivative lines                  QG     -> UR, US
//   5. per column (a, b): t-derivative, chain rule with the 7 factors,
//      t-transpose and the lambda wJ qg term, in registers (kept to step 7)
//   6. r- and s-transpose lines, in place          UR, US
//   7. per column: sum, t-projection               -> X3 (m x m x n)
//   8. s-projection lines (a, k)                  X3     -> X4 (m x n x n)
//   9. r-projection lines (j, k)                  X4     -> Aq (global)
#include "eo.cuh"

namespace fem {
namespace {

template <int N>
struct Bp30Cfg {
    static constexpr int n = N + 1, m = N + 2;
    static constexpr int NP = n * n * n, MP = m * m * m, mm = m * m;
    using B0 = Box<n, n, n>;
    using B1 = Box<m, n, n>;
    using B2 = Box<m, m, n>;
    using B3 = Box<m, m, m>;
    static constexpr int S = B3::size;  // every buffer holds one m^3 box
    static constexpr int per = 3 * S;
    static constexpr int EPB = pick_epb(m, per * 8);
    static constexpr int threads = ((mm * EPB + 31) / 32) * 32;
    static constexpr int smem = EPB * per * 8;
    static constexpr int oI = fold_offset(N, kFoldI), oIT = fold_offset(N, kFoldIT);
    static constexpr int oDt = fold_offset(N, kFoldDt), oDtT = fold_offset(N, kFoldDtT);
};

template <int N>
__global__ void __launch_bounds__(Bp30Cfg<N>::threads)
bp30_f64_kernel(int64_t E, const double *__restrict__ G, double lambda, const double *__restrict__ q,
                double *__restrict__ Aq) {
    using C = Bp30Cfg<N>;
    using B0 = typename C::B0;
    using B1 = typename C::B1;
    using B2 = typename C::B2;
    using B3 = typename C::B3;
    constexpr int n = C::n, m = C::m, NP = C::NP, MP = C::MP, mm = C::mm, EPB = C::EPB;
    constexpr int S = C::S, per = C::per;
    extern __shared__ double smem[];
    // per element: buffer A = smem + el*per, B = A + S, C = A + 2S

    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
        const int el = t / NP, p = t - el * NP;
        smem[el * per + S + B0::at(p % n, (p / n) % n, p / (n * n))] = __ldg(q + e0 * NP + t);
    }
    __syncthreads();

    // 1. r-interpolation (j, k): q (buffer B) -> X1 (buffer C)
    for_tasks<n * n, EPB>(nel, [&](int el, int r) {
        const int j = r % n, k = r / n;
        const double *X0 = smem + el * per + S;
        double *X1 = smem + el * per + 2 * S;
        double x[n], y[m];
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
        const double *X1 = smem + el * per + 2 * S;
        double *X2 = smem + el * per + S;
        double x[n], y[m];
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
        const double *X2 = smem + el * per + S;
        double *QG = smem + el * per;
        double x[n], y[m];
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
        const double *QG = smem + el * per;
        double *UR = smem + el * per + S, *US = smem + el * per + 2 * S;
        double x[m], y[m];
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

    // 5. column (a, b): t-derivative, chain rule, t-transpose, mass term.
    // Each thread has at most one column task (threads >= m*m*EPB), so acc
    // stays in its registers until step 7.
    const int cel = threadIdx.x / mm, cr = threadIdx.x - cel * mm;
    const int ca = cr % m, cb = cr / m;
    const bool cact = cel < nel;
    double acc[m];
    if (cact) {
        const double *QG = smem + cel * per;
        double *UR = smem + cel * per + S, *US = smem + cel * per + 2 * S;
        double x[m], ut[m], Rt[m];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = QG[B3::at(ca, cb, l)];
        eo_apply<m, m, -1, C::oDt>(x, ut);
        const double *Ge = G + (e0 + cel) * 7 * MP + cr;
#pragma unroll
        for (int c = 0; c < m; c++) {
            const int s = B3::at(ca, cb, c);
            const double ur = UR[s], us = US[s];
            double g[7];
#pragma unroll
            for (int h = 0; h < 7; h++) g[h] = __ldg(Ge + h * MP + c * mm);
            UR[s] = g[0] * ur + g[1] * us + g[2] * ut[c];
            US[s] = g[1] * ur + g[3] * us + g[4] * ut[c];
            Rt[c] = g[2] * ur + g[4] * us + g[5] * ut[c];
            acc[c] = (lambda != 0.0) ? (lambda * g[6]) * x[c] : 0.0;
        }
        double y[m];
        eo_apply<m, m, -1, C::oDtT>(Rt, y);
#pragma unroll
        for (int c = 0; c < m; c++) acc[c] += y[c];
    }
    __syncthreads();

    // 6. r- and s-transposes in place
    for_tasks<mm, EPB>(nel, [&](int el, int r) {
        const int u = r % m, v = r / m;
        double *UR = smem + el * per + S, *US = smem + el * per + 2 * S;
        double x[m], y[m];
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
    __syncthreads();

    // 7. column (a, b): sum of the three directions, t-projection -> X3 (A)
    if (cact) {
        const double *UR = smem + cel * per + S, *US = smem + cel * per + 2 * S;
        double *X3 = smem + cel * per;
        double y[n];
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

    // 8. s-projection (a, k): X3 (A) -> X4 (B)
    for_tasks<m * n, EPB>(nel, [&](int el, int r) {
        const int a = r % m, k = r / m;
        const double *X3 = smem + el * per;
        double *X4 = smem + el * per + S;
        double x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = X3[B2::at(a, l, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) X4[B1::at(a, l, k)] = y[l];
    });
    __syncthreads();

    // 9. r-projection (j, k): X4 (B) -> Aq
    for_tasks<n * n, EPB>(nel, [&](int el, int r) {
        const double *X4 = smem + el * per + S;
        const int j = r % n, k = r / n;
        double x[m], y[n];
#pragma unroll
        for (int l = 0; l < m; l++) x[l] = X4[B1::at(l, j, k)];
        eo_apply<n, m, 1, C::oIT>(x, y);
        double *o = Aq + (e0 + el) * NP + r * n;
#pragma unroll
        for (int l = 0; l < n; l++) o[l] = y[l];
    });
}

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp30_tu)

template <int N>
struct Bp30Launch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                           double *Aq, cudaStream_t s) {
        using C = Bp30Cfg<N>;
        (void)b;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp30_f64_kernel<N><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, lambda, q, Aq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp30Prepare {
    static cudaError_t run() {
        return cudaFuncSetAttribute(bp30_f64_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Bp30Cfg<N>::smem);
    }
};

}  // namespace

cudaError_t launch_bp30(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                        double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp30Launch>(b->host.N, b, E, G, lambda, q, Aq, s);
}

cudaError_t prepare_bp30(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp30_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<Bp30Prepare>(N);
}

}  // namespace fem
