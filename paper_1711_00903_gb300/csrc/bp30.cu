// BP3.0 dealiased screened-Poisson matvec, IEEE FP64 (Algorithm 5):
//   Aq = (I^T x I^T x I^T) [ Dt_r^T Rr + Dt_s^T Rs + Dt_t^T Rt + lambda wJ qg ],
//   qg = (I x I x I) q,  [Rr Rs Rt] = G [Dt_r qg, Dt_s qg, Dt_t qg],
// twelve one-dimensional contractions per element, all in one kernel with
// no global intermediates (Section 8: a three-kernel split was no faster,
// and removing global intermediates was the largest gain).
//
// GB300 design.  As for BP1.0 and BP3.5 the FP64 instruction count is the
// bound on this part (FP64 at about 1/64 of the FP32 rate), so:
//   * an m x m slab of threads per element, looping over the c slabs;
//   * q^e staged in shared memory once; the interpolated field qg, and the
//     r and s partial fluxes, kept whole in shared memory (3 m^3 doubles),
//     five barriers per element;
//   * the t-direction work of a thread's (a, b) column (t-interpolation,
//     t-derivative, t-transpose as a register scatter, t-projection) stays in
//     registers;
//   * coalesced loads of q and of each geometric-factor plane.
#include "kernels_common.cuh"

namespace fem {
namespace {

template <int n>
struct Bp30Cfg {
    static constexpr int m = n + 1;
    static constexpr int NP = n * n * n, MP = m * m * m;
    static constexpr int SE = pad2(MP);  // one m^3 plane
    static constexpr int smem_elem = 3 * SE * 8;
    static constexpr int EPB = pick_epb(m, smem_elem);
    static constexpr int threads = m * m * EPB;
    static constexpr int smem = (pad2(m * n) + pad2(m * m) + EPB * 3 * SE) * 8;
};

template <int n>
__global__ void __launch_bounds__(Bp30Cfg<n>::threads)
bp30_f64_kernel(int64_t E, const double *__restrict__ ops, const double *__restrict__ G,
                double lambda, const double *__restrict__ q, double *__restrict__ Aq) {
    using C = Bp30Cfg<n>;
    constexpr int m = C::m, NP = C::NP, MP = C::MP, EPB = C::EPB, mm = m * m, SE = C::SE;
    extern __shared__ double smem[];
    double *sI = smem;                  // I[a][i] at a*n + i
    double *sDt = sI + pad2(m * n);     // Dt[a][d] at a*m + d
    double *buf = sDt + pad2(m * m);
    const OpsLayout L{n, m};
    block_copy(sI, ops + L.offI(), m * n);
    block_copy(sDt, ops + L.offDt(), m * m);

    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int64_t nel = (E - e0) < EPB ? (E - e0) : EPB;
    // stage q into plane B of each element
    for (int t = threadIdx.x; t < EPB * NP; t += blockDim.x) {
        const int el = t / NP, p = t % NP;
        buf[el * 3 * SE + SE + p] = (el < nel) ? __ldg(q + (e0 + el) * NP + p) : 0.0;
    }

    const int el = threadIdx.x / mm, ab = threadIdx.x % mm;
    const int a = ab % m, b = ab / m;
    const int64_t e = e0 + el;
    const bool valid = el < nel;
    double *pA = buf + el * 3 * SE;  // qg [c][b][a], later u [k][b][a]
    double *pB = pA + SE;            // q, later Rr, later v [k][j][a]
    double *pC = pB + SE;            // t1 [k][j][a], later Rs
    __syncthreads();

    // r-interpolation: t1[k][j][a] = sum_i I[a][i] q[k][j][i]
    if (b < n) {
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < n; i++) s = fma(sI[a * n + i], pB[i + n * (b + n * k)], s);
            pC[a + m * (b + n * k)] = s;
        }
    }
    __syncthreads();

    // s- and t-interpolation of column (a, b) into registers and shared
    double qg[m];
    {
        double t2[n];
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int jj = 0; jj < n; jj++) s = fma(sI[b * n + jj], pC[a + m * (jj + n * k)], s);
            t2[k] = s;
        }
#pragma unroll
        for (int c = 0; c < m; c++) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < n; k++) s = fma(sI[c * n + k], t2[k], s);
            qg[c] = s;
            pA[ab + mm * c] = s;
        }
    }
    __syncthreads();

    // derivatives at the Gauss points, chain rule, t-transpose, mass term
    double acc[m];
#pragma unroll
    for (int c = 0; c < m; c++) acc[c] = 0.0;
    const double *Ge = G + (valid ? e : 0) * 7 * MP + ab;
#pragma unroll
    for (int c = 0; c < m; c++) {
        const double *qc = pA + mm * c;
        double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
        for (int d = 0; d < m; d++) {
            ur = fma(sDt[a * m + d], qc[d + m * b], ur);
            us = fma(sDt[b * m + d], qc[a + m * d], us);
            ut = fma(sDt[c * m + d], qg[d], ut);
        }
        double g[7];
#pragma unroll
        for (int h = 0; h < 7; h++) g[h] = valid ? __ldg(Ge + h * MP + c * mm) : 0.0;
        const double Rr = g[0] * ur + g[1] * us + g[2] * ut;
        const double Rs = g[1] * ur + g[3] * us + g[4] * ut;
        const double Rt = g[2] * ur + g[4] * us + g[5] * ut;
        pB[ab + mm * c] = Rr;  // q in pB was last read before two barriers ago
        pC[ab + mm * c] = Rs;  // t1 in pC was last read before the previous barrier
#pragma unroll
        for (int d = 0; d < m; d++) acc[d] = fma(sDt[c * m + d], Rt, acc[d]);
        if (lambda != 0.0) acc[c] = fma(lambda * g[6], qg[c], acc[c]);
    }
    __syncthreads();

    // r and s transposes, then t-projection into shared
    {
#pragma unroll
        for (int c = 0; c < m; c++) {
            const double *Rrc = pB + mm * c, *Rsc = pC + mm * c;
            double s = acc[c];
#pragma unroll
            for (int d = 0; d < m; d++) {
                s = fma(sDt[d * m + a], Rrc[d + m * b], s);
                s = fma(sDt[d * m + b], Rsc[a + m * d], s);
            }
            acc[c] = s;
        }
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < m; c++) s = fma(sI[c * n + k], acc[c], s);
            pA[ab + mm * k] = s;  // qg in pA was last read before the previous barrier
        }
    }
    __syncthreads();

    // s-projection: v[k][j][a] = sum_b I[b][j] u[k][b][a]
    if (b < n) {
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int bb = 0; bb < m; bb++) s = fma(sI[bb * n + b], pA[a + m * (bb + m * k)], s);
            pB[a + m * (b + n * k)] = s;  // Rr in pB was last read before the previous barrier
        }
    }
    __syncthreads();

    // r-projection and store
    if (a < n && b < n && valid) {
        double *oe = Aq + e * NP + a + n * b;
#pragma unroll
        for (int k = 0; k < n; k++) {
            double s = 0.0;
#pragma unroll
            for (int aa = 0; aa < m; aa++) s = fma(sI[aa * n + a], pB[aa + m * (b + n * k)], s);
            oe[n * n * k] = s;
        }
    }
}

template <int N>
struct Bp30Launch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda,
                           const double *q, double *Aq, cudaStream_t s) {
        using C = Bp30Cfg<N + 1>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp30_f64_kernel<N + 1><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, b->d_ops, G, lambda, q, Aq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp30Prepare {
    static cudaError_t run() {
        using C = Bp30Cfg<N + 1>;
        return cudaFuncSetAttribute(bp30_f64_kernel<N + 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    C::smem);
    }
};

}  // namespace

cudaError_t launch_bp30(const fem_basis *b, int64_t E, const double *G, double lambda,
                        const double *q, double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp30Launch>(b->host.N, b, E, G, lambda, q, Aq, s);
}

cudaError_t prepare_bp30(int N) { return dispatch_degree<Bp30Prepare>(N); }

}  // namespace fem
