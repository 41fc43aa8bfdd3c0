// BP3.5 collocated screened-Poisson matvec, IEEE FP64 (Algorithm 4):
//   Aq = D_r^T Rr + D_s^T Rs + D_t^T Rt + lambda wJ q,
//   [Rr Rs Rt] = G [q_r q_s q_t],  q_r = (D x I x I) q, ...
//
// GB300 design.  FP64 issues at 2 instructions per clock per SM on this
// part (1/64 of the FP32 rate), so the kernel is bound by its FP64
// instruction count, not by HBM or shared memory (ncu: FP64 pipe ~96 %
// busy, DRAM ~4-10 %).  The design therefore minimises FP64 instructions
// and spends shared memory, registers and integer issue freely:
//   * every one-dimensional contraction is one thread applying the even-odd
//     folded D or D^T to a whole line (eo.cuh): about n/2 + 2 FP64
//     instructions per node instead of n, with the operator entries as
//     constant-bank operands;
//   * q^e and the r and s partial results of the element live in shared
//     memory (padded boxes), the t-direction work of a thread's (i, j)
//     column stays in registers, four barriers per element;
//   * several elements per block (n^2 threads each), coalesced loads of q
//     and of each geometric-factor plane, coalesced stores.
#include "eo.cuh"

namespace fem {
namespace {

template <int N>
struct Bp35Cfg {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    using B = Box<n, n, n>;
    static constexpr int smem_elem = 3 * B::size * 8;
    static constexpr int EPB = pick_epb(n, smem_elem);
    static constexpr int threads = ((nn * EPB + 31) / 32) * 32;
    static constexpr int smem = EPB * 3 * B::size * 8;
    static constexpr int oD = fold_offset(N, kFoldD), oDT = fold_offset(N, kFoldDT);
};

template <int N>
__global__ void __launch_bounds__(Bp35Cfg<N>::threads)
bp35_f64_kernel(int64_t E, const double *__restrict__ G, double lambda, const double *__restrict__ q,
                double *__restrict__ Aq) {
    using C = Bp35Cfg<N>;
    using B = typename C::B;
    constexpr int n = C::n, nn = C::nn, NP = C::NP, EPB = C::EPB;
    extern __shared__ double smem[];

    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);

    // stage q of the block's elements (contiguous in memory)
    for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
        const int el = t / NP, p = t - el * NP;
        const int i = p % n, j = (p / n) % n, k = p / nn;
        smem[el * 3 * B::size + B::at(i, j, k)] = __ldg(q + e0 * NP + t);
    }
    const int el = threadIdx.x / nn, r = threadIdx.x - el * nn;
    const int u = r % n, v = r / n;
    const bool act = el < nel;
    double *sQ = smem + el * 3 * B::size, *sR = sQ + B::size, *sS = sR + B::size;
    __syncthreads();

    // derivatives: r-line at (j=u, k=v) and s-line at (i=u, k=v) to shared,
    // t-line at (i=u, j=v) kept in registers
    double qt[n];
    if (act) {
        double x[n], y[n];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = sQ[B::at(l, u, v)];
        eo_apply<n, n, -1, C::oD>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) sR[B::at(l, u, v)] = y[l];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = sQ[B::at(u, l, v)];
        eo_apply<n, n, -1, C::oD>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) sS[B::at(u, l, v)] = y[l];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = sQ[B::at(u, v, l)];
        eo_apply<n, n, -1, C::oD>(x, qt);
    }
    __syncthreads();

    // chain rule at the nodes of column (i=u, j=v), t-transpose in registers
    double acc[n];
    if (act) {
        const double *Ge = G + (e0 + el) * 7 * NP + r;
        double Rt[n];
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int s = B::at(u, v, k);
            const double qr = sR[s], qs = sS[s];
            double g[7];
#pragma unroll
            for (int h = 0; h < 7; h++) g[h] = __ldg(Ge + h * NP + k * nn);
            sR[s] = g[0] * qr + g[1] * qs + g[2] * qt[k];
            sS[s] = g[1] * qr + g[3] * qs + g[4] * qt[k];
            Rt[k] = g[2] * qr + g[4] * qs + g[5] * qt[k];
            acc[k] = (lambda != 0.0) ? (lambda * g[6]) * sQ[s] : 0.0;
        }
        double y[n];
        eo_apply<n, n, -1, C::oDT>(Rt, y);
#pragma unroll
        for (int k = 0; k < n; k++) acc[k] += y[k];
    }
    __syncthreads();

    // r- and s-transposes, in place
    if (act) {
        double x[n], y[n];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = sR[B::at(l, u, v)];
        eo_apply<n, n, -1, C::oDT>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) sR[B::at(l, u, v)] = y[l];
#pragma unroll
        for (int l = 0; l < n; l++) x[l] = sS[B::at(u, l, v)];
        eo_apply<n, n, -1, C::oDT>(x, y);
#pragma unroll
        for (int l = 0; l < n; l++) sS[B::at(u, l, v)] = y[l];
    }
    __syncthreads();

    if (act) {
        double *Ae = Aq + (e0 + el) * NP + r;
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int s = B::at(u, v, k);
            Ae[k * nn] = acc[k] + sR[s] + sS[s];
        }
    }
}

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp35_tu)

template <int N>
struct Bp35Launch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                           double *Aq, cudaStream_t s) {
        using C = Bp35Cfg<N>;
        (void)b;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp35_f64_kernel<N><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, lambda, q, Aq);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp35Prepare {
    static cudaError_t run() {
        return cudaFuncSetAttribute(bp35_f64_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Bp35Cfg<N>::smem);
    }
};

}  // namespace

cudaError_t launch_bp35(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                        double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp35Launch>(b->host.N, b, E, G, lambda, q, Aq, s);
}

cudaError_t prepare_bp35(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp35_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<Bp35Prepare>(N);
}

}  // namespace fem
