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
#include "bp30_body.cuh"

namespace fem {
namespace {

template <int N>
__global__ void __launch_bounds__(Bp30Cfg<N>::threads)
bp30_f64_kernel(int64_t E, const double *__restrict__ G, double lambda, const double *__restrict__ q,
                double *__restrict__ Aq) {
    using C = Bp30Cfg<N>;
    extern __shared__ double smem[];
    const int64_t e0 = (int64_t)blockIdx.x * C::EPB;
    const int nel = (int)((E - e0) < C::EPB ? (E - e0) : C::EPB);
    bp30_block<N, C::EPB>(smem, e0, nel, G, lambda, q, Aq);
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
