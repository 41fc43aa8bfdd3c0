// BP3.5 collocated screened-Poisson matvec (Algorithm 4):
//   Aq = D_r^T Rr + D_s^T Rs + D_t^T Rt + lambda wJ q,
//   [Rr Rs Rt] = G [q_r q_s q_t],  q_r = (D x I x I) q, ...
// in IEEE FP64 (the operator of the paper) and in FP32 (the inner operator
// of the mixed-precision solver), plus a variant fused with the PCG
// direction update p <- z + beta p and the p . Ap reduction.
//
// GB300 design.  FP64 issues at 2 instructions per clock per SM on this
// part (1/64 of the FP32 rate), so the FP64 kernel is bound by its FP64
// instruction count, not by HBM or shared memory (ncu: FP64 pipe 83-96 %
// busy, DRAM 4-11 %); the same code in FP32 is bound by HBM.  The design
// minimises FP64 instructions and spends shared memory, registers and
// integer issue freely:
//   * every one-dimensional contraction is one thread applying the even-odd
//     folded D or D^T to a whole line (eo.cuh): about n/2 + 2 instructions
//     per node instead of n, operator entries as constant-bank operands;
//   * q^e and the r and s partial results of the element live in shared
//     memory (padded boxes), the t-direction work of a thread's (i, j)
//     column stays in registers, four barriers per element;
//   * several elements per block (n^2 threads each), coalesced loads of q
//     and of each geometric-factor plane, coalesced stores.
#include "eo.cuh"

namespace fem {
namespace {

template <typename T, int N>
struct Bp35Cfg {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    using B = Box<n, n, n>;
    // FP32 is bound by HBM: at kernel start one thread asks the TMA engine
    // to prefetch the block's factor planes (one contiguous range) into L2,
    // so that the chain-rule phase finds them there.  FP64 is bound by FP64
    // issue and reads the factors directly.
    static constexpr bool PREFETCH = sizeof(T) == 4;
    static constexpr int smem_elem = 3 * B::size * (int)sizeof(T);
    static constexpr int EPB = pick_epb(n, smem_elem);
    static constexpr int threads = ((nn * EPB + 31) / 32) * 32;
    static constexpr int bytes = EPB * 3 * B::size * (int)sizeof(T);
    static constexpr int smem = bytes > threads * 8 ? bytes : threads * 8;
    static constexpr int oD = fold_offset(N, kFoldD), oDT = fold_offset(N, kFoldDT);
};

// PCG = true: the input field is p <- z + beta p (stored back to p; beta
// read from *beta, p not read when beta is 0), and each block writes
// sum p . Ap to partials[blockIdx.x].
template <typename T, int N, bool PCG>
__global__ void __launch_bounds__(Bp35Cfg<T, N>::threads)
bp35_kernel(int64_t E, const T *__restrict__ G, double lambda, const T *__restrict__ q, T *__restrict__ Aq,
            const T *__restrict__ z, T *__restrict__ p, const double *__restrict__ beta,
            double *__restrict__ partials) {
    using C = Bp35Cfg<T, N>;
    using B = typename C::B;
    constexpr int n = C::n, nn = C::nn, NP = C::NP, EPB = C::EPB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);

    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int nel = (int)((E - e0) < EPB ? (E - e0) : EPB);
    if (C::PREFETCH && threadIdx.x == 0)
        prefetch_l2(G + e0 * 7 * NP, (long long)nel * 7 * NP * (long long)sizeof(T));

    // stage the input field of the block's elements (contiguous in memory)
    if (PCG) {
        const T bt = (T)(*beta);
        for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
            const int el = t / NP, s = t - el * NP;
            const int64_t g = e0 * NP + t;
            const T v = (bt == T(0)) ? z[g] : fmx(bt, p[g], z[g]);
            p[g] = v;
            smem[el * 3 * B::size + B::at(s % n, (s / n) % n, s / nn)] = v;
        }
    } else {
        for (int t = threadIdx.x; t < nel * NP; t += blockDim.x) {
            const int el = t / NP, s = t - el * NP;
            smem[el * 3 * B::size + B::at(s % n, (s / n) % n, s / nn)] = __ldg(q + e0 * NP + t);
        }
    }
    const int el = threadIdx.x / nn, r = threadIdx.x - el * nn;
    const int u = r % n, v = r / n;
    const bool act = el < nel;
    T *sQ = smem + el * 3 * B::size, *sR = sQ + B::size, *sS = sR + B::size;
    __syncthreads();

    // derivatives: r-line at (j=u, k=v) and s-line at (i=u, k=v) to shared,
    // t-line at (i=u, j=v) kept in registers
    T qt[n];
    if (act) {
        T x[n], y[n];
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
    T acc[n];
    const T lam = (T)lambda;
    if (act) {
        const T *Ge = G + (e0 + el) * 7 * NP + r;
        T Rt[n];
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int s = B::at(u, v, k);
            const T qr = sR[s], qs = sS[s];
            T g[7];
#pragma unroll
            for (int h = 0; h < 7; h++) g[h] = __ldg(Ge + h * NP + k * nn);
            sR[s] = g[0] * qr + g[1] * qs + g[2] * qt[k];
            sS[s] = g[1] * qr + g[3] * qs + g[4] * qt[k];
            Rt[k] = g[2] * qr + g[4] * qs + g[5] * qt[k];
            acc[k] = (lambda != 0.0) ? (lam * g[6]) * sQ[s] : T(0);
        }
        T y[n];
        eo_apply<n, n, -1, C::oDT>(Rt, y);
#pragma unroll
        for (int k = 0; k < n; k++) acc[k] += y[k];
    }
    __syncthreads();

    // r- and s-transposes, in place
    if (act) {
        T x[n], y[n];
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

    T dot = T(0);  // p . Ap of the thread's column, in the data's precision
    if (act) {
        T *Ae = Aq + (e0 + el) * NP + r;
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int s = B::at(u, v, k);
            const T w = acc[k] + sR[s] + sS[s];
            Ae[k * nn] = w;
            if (PCG) dot = fmx(sQ[s], w, dot);
        }
    }
    if (PCG) {
        __syncthreads();  // the shared boxes are reused for the reduction
        const double tot = block_sum((double)dot, reinterpret_cast<double *>(smem_raw));
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

template <int N>
struct Bp35Launch {
    static cudaError_t run(int64_t E, const double *G, double lambda, const double *q, double *Aq,
                           cudaStream_t s) {
        using C = Bp35Cfg<double, N>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp35_kernel<double, N, false><<<(unsigned)blocks, C::threads, C::smem, s>>>(
            E, G, lambda, q, Aq, nullptr, nullptr, nullptr, nullptr);
        return cudaGetLastError();
    }
};

template <int N>
struct Bp35F32Launch {
    static cudaError_t run(int64_t E, const float *G, double lambda, const float *q, float *Aq,
                           cudaStream_t s) {
        using C = Bp35Cfg<float, N>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        bp35_kernel<float, N, false><<<(unsigned)blocks, C::threads, C::smem, s>>>(
            E, G, lambda, q, Aq, nullptr, nullptr, nullptr, nullptr);
        return cudaGetLastError();
    }
};

template <typename T>
struct Bp35PcgLaunchT {
    template <int N>
    struct L {
        static cudaError_t run(int64_t E, const T *G, double lambda, const T *z, T *p, const double *beta,
                               T *Ap, double *partials, cudaStream_t s) {
            using C = Bp35Cfg<T, N>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            bp35_kernel<T, N, true><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, G, lambda, nullptr, Ap, z,
                                                                                 p, beta, partials);
            return cudaGetLastError();
        }
    };
};

template <int N>
struct Bp35Blocks {
    static cudaError_t run(int64_t E, int which, int64_t *out) {
        using C = Bp35Cfg<double, N>;
        using F = Bp35Cfg<float, N>;
        const int64_t a = (E + C::EPB - 1) / C::EPB, b = (E + F::EPB - 1) / F::EPB;
        *out = which == 0 ? a : which == 1 ? b : (a > b ? a : b);
        return cudaSuccess;
    }
};

template <int N>
struct Bp35Prepare {
    template <typename T, bool PCG>
    static cudaError_t one() {
        return cudaFuncSetAttribute(bp35_kernel<T, N, PCG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Bp35Cfg<T, N>::smem);
    }
    static cudaError_t run() {
        cudaError_t e = one<double, false>();
        if (e == cudaSuccess) e = one<double, true>();
        if (e == cudaSuccess) e = one<float, false>();
        if (e == cudaSuccess) e = one<float, true>();
        return e;
    }
};

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp35_tu)

}  // namespace

cudaError_t launch_bp35(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                        double *Aq, cudaStream_t s) {
    return dispatch_degree<Bp35Launch>(b->host.N, E, G, lambda, q, Aq, s);
}

cudaError_t launch_bp35_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q,
                            float *Aq, cudaStream_t s) {
    return dispatch_degree<Bp35F32Launch>(b->host.N, E, G, lambda, q, Aq, s);
}

cudaError_t launch_bp35_pcg(const fem_basis *b, int64_t E, const double *G, double lambda, const double *z,
                            double *p, const double *beta, double *Ap, double *partials, cudaStream_t s) {
    return dispatch_degree<Bp35PcgLaunchT<double>::L>(b->host.N, E, G, lambda, z, p, beta, Ap, partials, s);
}

cudaError_t launch_bp35_pcg_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                float *p, const double *beta, float *Ap, double *partials, cudaStream_t s) {
    return dispatch_degree<Bp35PcgLaunchT<float>::L>(b->host.N, E, G, lambda, z, p, beta, Ap, partials, s);
}

int64_t bp35_max_blocks(int N, int64_t E) {
    int64_t out = 0;
    dispatch_degree<Bp35Blocks>(N, E, 2, &out);
    return out;
}

int64_t bp35_blocks(int N, int64_t E, bool f32) {
    int64_t out = 0;
    dispatch_degree<Bp35Blocks>(N, E, f32 ? 1 : 0, &out);
    return out;
}

cudaError_t prepare_bp35(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp35_tu(fold_table);
    if (e != cudaSuccess) return e;
    return dispatch_degree<Bp35Prepare>(N);
}

}  // namespace fem
