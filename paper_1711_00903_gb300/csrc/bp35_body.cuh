// Body of the BP3.5 kernels as a device function, shared by the stand-alone
// kernels (bp35.cu) and the batched persistent kernel (batch.cu).  See
// bp35.cu for the algorithm and the GB300 design.
#pragma once

#include <type_traits>

#include "eo.cuh"

namespace fem {
namespace {

// The n^3 box of the FP32 stream kernels (TMA-staged, bp35_stream.cuh) of
// degree N: at N = 7 and 15 the swizzled box (conflict-free in every
// direction); at N = 1, 3, 5, 9, 11 and 13 strides chosen by counting the
// bank conflicts of every access of bp35_core in the stream and block
// launches (a conflicting store weighted twice, as measured), among boxes
// no larger than the FP64 one; elsewhere the FP64 box, which no linear
// layout beat.  The block kernels keep the FP64 box: the swizzle's per-line
// address offsets cost registers, and there (at N = 13 and 15) they measured
// slower, spilling at N = 15.
template <int N, typename T>
struct Bp35Box {
    using type = Box<N + 1, N + 1, N + 1>;
};
template <int N>
struct Bp35Box<N, float> {
    static constexpr int n = N + 1;
    static constexpr int sj = N == 1 ? 2 : N == 3 ? 4 : N == 5 ? 6 : N == 9 ? 10 : N == 11 ? 12 : N == 13 ? 14 : 0;
    static constexpr int sk = N == 1 ? 5 : N == 3 ? 19 : N == 5 ? 41 : N == 9 ? 101 : N == 11 ? 145 : N == 13 ? 199 : 0;
    using type = typename std::conditional<
        (N == 7 || N == 15), SwizzledBox<n>,
        typename std::conditional<(sj > 0), StridedBox<n, n, n, (sj > 0 ? sj : n), (sk > 0 ? sk : n * n)>,
                                  Box<n, n, n>>::type>::type;
};

// Layout of one block of EPB elements (three padded n^3 boxes each);
// TUNED: the stream kernels' box (Bp35Box), else the FP64 box.
template <typename T, int N, int EPB_, bool TUNED = false>
struct Bp35Layout {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    using BX = typename std::conditional<TUNED, typename Bp35Box<N, T>::type, Box<n, n, n>>::type;
    static_assert(BX::size <= Box<n, n, n>::size, "an FP32 box outgrows the FP64 one");
    // elements sit as far apart as with the FP64 box (the strides above
    // were chosen for that spacing)
    struct B : BX {
        static constexpr int size = Box<n, n, n>::size;
    };
    // FP32 is bound by HBM: at kernel start one thread asks the TMA engine
    // to prefetch the block's factor planes (one contiguous range) into L2,
    // so that the chain-rule phase finds them there.  FP64 is bound by FP64
    // issue and reads the factors directly.
    static constexpr bool PREFETCH = sizeof(T) == 4;
    static constexpr int EPB = EPB_;
    static constexpr int threads = ((nn * EPB + 31) / 32) * 32;  // the block needs at least this many
    static constexpr int bytes = EPB * 3 * B::size * (int)sizeof(T);
    static constexpr int smem = bytes > threads * 8 ? bytes : threads * 8;
    static constexpr int oD = fold_offset(N, kFoldD), oDT = fold_offset(N, kFoldDT);
};

// Elements per block of the stand-alone kernels: as many as fit 256 threads
// under the shared-memory budget (512 for FP64 from N = 8 on, measured 9 %
// faster at N = 9 and 11; 128 for FP32 at N = 10, 6 % faster).
template <typename T, int N>
struct Bp35Cfg
    : Bp35Layout<T, N,
                 pick_epb(N + 1, 3 * Box<N + 1, N + 1, N + 1>::size * (int)sizeof(T),
                          sizeof(T) == 8 ? (N >= 8 ? 512 : 256) : (N == 10 ? 128 : 256))> {
};

// The operator on elements [e0, e0 + nel) (nel <= EPB) whose input field is
// already in the first box of each element (boxes: EPB x 3 boxes, filled
// before a barrier): derivatives, chain rule with the factors, transposes,
// output to Aq.  Gsrc points at the factors of element e0, in global memory
// or (G_SMEM) in shared memory, 7 planes of n^3 values per element, of type
// TG (T, or FP16 scaled by a power of two that gscale undoes on the output).
// Returns the thread's share of q . Aq (PCG; 0 otherwise).  Ends without a
// barrier.
template <typename T, int N, int EPB_, bool PCG, bool G_SMEM, typename TG = T, typename H = NoFactorHooks,
          bool TUNED = false>
__device__ __forceinline__ T bp35_core(T *smem, int64_t e0, int nel, const TG *__restrict__ Gsrc, double lambda,
                                       T *__restrict__ Aq, T gscale = T(1), const H &hooks = H()) {
    using C = Bp35Layout<T, N, EPB_, TUNED>;
    using B = typename C::B;
    constexpr int n = C::n, nn = C::nn, NP = C::NP;
    const int el = threadIdx.x / nn, r = threadIdx.x - el * nn;
    const int u = r % n, v = r / n;
    const bool act = el < nel;
    T *sQ = smem + el * 3 * B::size, *sR = sQ + B::size, *sS = sR + B::size;

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
    if (!hooks.before()) return T(0);

    // chain rule at the nodes of column (i=u, j=v), t-transpose in registers
    T acc[n];
    const T lam = (T)lambda;
    if (act) {
        const TG *Ge = Gsrc + el * 7 * NP + r;
        T Rt[n];
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int s = B::at(u, v, k);
            const T qr = sR[s], qs = sS[s];
            T g[7];
#pragma unroll
            for (int h = 0; h < 7; h++)
                g[h] = G_SMEM ? factor_ld<T>(Ge + h * NP + k * nn) : factor_ldg<T>(Ge + h * NP + k * nn);
            sR[s] = g[0] * qr + g[1] * qs + g[2] * qt[k];
            sS[s] = g[1] * qr + g[3] * qs + g[4] * qt[k];
            Rt[k] = g[2] * qr + g[4] * qs + g[5] * qt[k];
            acc[k] = g[6] * sQ[s];  // wJ q
        }
        T y[n];
        eo_apply<n, n, -1, C::oDT>(Rt, y);
#pragma unroll
        for (int k = 0; k < n; k++) acc[k] = (lambda != 0.0) ? fmx(lam, acc[k], y[k]) : y[k];
    }
    __syncthreads();
    hooks.after();

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
            T w = acc[k] + sR[s] + sS[s];
            if (!std::is_same<TG, T>::value) w *= gscale;
            Ae[k * nn] = w;
            if (PCG) dot = fmx(sQ[s], w, dot);
        }
    }
    return dot;
}

// BP3.5 of elements [e0, e0 + nel) (nel <= EPB) by the whole block
// (blockDim.x >= Layout::threads), shared memory at smem_raw (Layout::smem
// bytes).  PCG = true: the input field is p <- z + beta p (stored back to p;
// beta read from *beta, p not read when beta is 0), and thread 0 writes the
// block's p . Ap to *part_out.
template <typename T, int N, int EPB_, bool PCG, typename TG = T>
__device__ __forceinline__ void bp35_block(unsigned char *smem_raw, int64_t e0, int nel, const TG *__restrict__ G,
                                           double lambda, const T *__restrict__ q, T *__restrict__ Aq,
                                           const T *__restrict__ z, T *__restrict__ p,
                                           const double *__restrict__ beta, double *__restrict__ part_out,
                                           const double *__restrict__ ginv = nullptr) {
    using C = Bp35Layout<T, N, EPB_>;
    using B = typename C::B;
    constexpr int n = C::n, nn = C::nn, NP = C::NP;
    T *smem = reinterpret_cast<T *>(smem_raw);
    if (C::PREFETCH && threadIdx.x == 0)
        prefetch_l2(G + e0 * 7 * NP, (long long)nel * 7 * NP * (long long)sizeof(TG));

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
    __syncthreads();
    const T dot = bp35_core<T, N, EPB_, PCG, false, TG>(smem, e0, nel, G + e0 * 7 * NP, lambda, Aq,
                                                        factor_unscale<T>(ginv));
    if (PCG) {
        __syncthreads();  // the shared boxes are reused for the reduction
        const double tot = block_sum((double)dot, reinterpret_cast<double *>(smem_raw));
        if (threadIdx.x == 0) *part_out = tot;
    }
}

// Minimum resident blocks per SM that the register allocation must allow
// (0: the compiler's own heuristic).  At high degree the fully unrolled line
// kernels take up to 255 registers and leave one block per SM; capping them
// trades a few spills for latency hiding.  Chosen per precision and degree
// from the operator sweep on GB300.
template <typename T, int N>
constexpr int bp35_min_blocks() {
    if (sizeof(T) == 8) return N >= 10 ? 3 : 0;
    return N == 15 ? 3 : 0;
}

}  // namespace
}  // namespace fem
