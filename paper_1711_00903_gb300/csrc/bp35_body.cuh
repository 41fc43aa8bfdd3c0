// Body of the BP3.5 kernels as a device function, shared by the stand-alone
// kernels (bp35.cu) and the batched persistent kernel (batch.cu).  See
// bp35.cu for the algorithm and the GB300 design.
#pragma once

#include "eo.cuh"

namespace fem {
namespace {

// Layout of one block of EPB elements (three padded n^3 boxes each).
// SMEM_G: the block's factor planes (one contiguous range of EPB*7*n^3
// values) are brought into shared memory by one TMA bulk copy issued at
// block start, completing on an mbarrier, and the chain-rule phase reads
// them there; shared memory then holds [mbarrier | factors | boxes].
template <typename T, int N, int EPB_, bool SMEM_G = false>
struct Bp35Layout {
    static constexpr int n = N + 1, nn = n * n, NP = n * n * n;
    using B = Box<n, n, n>;
    // FP32 without SMEM_G: at kernel start one thread asks the TMA engine to
    // prefetch the block's factor planes into L2, so that the chain-rule
    // phase finds them there.  FP64 is bound by FP64 issue and reads the
    // factors directly.
    static constexpr bool PREFETCH = sizeof(T) == 4 && !SMEM_G;
    static constexpr bool STAGE_G = SMEM_G;
    static constexpr int EPB = EPB_;
    static constexpr int threads = ((nn * EPB + 31) / 32) * 32;  // the block needs at least this many
    static constexpr int gbytes = SMEM_G ? EPB * 7 * NP * (int)sizeof(T) : 0;
    static constexpr int oG = SMEM_G ? 16 : 0;          // factors (16-byte aligned)
    static constexpr int oBox = oG + gbytes;            // element boxes
    static constexpr int bytes = oBox + EPB * 3 * B::size * (int)sizeof(T);
    static constexpr int smem = bytes > oBox + threads * 8 ? bytes : oBox + threads * 8;
    static constexpr int oD = fold_offset(N, kFoldD), oDT = fold_offset(N, kFoldDT);
    static_assert(!SMEM_G || (gbytes / EPB) % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// FP32 factors staged by TMA into shared memory: possible for odd degrees
// (n even, so every element's planes span a multiple of 16 bytes), but two
// elements per block holding their factors in shared memory were measured
// slower than the L2 prefetch from N = 5 on (0.63 against 0.73 of the copy
// rate at N = 7), so only N = 3 uses it.
constexpr bool bp35_f32_staged(int N) { return N == 3; }
constexpr int bp35_f32_staged_epb(int N) { return (128 / ((N + 1) * (N + 1))) > 1 ? 128 / ((N + 1) * (N + 1)) : 1; }

// Elements per block of the stand-alone kernels: as many as fit 256 threads
// under the shared-memory budget, or the staged FP32 configuration.
template <typename T, int N, bool STAGED = (sizeof(T) == 4 && bp35_f32_staged(N))>
struct Bp35Cfg : Bp35Layout<T, N, pick_epb(N + 1, 3 * Box<N + 1, N + 1, N + 1>::size * (int)sizeof(T))> {};
template <typename T, int N>
struct Bp35Cfg<T, N, true> : Bp35Layout<T, N, bp35_f32_staged_epb(N), true> {};

// BP3.5 of elements [e0, e0 + nel) (nel <= EPB) by the whole block
// (blockDim.x >= Layout::threads), shared memory at smem_raw (Layout::smem
// bytes).  PCG = true: the input field is p <- z + beta p (stored back to p;
// beta read from *beta, p not read when beta is 0), and thread 0 writes the
// block's p . Ap to *part_out.
template <typename T, int N, int EPB_, bool PCG, bool SMEM_G = false>
__device__ __forceinline__ void bp35_block(unsigned char *smem_raw, int64_t e0, int nel, const T *__restrict__ G,
                                           double lambda, const T *__restrict__ q, T *__restrict__ Aq,
                                           const T *__restrict__ z, T *__restrict__ p,
                                           const double *__restrict__ beta, double *__restrict__ part_out) {
    using C = Bp35Layout<T, N, EPB_, SMEM_G>;
    using B = typename C::B;
    constexpr int n = C::n, nn = C::nn, NP = C::NP;
    T *smem = reinterpret_cast<T *>(smem_raw + C::oBox);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    const T *sG = reinterpret_cast<const T *>(smem_raw + C::oG);
    if (C::PREFETCH && threadIdx.x == 0)
        prefetch_l2(G + e0 * 7 * NP, (long long)nel * 7 * NP * (long long)sizeof(T));
    if (SMEM_G && threadIdx.x == 0) {
        const unsigned bytes = (unsigned)(nel * 7 * NP * (int)sizeof(T));
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(smem_raw + C::oG, G + e0 * 7 * NP, bytes, bar);
    }

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
    const bool staged_ok = !SMEM_G || mbar_wait(bar, 0);
    if (!staged_ok && (threadIdx.x & 31) == 0) atomicAdd(&g_wait_timeouts, 1ull);
    T acc[n];
    const T lam = (T)lambda;
    if (act) {
        const T *Ge = G + (e0 + el) * 7 * NP + r;
        const T *Gs = sG + el * 7 * NP + r;
        T Rt[n];
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int s = B::at(u, v, k);
            const T qr = sR[s], qs = sS[s];
            T g[7];
#pragma unroll
            for (int h = 0; h < 7; h++) g[h] = SMEM_G ? Gs[h * NP + k * nn] : __ldg(Ge + h * NP + k * nn);
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
        const double tot = block_sum((double)dot, reinterpret_cast<double *>(smem_raw + C::oBox));
        if (threadIdx.x == 0) *part_out = tot;
    }
    // a copy that did not complete in time may still be in flight: wait for
    // it once more (bounded) before the block's shared memory is released
    if (!staged_ok) mbar_wait(bar, 0);
}

}  // namespace
}  // namespace fem
