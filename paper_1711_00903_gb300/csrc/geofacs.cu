// Geometric factors of trilinear hexahedra, IEEE FP64 (Section 4):
//   X = dx/d(r,s,t),  |J| = det X,  G = |J| X^{-1} X^{-T},
// each multiplied by the tensor quadrature weight w_a w_b w_c, stored as the
// planes Grr, Grs, Grt, Gss, Gst, Gtt, wJ (BP3.5 at GLL nodes, BP3.0 at
// Gauss points) or wJ alone (BP1.0 at Gauss points).
//
// GB300 design.  FP64-issue bound like the operators.  The columns of X of
// a trilinear map factor over the tensor grid: dx/dr depends on (s, t) only,
// dx/ds on (r, t) and dx/dt on (r, s), so each block first tabulates the
// three q x q column tables of its element in shared memory (O(q^2) work),
// then every point needs only the cofactor vectors C_r = X_s x X_t,
// C_s = X_t x X_r, C_t = X_r x X_s (the rows of |J| X^{-1}), the
// determinant X_r . C_r and the six products G = C C^T / |J|.  Stores are
// coalesced per plane.
#include "kernels_common.cuh"

namespace fem {
namespace {

template <int qn>
struct GeoCfg {
    static constexpr int QP = qn * qn * qn, qq = qn * qn;
    static constexpr int SD = (qq > 36) ? qq : 36;  // per-thread minima, or the 36 map coefficients
    static constexpr int smem_elem = (24 + 9 * qq + SD) * 8;
    // about 512 threads per block (measured faster than 256 and 128 at N = 7)
    static constexpr int EPB = pick_epb(qn, smem_elem, 512);
    static constexpr int threads = qq * EPB;
    static constexpr int smem = (2 * pad2(qn) + EPB * pad2(24 + 9 * qq + SD)) * 8;
};

// 1 / d in FP64: an FP32 reciprocal seed refined by two Newton steps
// r <- r + r (1 - d r), each doubling the correct bits (about 22, 44, then
// the full 53).  The seed's conversions between the IEEE binary64 and
// binary32 formats are done on the bit fields with integer operations
// (sign; exponent rebiased from 1023 to 127; the top 23 mantissa bits,
// truncated), so the FP64 pipe, the part's bottleneck, executes only the
// four FMAs.  Falls back to a division when |d| is outside 2^-120..2^121,
// where the seed or its reciprocal would leave the binary32 normal range.
__device__ __forceinline__ double recip(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32);
    const int ex = (int)((hi >> 20) & 0x7FFu) - 1023;  // unbiased binary64 exponent
    if (ex < -120 || ex > 120) return 1.0 / d;
    const unsigned fb = (hi & 0x80000000u) | ((unsigned)(ex + 127) << 23) | ((hi & 0xFFFFFu) << 3) |
                        (unsigned)((b >> 29) & 0x7u);
    const unsigned rb = __float_as_uint(__frcp_rn(__uint_as_float(fb)));
    const int rex = (int)((rb >> 23) & 0xFFu) - 127;   // unbiased binary32 exponent of the seed
    const unsigned rhi = (rb & 0x80000000u) | ((unsigned)(rex + 1023) << 20) | ((rb & 0x7FFFFFu) >> 3);
    double r = __longlong_as_double((long long)(((unsigned long long)rhi << 32) |
                                                ((unsigned long long)(rb & 0x7u) << 29)));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// kind: 1 = wJ only, 2 and 3 = 7 planes, 4 = 7 planes and, in wj2, a copy
// of the wJ plane in the BP1.0 layout (BP3.0 and BP1.0 factors live at the
// same Gauss points, so one pass serves both); MIN: also the per-element
// minimum |J|.
template <int qn, int kind, bool MIN>
__device__ __forceinline__ void geofacs_body(int64_t E, const double *__restrict__ nodes,
                                             const double *__restrict__ weights, const double *__restrict__ verts,
                                             double *__restrict__ geo, double *__restrict__ detJ_min,
                                             double *__restrict__ wj2) {
    using C = GeoCfg<qn>;
    constexpr int QP = C::QP, qq = C::qq, EPB = C::EPB;
    constexpr int PER = pad2(24 + 9 * qq + C::SD);
    extern __shared__ double smem[];
    double *sx = smem, *sw = sx + pad2(qn);
    double *buf = sw + pad2(qn);
    for (int t = threadIdx.x; t < qn; t += blockDim.x) {
        sx[t] = __ldg(nodes + t);
        sw[t] = __ldg(weights + t);
    }
    const int64_t e0 = (int64_t)blockIdx.x * EPB;
    const int64_t nel = (E - e0) < EPB ? (E - e0) : EPB;
    for (int t = threadIdx.x; t < EPB * 24; t += blockDim.x) {
        const int el = t / 24, p = t % 24;
        buf[el * PER + p] = (el < nel) ? __ldg(verts + (e0 + el) * 24 + p) : 0.0;
    }
    __syncthreads();

    const int el = threadIdx.x / qq, ab = threadIdx.x % qq;
    const int u = ab % qn, v = ab / qn;
    const bool valid = el < nel;
    const int64_t e = e0 + el;
    const double *vx = buf + el * PER;     // vertices [c][d]
    double *Xr = buf + el * PER + 24;      // dx/dr at (s_u, t_v): [u][v][d]
    double *Xs = Xr + 3 * qq;              // dx/ds at (r_u, t_v)
    double *Xt = Xs + 3 * qq;              // dx/dt at (r_u, s_v)
    double *sdet = Xt + 3 * qq;            // per-thread minimum |J|

    // tabulate the three column tables of X.  Along r the map's derivative is
    // dx/dr(s, t) = 1/8 [ A (1-s)(1-t) + B (1+s)(1-t) + C (1-s)(1+t) + D (1+s)(1+t) ]
    // with the r-edge vectors A = x1 - x0, B = x3 - x2, C = x5 - x4,
    // D = x7 - x6, i.e. the bilinear form K0 + s K1 + t (K2 + s K3); the same
    // holds along s and t with their own edges.  The 3 x 4 x 3 coefficients
    // of an element are formed once (in shared memory), then each table entry
    // costs three FMAs per component.
    double *K = sdet;  // 36 coefficients, reused below for the minimum
    for (int ci = ab; ci < 36; ci += qq) {
        // K[(dir*4 + w)*3 + d]: dir 0 = r, 1 = s, 2 = t; w = coefficient
        const int dir = ci / 12, w = (ci / 3) % 4, d = ci % 3;
        // corner pairs (lower, upper) of the four edges along dir, in the
        // order (-,-), (+,-), (-,+), (+,+) of the two other coordinates
        const int stride = 1 << dir;
        int base[4];
        {
            const int o1 = (dir == 0) ? 2 : 1, o2 = (dir == 2) ? 2 : 4;
            base[0] = 0;
            base[1] = o1;
            base[2] = o2;
            base[3] = o1 + o2;
        }
        double ed[4];
#pragma unroll
        for (int h = 0; h < 4; h++) ed[h] = vx[(base[h] + stride) * 3 + d] - vx[base[h] * 3 + d];
        // (1-p)(1-q) A + (1+p)(1-q) B + (1-p)(1+q) C + (1+p)(1+q) D
        //   = (A+B+C+D) + p (B-A+D-C) + q (C+D-A-B) + p q (A-B-C+D)
        double kv;
        if (w == 0) kv = ed[0] + ed[1] + ed[2] + ed[3];
        else if (w == 1) kv = (ed[1] - ed[0]) + (ed[3] - ed[2]);
        else if (w == 2) kv = (ed[2] + ed[3]) - (ed[0] + ed[1]);
        else kv = (ed[0] - ed[1]) - (ed[2] - ed[3]);
        K[ci] = 0.125 * kv;
    }
    __syncthreads();
    {
        // entry (u, v): X_r at (s_u, t_v), X_s at (r_u, t_v), X_t at (r_u, s_v)
        const double p = sx[u], w2 = sx[v];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            Xr[ab * 3 + d] = fma(w2, fma(p, K[(0 * 4 + 3) * 3 + d], K[(0 * 4 + 2) * 3 + d]),
                                 fma(p, K[(0 * 4 + 1) * 3 + d], K[(0 * 4 + 0) * 3 + d]));
            Xs[ab * 3 + d] = fma(w2, fma(p, K[(1 * 4 + 3) * 3 + d], K[(1 * 4 + 2) * 3 + d]),
                                 fma(p, K[(1 * 4 + 1) * 3 + d], K[(1 * 4 + 0) * 3 + d]));
            Xt[ab * 3 + d] = fma(w2, fma(p, K[(2 * 4 + 3) * 3 + d], K[(2 * 4 + 2) * 3 + d]),
                                 fma(p, K[(2 * 4 + 1) * 3 + d], K[(2 * 4 + 0) * 3 + d]));
        }
    }
    __syncthreads();

    // thread (a, b) = (u, v) walks the c direction
    const int a = u, b = v;
    const double wab = sw[a] * sw[b];
    double xt[3];
#pragma unroll
    for (int d = 0; d < 3; d++) xt[d] = Xt[(a + qn * b) * 3 + d];  // dx/dt at (r_a, s_b)
    double mindet = 1e300;
    double *ge = geo + (valid ? e : 0) * (kind == 1 ? 1 : 7) * (int64_t)QP + ab;
#pragma unroll 1
    for (int c = 0; c < qn; c++) {
        double xr[3], xs[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            xr[d] = Xr[(b + qn * c) * 3 + d];  // dx/dr at (s_b, t_c)
            xs[d] = Xs[(a + qn * c) * 3 + d];  // dx/ds at (r_a, t_c)
        }
        // C_r = X_s x X_t
        const double Cr0 = xs[1] * xt[2] - xs[2] * xt[1];
        const double Cr1 = xs[2] * xt[0] - xs[0] * xt[2];
        const double Cr2 = xs[0] * xt[1] - xs[1] * xt[0];
        const double det = xr[0] * Cr0 + xr[1] * Cr1 + xr[2] * Cr2;
        const double W = wab * sw[c];
        if (MIN) mindet = fmin(mindet, det);
        if (kind == 1) {
            if (valid) ge[c * qq] = W * det;
        } else {
            const double Cs0 = xt[1] * xr[2] - xt[2] * xr[1];
            const double Cs1 = xt[2] * xr[0] - xt[0] * xr[2];
            const double Cs2 = xt[0] * xr[1] - xt[1] * xr[0];
            const double Ct0 = xr[1] * xs[2] - xr[2] * xs[1];
            const double Ct1 = xr[2] * xs[0] - xr[0] * xs[2];
            const double Ct2 = xr[0] * xs[1] - xr[1] * xs[0];
            const double f = W * recip(det);
            if (valid) {
                double *g = ge + c * qq;
                g[0 * QP] = f * (Cr0 * Cr0 + Cr1 * Cr1 + Cr2 * Cr2);
                g[1 * QP] = f * (Cr0 * Cs0 + Cr1 * Cs1 + Cr2 * Cs2);
                g[2 * QP] = f * (Cr0 * Ct0 + Cr1 * Ct1 + Cr2 * Ct2);
                g[3 * QP] = f * (Cs0 * Cs0 + Cs1 * Cs1 + Cs2 * Cs2);
                g[4 * QP] = f * (Cs0 * Ct0 + Cs1 * Ct1 + Cs2 * Ct2);
                g[5 * QP] = f * (Ct0 * Ct0 + Ct1 * Ct1 + Ct2 * Ct2);
                g[6 * QP] = W * det;
                if (kind == 4) wj2[e * (int64_t)QP + c * qq + ab] = W * det;
            }
        }
    }
    if (MIN) {
        sdet[ab] = mindet;
        __syncthreads();
        for (int s = 1; s < qq; s *= 2) {
            if ((ab % (2 * s)) == 0 && ab + s < qq) sdet[ab] = fmin(sdet[ab], sdet[ab + s]);
            __syncthreads();
        }
        if (ab == 0 && valid) detJ_min[e] = sdet[0];
    }
}

// Two resident blocks of about 512 threads per SM (a register cap of 64)
// up to 10 points per direction, measured faster than the compiler's own
// choice; above that the cap would spill.
constexpr int geo_min_blocks(int qn) { return qn <= 10 ? 2 : 0; }

template <int qn, int kind, bool MIN>
__global__ void __launch_bounds__(GeoCfg<qn>::threads)
geofacs_kernel(int64_t E, const double *__restrict__ nodes, const double *__restrict__ weights,
               const double *__restrict__ verts, double *__restrict__ geo, double *__restrict__ detJ_min,
               double *__restrict__ wj2) {
    geofacs_body<qn, kind, MIN>(E, nodes, weights, verts, geo, detJ_min, wj2);
}

template <int qn, int kind, bool MIN>
__global__ void __launch_bounds__(GeoCfg<qn>::threads, geo_min_blocks(qn) > 0 ? geo_min_blocks(qn) : 1)
geofacs_kernel_capped(int64_t E, const double *__restrict__ nodes, const double *__restrict__ weights,
                      const double *__restrict__ verts, double *__restrict__ geo, double *__restrict__ detJ_min,
                      double *__restrict__ wj2) {
    geofacs_body<qn, kind, MIN>(E, nodes, weights, verts, geo, detJ_min, wj2);
}

template <int qn, int kind, bool MIN>
constexpr auto geo_fn() {
    if constexpr (geo_min_blocks(qn) > 0)
        return &geofacs_kernel_capped<qn, kind, MIN>;
    else
        return &geofacs_kernel<qn, kind, MIN>;
}

template <int N>
struct GeoLaunch {
    static cudaError_t run(const fem_basis *b, int kind, int64_t E, const double *verts, double *geo,
                           double *detJ_min, cudaStream_t s) {
        const OpsLayout L{N + 1, N + 2};
        if (kind == FEM_GEO_BP35) {
            using C = GeoCfg<N + 1>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            auto k = detJ_min ? geo_fn<N + 1, 2, true>() : geo_fn<N + 1, 2, false>();
            k<<<(unsigned)blocks, C::threads, C::smem, s>>>(E, b->d_ops + L.offR(), b->d_ops + L.offW(), verts,
                                                            geo, detJ_min, nullptr);
        } else {
            using C = GeoCfg<N + 2>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            const double *x = b->d_ops + L.offRt(), *w = b->d_ops + L.offWt();
            auto k = (kind == FEM_GEO_BP1) ? (detJ_min ? geo_fn<N + 2, 1, true>() : geo_fn<N + 2, 1, false>())
                                           : (detJ_min ? geo_fn<N + 2, 3, true>() : geo_fn<N + 2, 3, false>());
            k<<<(unsigned)blocks, C::threads, C::smem, s>>>(E, x, w, verts, geo, detJ_min, nullptr);
        }
        return cudaGetLastError();
    }
};

template <int N>
struct GeoPairLaunch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *verts, double *G30, double *wJ,
                           cudaStream_t s) {
        const OpsLayout L{N + 1, N + 2};
        using C = GeoCfg<N + 2>;
        const int64_t blocks = (E + C::EPB - 1) / C::EPB;
        geo_fn<N + 2, 4, false>()<<<(unsigned)blocks, C::threads, C::smem, s>>>(
            E, b->d_ops + L.offRt(), b->d_ops + L.offWt(), verts, G30, nullptr, wJ);
        return cudaGetLastError();
    }
};

template <int N>
struct GeoPrepare {
    template <int qn, int kind, bool MIN>
    static cudaError_t one() {
        return cudaFuncSetAttribute(geo_fn<qn, kind, MIN>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    GeoCfg<qn>::smem);
    }
    static cudaError_t run() {
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = one<N + 1, 2, false>();
        if (e == cudaSuccess) e = one<N + 1, 2, true>();
        if (e == cudaSuccess) e = one<N + 2, 1, false>();
        if (e == cudaSuccess) e = one<N + 2, 1, true>();
        if (e == cudaSuccess) e = one<N + 2, 3, false>();
        if (e == cudaSuccess) e = one<N + 2, 3, true>();
        if (e == cudaSuccess) e = one<N + 2, 4, false>();
        return e;
    }
};

}  // namespace

cudaError_t launch_geofacs(const fem_basis *b, int kind, int64_t E, const double *verts, double *geo,
                           double *detJ_min, cudaStream_t s) {
    return dispatch_degree<GeoLaunch>(b->host.N, b, kind, E, verts, geo, detJ_min, s);
}

cudaError_t launch_geofacs_gauss_pair(const fem_basis *b, int64_t E, const double *verts, double *G30, double *wJ,
                                      cudaStream_t s) {
    return dispatch_degree<GeoPairLaunch>(b->host.N, b, E, verts, G30, wJ, s);
}

cudaError_t prepare_geofacs(int N) { return dispatch_degree<GeoPrepare>(N); }

}  // namespace fem
