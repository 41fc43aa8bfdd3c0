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
    static constexpr int smem_elem = (24 + 9 * qq + qq) * 8;
    static constexpr int EPB = pick_epb(qn, smem_elem);
    static constexpr int threads = qq * EPB;
    static constexpr int smem = (2 * pad2(qn) + EPB * pad2(24 + 9 * qq + qq)) * 8;
};

// kind: 1 = wJ only, otherwise 7 planes.
template <int qn, int kind>
__global__ void __launch_bounds__(GeoCfg<qn>::threads)
geofacs_kernel(int64_t E, const double *__restrict__ nodes, const double *__restrict__ weights,
               const double *__restrict__ verts, double *__restrict__ geo,
               double *__restrict__ detJ_min) {
    using C = GeoCfg<qn>;
    constexpr int QP = C::QP, qq = C::qq, EPB = C::EPB;
    constexpr int PER = pad2(24 + 9 * qq + qq);
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

    // tabulate the three column tables of X: with x = sum_c x_c phi_c,
    // dx/dr = 1/8 sum_c x_c sr_c (1 + ss_c s)(1 + st_c t), etc.
    {
        const double p = sx[u], w2 = sx[v];
        double cr[3] = {0, 0, 0}, cs[3] = {0, 0, 0}, ct[3] = {0, 0, 0};
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const double sr = (c & 1) ? 1.0 : -1.0, ss = (c & 2) ? 1.0 : -1.0, st = (c & 4) ? 1.0 : -1.0;
            // X_r at (s = p, t = w2); X_s at (r = p, t = w2); X_t at (r = p, s = w2)
            const double fr = sr * (1.0 + ss * p) * (1.0 + st * w2);
            const double fs = ss * (1.0 + sr * p) * (1.0 + st * w2);
            const double ft = st * (1.0 + sr * p) * (1.0 + ss * w2);
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const double xc = vx[c * 3 + d];
                cr[d] = fma(xc, fr, cr[d]);
                cs[d] = fma(xc, fs, cs[d]);
                ct[d] = fma(xc, ft, ct[d]);
            }
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            Xr[ab * 3 + d] = 0.125 * cr[d];
            Xs[ab * 3 + d] = 0.125 * cs[d];
            Xt[ab * 3 + d] = 0.125 * ct[d];
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
        mindet = fmin(mindet, det);
        if (kind == 1) {
            if (valid) ge[c * qq] = W * det;
        } else {
            const double Cs0 = xt[1] * xr[2] - xt[2] * xr[1];
            const double Cs1 = xt[2] * xr[0] - xt[0] * xr[2];
            const double Cs2 = xt[0] * xr[1] - xt[1] * xr[0];
            const double Ct0 = xr[1] * xs[2] - xr[2] * xs[1];
            const double Ct1 = xr[2] * xs[0] - xr[0] * xs[2];
            const double Ct2 = xr[0] * xs[1] - xr[1] * xs[0];
            const double f = W / det;
            if (valid) {
                double *g = ge + c * qq;
                g[0 * QP] = f * (Cr0 * Cr0 + Cr1 * Cr1 + Cr2 * Cr2);
                g[1 * QP] = f * (Cr0 * Cs0 + Cr1 * Cs1 + Cr2 * Cs2);
                g[2 * QP] = f * (Cr0 * Ct0 + Cr1 * Ct1 + Cr2 * Ct2);
                g[3 * QP] = f * (Cs0 * Cs0 + Cs1 * Cs1 + Cs2 * Cs2);
                g[4 * QP] = f * (Cs0 * Ct0 + Cs1 * Ct1 + Cs2 * Ct2);
                g[5 * QP] = f * (Ct0 * Ct0 + Ct1 * Ct1 + Ct2 * Ct2);
                g[6 * QP] = W * det;
            }
        }
    }
    if (detJ_min) {
        sdet[ab] = mindet;
        __syncthreads();
        for (int s = 1; s < qq; s *= 2) {
            if ((ab % (2 * s)) == 0 && ab + s < qq) sdet[ab] = fmin(sdet[ab], sdet[ab + s]);
            __syncthreads();
        }
        if (ab == 0 && valid) detJ_min[e] = sdet[0];
    }
}

template <int N>
struct GeoLaunch {
    static cudaError_t run(const fem_basis *b, int kind, int64_t E, const double *verts, double *geo,
                           double *detJ_min, cudaStream_t s) {
        const OpsLayout L{N + 1, N + 2};
        if (kind == FEM_GEO_BP35) {
            using C = GeoCfg<N + 1>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            geofacs_kernel<N + 1, 2><<<(unsigned)blocks, C::threads, C::smem, s>>>(
                E, b->d_ops + L.offR(), b->d_ops + L.offW(), verts, geo, detJ_min);
        } else {
            using C = GeoCfg<N + 2>;
            const int64_t blocks = (E + C::EPB - 1) / C::EPB;
            const double *x = b->d_ops + L.offRt(), *w = b->d_ops + L.offWt();
            if (kind == FEM_GEO_BP1)
                geofacs_kernel<N + 2, 1><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, x, w, verts, geo, detJ_min);
            else
                geofacs_kernel<N + 2, 3><<<(unsigned)blocks, C::threads, C::smem, s>>>(E, x, w, verts, geo, detJ_min);
        }
        return cudaGetLastError();
    }
};

template <int N>
struct GeoPrepare {
    static cudaError_t run() {
        cudaError_t err = cudaFuncSetAttribute(geofacs_kernel<N + 1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               GeoCfg<N + 1>::smem);
        if (err != cudaSuccess) return err;
        err = cudaFuncSetAttribute(geofacs_kernel<N + 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   GeoCfg<N + 2>::smem);
        if (err != cudaSuccess) return err;
        return cudaFuncSetAttribute(geofacs_kernel<N + 2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    GeoCfg<N + 2>::smem);
    }
};

}  // namespace

cudaError_t launch_geofacs(const fem_basis *b, int kind, int64_t E, const double *verts, double *geo,
                           double *detJ_min, cudaStream_t s) {
    return dispatch_degree<GeoLaunch>(b->host.N, b, kind, E, verts, geo, detJ_min, s);
}

cudaError_t prepare_geofacs(int N) { return dispatch_degree<GeoPrepare>(N); }

}  // namespace fem
