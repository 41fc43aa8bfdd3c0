// Jacobi-preconditioned conjugate gradients (Saad, "Iterative Methods for
// Sparse Linear Systems", Algorithm 9.1, M = diag A) for the unassembled
// BP3.5 screened-Poisson system S u + lambda M u = f of Section 4, in two
// modes:
//   FP64   all-FP64 PCG;
//   mixed  FP64 defect correction (iterative refinement): the residual
//          b - A x, its norm, the dot products and the solution update stay
//          in FP64, while each correction equation A d = r is solved to a
//          loose tolerance by an FP32 PCG whose matvec reads FP32 geometric
//          factors (FEM_PCG_MIXED), FP16 factors (FEM_PCG_MIXED16), or FP32
//          factors with the contractions on the tensor cores
//          (FEM_PCG_MIXED_TC).
//
// Device-resident state: every scalar of the recurrence (rho, p.Ap, alpha,
// beta, ||r||^2, convergence and breakdown flags, the iteration count) lives
// in device memory and is produced by deterministic single-block
// reductions, so the host reads back a few scalars only every few
// iterations.  One iteration is four launches: the BP3.5 matvec fused with
// p <- z + beta p and the p.Ap partial sums, a reduction, the fused update
// x += alpha p, r -= alpha Ap, z = r / diag with the r.z and r.r partial
// sums, and a reduction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "fem_internal.h"
#include "kernels_common.cuh"

namespace fem {

enum {
    S_RHO = 0,   // r . z of the current iterate
    S_PQ,        // p . Ap
    S_ALPHA,
    S_BETA,
    S_RR,        // r . r (of the solver in progress)
    S_BB,        // b . b
    S_TOL2,      // squared absolute stopping threshold on r . r
    S_DONE,      // 1 once r . r <= S_TOL2 (further iterations are frozen)
    S_BREAK,     // 1 on p . Ap <= 0 or a non-finite value
    S_ITER,      // iterations completed
    S_RR_OUTER,  // FP64 residual norm^2 of the defect-correction loop
    S_GMAX,      // FEM_PCG_MIXED16: largest |factor| (bits of a non-negative double)
    S_GINV,      // FEM_PCG_MIXED16: inverse of the FP16 factor scale
    S_WAITFAIL,  // set to 1 by a kernel whose bounded device wait gave up
    S_COUNT
};

constexpr int kVecBlocks = 152 * 8;  // grid of the vector kernels (grid-stride)
constexpr int kVecThreads = 256;
constexpr int kRedThreads = 1024;

namespace {

// ------------------------------------------------------------------ kernels

template <int N>
__global__ void __launch_bounds__(256)
bp35_dinv_kernel(int64_t E, const double *__restrict__ ops, const double *__restrict__ G, double lambda,
                 double *__restrict__ dinv, float *__restrict__ dinv32) {
    constexpr int n = N + 1, NP = n * n * n;
    __shared__ double sD[n * n];
    const OpsLayout L{n, n + 1};
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = ops[L.offD() + t];
    __syncthreads();
    const int64_t total = E * NP;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = g / NP;
        const int p = (int)(g - e * NP), i = p % n, j = (p / n) % n, k = p / (n * n);
        const double *Ge = G + e * 7 * NP;
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < n; l++) {
            const double a = sD[l * n + i], b = sD[l * n + j], c = sD[l * n + k];
            s = fma(a * a, Ge[0 * NP + l + n * (j + n * k)], s);
            s = fma(b * b, Ge[3 * NP + i + n * (l + n * k)], s);
            s = fma(c * c, Ge[5 * NP + i + n * (j + n * l)], s);
        }
        const double Di = sD[i * n + i], Dj = sD[j * n + j], Dk = sD[k * n + k];
        s += 2.0 * (Di * Dj * Ge[1 * NP + p] + Di * Dk * Ge[2 * NP + p] + Dj * Dk * Ge[4 * NP + p]);
        s += lambda * Ge[6 * NP + p];
        const double v = 1.0 / s;
        if (dinv) dinv[g] = v;
        if (dinv32) dinv32[g] = (float)v;
    }
}

// Inverse diagonal of the BP3.0 operator I^T (Dt^T G Dt + lambda J) I.  With
// B = I and C = Dt I (m x n), the gradient of basis function (i,j,k) at Gauss
// point (a,b,c) is (C_ai B_bj B_ck, B_ai C_bj B_ck, B_ai B_bj C_ck), so the
// diagonal is a sum of seven sum-factorised projections
//   sum_abc X_ai Y_bj Z_ck F_abc,  X, Y, Z in {P = B*B, Q = C*C, R = B*C}
// (elementwise products) of the factor planes F.  One element per block
// (grid-stride), FP64.
template <int N>
__global__ void __launch_bounds__(256)
bp30_dinv_kernel(int64_t E, const double *__restrict__ ops, const double *__restrict__ G, double lambda,
                 double *__restrict__ dinv, float *__restrict__ dinv32) {
    constexpr int n = N + 1, m = N + 2, NP = n * n * n, MP = m * m * m, mn = m * n;
    extern __shared__ double sm[];
    double *sP = sm, *sQ = sP + mn, *sR = sQ + mn;
    double *F = sR + mn, *T1 = F + MP, *T2 = T1 + m * m * n;
    const OpsLayout L{n, m};
    for (int t = threadIdx.x; t < mn; t += blockDim.x) {
        const double b = ops[L.offI() + t], c = ops[L.offC() + t];
        sP[t] = b * b;
        sQ[t] = c * c;
        sR[t] = b * c;
    }
    // terms: X (along r), Y (along s), Z (along t), factor plane, coefficient
    const double *X[7] = {sQ, sP, sP, sR, sR, sP, sP};
    const double *Y[7] = {sP, sQ, sP, sR, sP, sR, sP};
    const double *Z[7] = {sP, sP, sQ, sP, sR, sR, sP};
    const int plane[7] = {0, 3, 5, 1, 2, 4, 6};
    const double coef[7] = {1.0, 1.0, 1.0, 2.0, 2.0, 2.0, lambda};
    const int jk = threadIdx.x, j = jk % n, k = jk / n;  // output line (j, k), i along it
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        double out[n];
#pragma unroll
        for (int i = 0; i < n; i++) out[i] = 0.0;
        for (int term = 0; term < 7; term++) {
            __syncthreads();
            const double *Fe = G + (e * 7 + plane[term]) * MP;
            for (int t = threadIdx.x; t < MP; t += blockDim.x) F[t] = Fe[t];
            __syncthreads();
            // T1[a][b][k] = sum_c Z_ck F[a][b][c]
            for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
                const int a = t % m, b = t / m;
                for (int kk = 0; kk < n; kk++) {
                    double acc = 0.0;
                    for (int c = 0; c < m; c++) acc = fma(Z[term][c * n + kk], F[a + m * (b + m * c)], acc);
                    T1[a + m * (b + m * kk)] = acc;
                }
            }
            __syncthreads();
            // T2[a][j][k] = sum_b Y_bj T1[a][b][k]
            for (int t = threadIdx.x; t < m * n; t += blockDim.x) {
                const int a = t % m, kk = t / m;
                for (int jj = 0; jj < n; jj++) {
                    double acc = 0.0;
                    for (int b = 0; b < m; b++) acc = fma(Y[term][b * n + jj], T1[a + m * (b + m * kk)], acc);
                    T2[a + m * (jj + n * kk)] = acc;
                }
            }
            __syncthreads();
            if (jk < n * n) {
#pragma unroll
                for (int i = 0; i < n; i++) {
                    double acc = 0.0;
                    for (int a = 0; a < m; a++) acc = fma(X[term][a * n + i], T2[a + m * (j + n * k)], acc);
                    out[i] = fma(coef[term], acc, out[i]);
                }
            }
        }
        if (jk < n * n) {
#pragma unroll
            for (int i = 0; i < n; i++) {
                const int64_t g = e * NP + i + n * (j + n * k);
                const double v = 1.0 / out[i];
                if (dinv) dinv[g] = v;
                if (dinv32) dinv32[g] = (float)v;
            }
        }
    }
}

template <int N>
constexpr int bp30_dinv_smem() {
    return (3 * (N + 2) * (N + 1) + (N + 2) * (N + 2) * (N + 2) + (N + 2) * (N + 2) * (N + 1) +
            (N + 2) * (N + 1) * (N + 1)) *
           8;
}

__global__ void __launch_bounds__(kVecThreads) cast_f32_kernel(int64_t n, const double *__restrict__ a,
                                                               float *__restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// FP16 factors: the largest |a| (atomic maximum on the bit pattern, which
// orders non-negative doubles like their values) ...
__global__ void __launch_bounds__(kVecThreads) absmax_kernel(int64_t n, const double *__restrict__ a,
                                                             unsigned long long *__restrict__ out) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ... then a[i] * s rounded to binary16 with s = 2^(14 - e), max|a| < 2^e:
// the largest factor lands in [2^13, 2^14), far from the binary16 overflow
// (65504), and the small off-diagonal factors stay normal numbers.  The
// inverse 1/s goes to *ginv for the operator kernels.
__global__ void __launch_bounds__(kVecThreads) cast_f16_kernel(int64_t n, const double *__restrict__ a,
                                                               __half *__restrict__ b,
                                                               const unsigned long long *__restrict__ gmax,
                                                               double *__restrict__ ginv) {
    const double mx = __longlong_as_double((long long)*gmax);
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);  // mx = f 2^ex, f in [0.5, 1)
    const double sc = ldexp(1.0, 14 - ex);
    if (blockIdx.x == 0 && threadIdx.x == 0) *ginv = ldexp(1.0, ex - 14);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __double2half(a[i] * sc);
}

// partial sums of x . y per block (grid-stride, fixed order)
__global__ void __launch_bounds__(kVecThreads) dot_kernel(int64_t n, const double *__restrict__ x,
                                                          const double *__restrict__ y, double *__restrict__ part) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(x[i], y[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// FP64 PCG start: r = b - Ax, z = dinv r; partials (r.z, r.r)
__global__ void __launch_bounds__(kVecThreads)
init_kernel(int64_t n, const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ r,
            double *__restrict__ z, const double *__restrict__ dinv, double *__restrict__ part) {
    __shared__ double sh[32];
    double rz = 0.0, rr = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - Ax[i], zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        rz = fma(ri, zi, rz);
        rr = fma(ri, ri, rr);
    }
    rz = block_sum(rz, sh);
    __syncthreads();
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = rz;
        part[2 * blockIdx.x + 1] = rr;
    }
}

// Defect-correction step: r64 = b - Ax (FP64), r = (float) r64, z = dinv r,
// d = 0; partials (r.z, r.r, r64.r64)
__global__ void __launch_bounds__(kVecThreads)
outer_kernel(int64_t n, const double *__restrict__ b, const double *__restrict__ Ax, float *__restrict__ r,
             float *__restrict__ z, float *__restrict__ d, const float *__restrict__ dinv, double *__restrict__ part) {
    __shared__ double sh[32];
    double rz = 0.0, rr = 0.0, r64 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - Ax[i];
        const float rf = (float)ri, zf = dinv[i] * rf;
        r[i] = rf;
        z[i] = zf;
        d[i] = 0.0f;
        rz = fma((double)rf, (double)zf, rz);
        rr = fma((double)rf, (double)rf, rr);
        r64 = fma(ri, ri, r64);
    }
    rz = block_sum(rz, sh);
    __syncthreads();
    rr = block_sum(rr, sh);
    __syncthreads();
    r64 = block_sum(r64, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = rz;
        part[3 * blockIdx.x + 1] = rr;
        part[3 * blockIdx.x + 2] = r64;
    }
}

// x += alpha p, r -= alpha Ap, z = dinv r; partials (r.z, r.r).  The
// arithmetic is in the recurrence's own precision T (in FP32 the per-thread
// partial sums too, so the FP32 inner solver issues no FP64 instruction per
// entry); the per-block sums are FP64.
template <typename T, typename XT>
__global__ void __launch_bounds__(kVecThreads)
update_kernel(int64_t n, const double *__restrict__ scal, XT *__restrict__ x, const T *__restrict__ p,
              T *__restrict__ r, const T *__restrict__ Ap, T *__restrict__ z, const T *__restrict__ dinv,
              double *__restrict__ part) {
    __shared__ double sh[32];
    const double alpha = scal[S_ALPHA];
    const T a = (T)alpha;
    T rz = T(0), rr = T(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T ri = r[i];
        if (alpha != 0.0) {
            x[i] = fmx((XT)a, (XT)p[i], x[i]);
            ri = ri - a * Ap[i];
            r[i] = ri;
        }
        const T zi = dinv[i] * ri;
        z[i] = zi;
        rz = fmx(ri, zi, rz);
        rr = fmx(ri, ri, rr);
    }
    double drz = block_sum((double)rz, sh);
    __syncthreads();
    double drr = block_sum((double)rr, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = drz;
        part[2 * blockIdx.x + 1] = drr;
    }
}

// The FP32 update with 16-byte vector accesses (n a multiple of 4, every
// array 16-byte aligned): four entries per thread and iteration.
__global__ void __launch_bounds__(kVecThreads)
update_f32x4_kernel(int64_t n4, const double *__restrict__ scal, float4 *__restrict__ x, const float4 *__restrict__ p,
                    float4 *__restrict__ r, const float4 *__restrict__ Ap, float4 *__restrict__ z,
                    const float4 *__restrict__ dinv, double *__restrict__ part) {
    __shared__ double sh[32];
    const double alpha = scal[S_ALPHA];
    const float a = (float)alpha;
    float rz = 0.0f, rr = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 ri = r[i];
        const float4 di = dinv[i];
        if (alpha != 0.0) {
            const float4 pi = p[i], qi = Ap[i];
            float4 xi = x[i];
            xi.x += a * pi.x; xi.y += a * pi.y; xi.z += a * pi.z; xi.w += a * pi.w;
            x[i] = xi;
            ri.x -= a * qi.x; ri.y -= a * qi.y; ri.z -= a * qi.z; ri.w -= a * qi.w;
            r[i] = ri;
        }
        const float4 zi = make_float4(di.x * ri.x, di.y * ri.y, di.z * ri.z, di.w * ri.w);
        z[i] = zi;
        rz += ri.x * zi.x + ri.y * zi.y + ri.z * zi.z + ri.w * zi.w;
        rr += ri.x * ri.x + ri.y * ri.y + ri.z * ri.z + ri.w * ri.w;
    }
    double drz = block_sum((double)rz, sh);
    __syncthreads();
    double drr = block_sum((double)rr, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = drz;
        part[2 * blockIdx.x + 1] = drr;
    }
}

// x (FP64) += d (FP32)
__global__ void __launch_bounds__(kVecThreads) add_f32_kernel(int64_t n, double *__restrict__ x,
                                                              const float *__restrict__ d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

enum RedMode { R_SUM = 0, R_PQ, R_RZ, R_INIT, R_OUTER };

// Single-block reduction of `nparts` records of `stride` partial sums and
// the scalar logic of the recurrence.
__global__ void __launch_bounds__(kRedThreads)
reduce_kernel(int mode, int64_t nparts, const double *__restrict__ part, double *__restrict__ scal,
              double *__restrict__ out, double tol2_rel, double floor2_rel = 0.0) {
    __shared__ double sh[32];
    const int stride = (mode == R_OUTER) ? 3 : (mode == R_RZ || mode == R_INIT) ? 2 : 1;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < nparts; i += blockDim.x)
        for (int c = 0; c < stride; c++) acc[c] += part[i * stride + c];
    double tot[3];
    for (int c = 0; c < stride; c++) {
        tot[c] = block_sum(acc[c], sh);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if (mode == R_SUM) {
        *out = tot[0];
    } else if (mode == R_PQ) {
        const double pq = tot[0];
        scal[S_PQ] = pq;
        double alpha = 0.0;
        if (scal[S_DONE] == 0.0 && scal[S_BREAK] == 0.0) {
            if (pq > 0.0 && isfinite(pq))
                alpha = scal[S_RHO] / pq;
            else
                scal[S_BREAK] = 1.0;
        }
        scal[S_ALPHA] = alpha;
    } else if (mode == R_RZ) {
        const bool active = scal[S_DONE] == 0.0 && scal[S_BREAK] == 0.0;
        const double rz = tot[0], rr = tot[1];
        scal[S_BETA] = (scal[S_RHO] != 0.0) ? rz / scal[S_RHO] : 0.0;
        scal[S_RHO] = rz;
        scal[S_RR] = rr;
        if (active) {
            scal[S_ITER] += 1.0;
            if (!isfinite(rr))
                scal[S_BREAK] = 1.0;
            else if (rr <= scal[S_TOL2])
                scal[S_DONE] = 1.0;
        }
    } else {  // R_INIT, R_OUTER: start of a PCG run
        scal[S_RHO] = tot[0];
        scal[S_RR] = tot[1];
        scal[S_BETA] = 0.0;
        scal[S_ITER] = 0.0;
        scal[S_BREAK] = 0.0;
        // R_OUTER: the inner solve reduces the defect by inner_tol, but need
        // not go below the floor floor2_rel * b.b (a fraction of the outer
        // tolerance): the last defect-correction step then stops as soon as
        // the outer target is in reach instead of over-solving
        scal[S_TOL2] = (mode == R_INIT) ? tol2_rel * scal[S_BB] : fmax(tol2_rel * tot[1], floor2_rel * scal[S_BB]);
        scal[S_DONE] = (tot[1] <= scal[S_TOL2]) ? 1.0 : 0.0;
        if (mode == R_OUTER) scal[S_RR_OUTER] = tot[2];
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers used by the ABI

template <int N>
struct DinvLaunch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda, double *dinv, float *dinv32,
                           cudaStream_t s) {
        const int64_t total = E * (int64_t)(N + 1) * (N + 1) * (N + 1);
        int64_t blocks = (total + 255) / 256;
        if (blocks > 152 * 32) blocks = 152 * 32;
        bp35_dinv_kernel<N><<<(unsigned)blocks, 256, 0, s>>>(E, b->d_ops, G, lambda, dinv, dinv32);
        return cudaGetLastError();
    }
};

template <int N>
struct Dinv30Launch {
    static cudaError_t run(const fem_basis *b, int64_t E, const double *G, double lambda, double *dinv, float *dinv32,
                           cudaStream_t s) {
        constexpr int smem = bp30_dinv_smem<N>();
        cudaError_t e = cudaFuncSetAttribute(bp30_dinv_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        const int64_t blocks = E < 152 * 4 ? E : 152 * 4;
        bp30_dinv_kernel<N><<<(unsigned)blocks, 256, smem, s>>>(E, b->d_ops, G, lambda, dinv, dinv32);
        return cudaGetLastError();
    }
};

int64_t dot_scratch_size() { return kVecBlocks; }

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *result, double *scratch,
                       cudaStream_t s) {
    dot_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(n, x, y, scratch);
    reduce_kernel<<<1, kRedThreads, 0, s>>>(R_SUM, kVecBlocks, scratch, nullptr, result, 0.0);
    return cudaGetLastError();
}

}  // namespace fem

// ---------------------------------------------------------------------- solver context

namespace fem {
enum PcgState { PS_IDLE = 0, PS_BB, PS_RUN64, PS_FINAL64, PS_OUTER, PS_INNER, PS_DONE };
}  // namespace fem

struct fem_pcg {
    const fem_basis *basis;
    int op;        // FEM_OP_BP35 or FEM_OP_BP30
    int64_t gpts;  // factor points per element (n^3 or m^3)
    int64_t E, len;
    const double *G;
    double lambda;
    int mode;
    int device;
    double *r, *z, *p, *q, *dinv;                   // FP64 recurrence (q also holds A x)
    float *G32, *dinv32, *d32, *r32, *z32, *p32, *q32;  // FP32 inner recurrence (mixed mode)
    __half *G16;                                        // FP16 factors (FEM_PCG_MIXED16)
    double *part;
    int64_t nparts;
    double *scal;       // device scalars
    double *hscal;      // pinned host copy
    bool own_hscal;     // allocated here (not lent by a server)
    cudaStream_t ws;    // stream the workspace was allocated on
    // resumable solve
    cudaEvent_t ev;
    int state;
    bool pending;
    const double *b;
    double *x;
    cudaStream_t st;
    double tol, itol, bb;
    int maxit, imaxit, every, chunk_done, inner_iters, outer, status;
    int restarts;       // FP64: residual replacements so far
    double restart_rr;  // FP64: true residual norm^2 at the last replacement
    fem_pcg_info info;
    // CUDA graphs of one full chunk of iterations (and of the outer
    // defect-correction step), captured on first use and replayed
    cudaGraphExec_t g_iter64, g_iter32, g_outer;
    int g_every;                   // chunk length the iteration graphs were captured with
    const double *g_b;             // right-hand side and solution the graphs were captured with
    double *g_x;
    double g_tol, g_itol;          // and the tolerances
    bool use_graphs;               // not on the legacy default stream, which cannot be captured
    bool wait_fault_armed;         // host-side fault injection (fem_pcg_inject_fault)
};

namespace fem {

cudaError_t launch_bp35_pcg(const fem_basis *b, int64_t E, const double *G, double lambda, const double *z,
                            double *p, const double *beta, double *Ap, double *partials, cudaStream_t s);
cudaError_t launch_bp35_pcg_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                float *p, const double *beta, float *Ap, double *partials, cudaStream_t s,
                                double *status);
int64_t bp35_max_blocks(int N, int64_t E);
int64_t bp35_blocks(int N, int64_t E, bool f32);
cudaError_t launch_bp35(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q, double *Aq,
                        cudaStream_t s);

namespace {

// Operator dispatch of the solver.
cudaError_t op_apply64(fem_pcg *s, const double *x, double *out, cudaStream_t st) {
    return s->op == FEM_OP_BP30 ? launch_bp30(s->basis, s->E, s->G, s->lambda, x, out, st)
                                : launch_bp35(s->basis, s->E, s->G, s->lambda, x, out, st);
}
int64_t op_blocks(const fem_pcg *s, bool f32) {
    if (f32 && s->mode == FEM_PCG_MIXED_TC) return s->E;  // one block per element
    if (f32 && s->mode == FEM_PCG_MIXED16)
        return s->op == FEM_OP_BP30 ? bp30_f16_blocks(s->basis->host.N, s->E) : bp35_f16_blocks(s->basis->host.N, s->E);
    return s->op == FEM_OP_BP30 ? bp30_blocks(s->basis->host.N, s->E, f32) : bp35_blocks(s->basis->host.N, s->E, f32);
}
cudaError_t op_pcg(fem_pcg *s, const double *G, const double *z, double *p, double *Ap, cudaStream_t st) {
    return s->op == FEM_OP_BP30
               ? launch_bp30_pcg(s->basis, s->E, G, s->lambda, z, p, s->scal + S_BETA, Ap, s->part, st)
               : launch_bp35_pcg(s->basis, s->E, G, s->lambda, z, p, s->scal + S_BETA, Ap, s->part, st);
}
cudaError_t op_pcg(fem_pcg *s, const float *G, const float *z, float *p, float *Ap, cudaStream_t st) {
    if (s->mode == FEM_PCG_MIXED_TC)
        return s->op == FEM_OP_BP30
                   ? launch_bp30_pcg_tc(s->basis, s->E, G, s->lambda, z, p, s->scal + S_BETA, Ap, s->part, st)
                   : launch_bp35_pcg_tc(s->basis, s->E, G, s->lambda, z, p, s->scal + S_BETA, Ap, s->part, st);
    if (s->mode == FEM_PCG_MIXED16)
        return s->op == FEM_OP_BP30 ? launch_bp30_pcg_f16g(s->basis, s->E, s->G16, s->scal + S_GINV, s->lambda, z, p,
                                                           s->scal + S_BETA, Ap, s->part, st, s->scal + S_WAITFAIL)
                                    : launch_bp35_pcg_f16g(s->basis, s->E, s->G16, s->scal + S_GINV, s->lambda, z, p,
                                                           s->scal + S_BETA, Ap, s->part, st, s->scal + S_WAITFAIL);
    return s->op == FEM_OP_BP30
               ? launch_bp30_pcg_f32(s->basis, s->E, G, s->lambda, z, p, s->scal + S_BETA, Ap, s->part, st,
                                     s->scal + S_WAITFAIL)
               : launch_bp35_pcg_f32(s->basis, s->E, G, s->lambda, z, p, s->scal + S_BETA, Ap, s->part, st,
                                     s->scal + S_WAITFAIL);
}

template <typename P>
cudaError_t alloc(P **ptr, int64_t count, cudaStream_t st) {
    return cudaMallocAsync((void **)ptr, sizeof(P) * (size_t)(count > 0 ? count : 1), st);
}

// Enqueues the scalar read-back and the event that marks the end of a step.
cudaError_t end_step(fem_pcg *s) {
    cudaError_t e = cudaMemcpyAsync(s->hscal, s->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->st);
    s->pending = (e == cudaSuccess);
    return e;
}

// Enqueues up to `chunk` PCG iterations on (x, p, r, Ap, z).
template <typename T, typename XT>
cudaError_t enqueue_iterations(fem_pcg *s, const T *G, XT *x, T *p, T *r, T *Ap, T *z, const T *dinv, int chunk) {
    cudaError_t e = cudaSuccess;
    const int64_t len = s->len;
    for (int c = 0; c < chunk && e == cudaSuccess; c++) {
        e = op_pcg(s, G, z, p, Ap, s->st);
        if (e != cudaSuccess) break;
        reduce_kernel<<<1, kRedThreads, 0, s->st>>>(R_PQ, op_blocks(s, sizeof(T) == 4), s->part, s->scal, nullptr,
                                                    0.0);
        if (sizeof(T) == 4 && sizeof(XT) == 4 && len % 4 == 0)
            update_f32x4_kernel<<<kVecBlocks, kVecThreads, 0, s->st>>>(
                len / 4, s->scal, (float4 *)x, (const float4 *)p, (float4 *)r, (const float4 *)Ap, (float4 *)z,
                (const float4 *)dinv, s->part);
        else
            update_kernel<T, XT><<<kVecBlocks, kVecThreads, 0, s->st>>>(len, s->scal, x, p, r, Ap, z, dinv, s->part);
        reduce_kernel<<<1, kRedThreads, 0, s->st>>>(R_RZ, kVecBlocks, s->part, s->scal, nullptr, 0.0);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t outer_body(fem_pcg *s) {
    cudaError_t e = op_apply64(s, s->x, s->q, s->st);
    if (e != cudaSuccess) return e;
    outer_kernel<<<kVecBlocks, kVecThreads, 0, s->st>>>(s->len, s->b, s->q, s->r32, s->z32, s->d32, s->dinv32, s->part);
    reduce_kernel<<<1, kRedThreads, 0, s->st>>>(R_OUTER, kVecBlocks, s->part, s->scal, nullptr, s->itol * s->itol,
                                                0.25 * s->tol * s->tol);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->hscal, s->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s->st);
    return e;
}

__global__ void set_scalar_kernel(double *p, double v) { *p = v; }

// Host-side fault injection: writes the wait-failure word exactly as a
// kernel whose bounded wait gave up would, once, before the first chunk.
cudaError_t inject_armed_fault(fem_pcg *s) {
    if (!s->wait_fault_armed) return cudaSuccess;
    s->wait_fault_armed = false;
    set_scalar_kernel<<<1, 1, 0, s->st>>>(s->scal + S_WAITFAIL, 1.0);
    return cudaGetLastError();
}

// Captures whatever `body` enqueues on s->st into an executable graph.
template <class F>
cudaError_t capture(fem_pcg *s, cudaGraphExec_t *exec, F body) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t be = body();
    e = cudaStreamEndCapture(s->st, &g);
    if (be != cudaSuccess) e = be;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

cudaError_t enqueue_outer(fem_pcg *s) {
    cudaError_t e = cudaSuccess;
    if (!s->use_graphs) {
        e = outer_body(s);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->st);
        s->pending = (e == cudaSuccess);
        return e;
    }
    if (!s->g_outer) e = capture(s, &s->g_outer, [&] { return outer_body(s); });
    if (e == cudaSuccess) e = cudaGraphLaunch(s->g_outer, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->st);
    s->pending = (e == cudaSuccess);
    return e;
}

// A chunk of iterations followed by the scalar read-back and the event; a
// full chunk replays its captured graph.
template <typename T, typename XT>
cudaError_t enqueue_chunk(fem_pcg *s, const T *G, XT *x, T *p, T *r, T *Ap, T *z, const T *dinv, int chunk) {
    cudaError_t e = cudaSuccess;
    cudaGraphExec_t *g = sizeof(T) == 8 ? &s->g_iter64 : &s->g_iter32;
    if (chunk == s->every && s->use_graphs) {
        if (*g && s->g_every != s->every) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
        if (!*g) {
            e = capture(s, g, [&] {
                cudaError_t ce = enqueue_iterations<T, XT>(s, G, x, p, r, Ap, z, dinv, chunk);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(s->hscal, s->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s->st);
                return ce;
            });
            s->g_every = s->every;
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(*g, s->st);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->st);
        s->pending = (e == cudaSuccess);
        return e;
    }
    e = enqueue_iterations<T, XT>(s, G, x, p, r, Ap, z, dinv, chunk);
    if (e == cudaSuccess) e = end_step(s);
    return e;
}

int next_chunk(const fem_pcg *s, int done, int limit) {
    int c = s->every;
    if (c > limit - done) c = limit - done;
    return c > 0 ? c : 0;
}

}  // namespace

// Allocates the workspace on stream st (stream-ordered, no device-wide
// synchronisation) and enqueues the Jacobi diagonal and the FP32 factor copy.
cudaError_t pcg_create_on(fem_pcg *s, cudaStream_t st, double *lent_hscal) {
    cudaError_t e = cudaSuccess;
    const int64_t len = s->len;
    s->ws = st;
    s->nparts = std::max(op_blocks(s, false), op_blocks(s, true));
    if (s->nparts < 3 * (int64_t)kVecBlocks) s->nparts = 3 * (int64_t)kVecBlocks;
    if (e == cudaSuccess) e = alloc(&s->part, 3 * s->nparts, st);
    if (e == cudaSuccess) e = alloc(&s->scal, S_COUNT, st);
    if (e == cudaSuccess) e = alloc(&s->q, len, st);
    if (s->mode == FEM_PCG_FP64) {
        if (e == cudaSuccess) e = alloc(&s->r, len, st);
        if (e == cudaSuccess) e = alloc(&s->z, len, st);
        if (e == cudaSuccess) e = alloc(&s->p, len, st);
        if (e == cudaSuccess) e = alloc(&s->dinv, len, st);
    } else {
        if (s->mode == FEM_PCG_MIXED16) {
            if (e == cudaSuccess) e = alloc(&s->G16, 7 * s->E * s->gpts, st);
        } else {
            if (e == cudaSuccess) e = alloc(&s->G32, 7 * s->E * s->gpts, st);
        }
        if (e == cudaSuccess) e = alloc(&s->dinv32, len, st);
        if (e == cudaSuccess) e = alloc(&s->d32, len, st);
        if (e == cudaSuccess) e = alloc(&s->r32, len, st);
        if (e == cudaSuccess) e = alloc(&s->z32, len, st);
        if (e == cudaSuccess) e = alloc(&s->p32, len, st);
        if (e == cudaSuccess) e = alloc(&s->q32, len, st);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        if (lent_hscal) {
            s->hscal = lent_hscal;
            s->own_hscal = false;
        } else {
            e = cudaMallocHost((void **)&s->hscal, sizeof(double) * S_COUNT);
            s->own_hscal = (e == cudaSuccess);
        }
    }
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s->scal, 0, sizeof(double) * S_COUNT, st);
    if (e != cudaSuccess) return e;
    if (s->op == FEM_OP_BP30)
        e = dispatch_degree<Dinv30Launch>(s->basis->host.N, s->basis, s->E, s->G, s->lambda, s->dinv, s->dinv32, st);
    else
        e = dispatch_degree<DinvLaunch>(s->basis->host.N, s->basis, s->E, s->G, s->lambda, s->dinv, s->dinv32, st);
    if (e == cudaSuccess && (s->mode == FEM_PCG_MIXED || s->mode == FEM_PCG_MIXED_TC))
        cast_f32_kernel<<<kVecBlocks, kVecThreads, 0, st>>>(7 * s->E * s->gpts, s->G, s->G32);
    if (e == cudaSuccess && s->mode == FEM_PCG_MIXED16) {
        unsigned long long *gmax = reinterpret_cast<unsigned long long *>(s->scal + S_GMAX);
        absmax_kernel<<<kVecBlocks, kVecThreads, 0, st>>>(7 * s->E * s->gpts, s->G, gmax);
        cast_f16_kernel<<<kVecBlocks, kVecThreads, 0, st>>>(7 * s->E * s->gpts, s->G, s->G16, gmax, s->scal + S_GINV);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t pcg_create(fem_pcg *s) {
    cudaError_t e = pcg_create_on(s, (cudaStream_t)0, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)0);
    return e;
}

// Frees the workspace, stream-ordered on st (the workspace must not be in
// use by work on other streams).
void pcg_release_on(fem_pcg *s, cudaStream_t st) {
    void *bufs[] = {s->r,   s->z,   s->p,   s->q,    s->dinv, s->G32,  s->dinv32, s->d32,
                    s->r32, s->z32, s->p32, s->q32, s->G16,  s->part, s->scal};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, st);
    if (s->ev) cudaEventDestroy(s->ev);
    if (s->hscal && s->own_hscal) cudaFreeHost(s->hscal);
    cudaGraphExec_t gs[] = {s->g_iter64, s->g_iter32, s->g_outer};
    for (cudaGraphExec_t g : gs)
        if (g) cudaGraphExecDestroy(g);
    s->g_iter64 = s->g_iter32 = s->g_outer = nullptr;
    s->ev = nullptr;
    s->hscal = nullptr;
}

void pcg_release(fem_pcg *s) {
    if (s->pending && s->ev) cudaEventSynchronize(s->ev);
    pcg_release_on(s, s->ws);
    cudaStreamSynchronize(s->ws);
}

// Starts a solve of A x = b on stream st: enqueues b . b and returns.
cudaError_t pcg_begin(fem_pcg *s, const double *b, double *x, const fem_pcg_opts *o, cudaStream_t st) {
    s->tol = (o && o->tol > 0) ? o->tol : 1e-10;
    s->maxit = (o && o->maxit > 0) ? o->maxit : 100000;
    s->itol = (o && o->inner_tol > 0) ? o->inner_tol : 1e-4;
    s->imaxit = (o && o->inner_maxit > 0) ? o->inner_maxit : 100000;
    s->every = (o && o->check_every > 0) ? o->check_every : (s->mode == FEM_PCG_FP64 ? 8 : 16);
    // the captured graphs name the vectors and the tolerances they were
    // captured with
    if (s->g_b != b || s->g_x != x || s->g_tol != s->tol || s->g_itol != s->itol) {
        cudaGraphExec_t gs[] = {s->g_iter64, s->g_iter32, s->g_outer};
        for (cudaGraphExec_t g : gs)
            if (g) cudaGraphExecDestroy(g);
        s->g_iter64 = s->g_iter32 = s->g_outer = nullptr;
        s->g_b = b;
        s->g_x = x;
        s->g_tol = s->tol;
        s->g_itol = s->itol;
    }
    s->b = b;
    s->x = x;
    s->st = st;
    s->use_graphs = !(st == (cudaStream_t)0 || st == cudaStreamLegacy || st == cudaStreamPerThread);
    s->chunk_done = 0;
    s->inner_iters = 0;
    s->outer = 0;
    s->restarts = 0;
    s->restart_rr = 0.0;
    s->status = FEM_OK;
    std::memset(&s->info, 0, sizeof s->info);
    cudaError_t e = cudaMemsetAsync(s->scal + S_WAITFAIL, 0, sizeof(double), st);
    if (e == cudaSuccess) e = launch_dot(s->len, b, b, s->scal + S_BB, s->part, st);
    if (e == cudaSuccess) e = end_step(s);
    s->state = PS_BB;
    return e;
}

// Advances a solve by at most one step.  Returns 1 when the solve has
// finished (s->status, s->info hold the outcome), 0 when work is in flight,
// or -1 on a CUDA error.  blocking: wait for the step in flight instead of
// polling it.
int pcg_advance(fem_pcg *s, bool blocking) {
    if (s->state == PS_DONE) return 1;
    if (s->pending) {
        if (blocking) {
            if (cudaEventSynchronize(s->ev) != cudaSuccess) return -1;
        } else {
            const cudaError_t q = cudaEventQuery(s->ev);
            if (q == cudaErrorNotReady) return 0;
            if (q != cudaSuccess) return -1;
        }
        s->pending = false;
    }
    const double *h = s->hscal;
    cudaError_t e = cudaSuccess;
    if (h[S_WAITFAIL] != 0.0) {
        // a kernel of the last step gave up a bounded device wait: its
        // output, and so x, are not to be trusted
        s->status = FEM_ETIMEDOUT;
        s->info.iters = s->inner_iters + (s->mode == FEM_PCG_FP64 ? (int)h[S_ITER] : 0);
        s->info.outer = s->outer;
        s->state = PS_DONE;
        return 1;
    }
    switch (s->state) {
        case PS_BB:
            s->bb = h[S_BB];
            if (!std::isfinite(s->bb)) {  // a NaN or an infinity in the right-hand side
                s->status = FEM_EBREAKDOWN;
                s->state = PS_DONE;
                return 1;
            }
            if (s->bb == 0.0) {  // the solution of A x = 0 is 0
                e = cudaMemsetAsync(s->x, 0, sizeof(double) * s->len, s->st);
                s->state = PS_DONE;
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
                return e == cudaSuccess ? 1 : -1;
            }
            if (s->mode == FEM_PCG_FP64) {
                e = op_apply64(s, s->x, s->q, s->st);
                if (e == cudaSuccess) {
                    init_kernel<<<kVecBlocks, kVecThreads, 0, s->st>>>(s->len, s->b, s->q, s->r, s->z, s->dinv, s->part);
                    reduce_kernel<<<1, kRedThreads, 0, s->st>>>(R_INIT, kVecBlocks, s->part, s->scal, nullptr,
                                                                s->tol * s->tol);
                    e = cudaGetLastError();
                }
                const int c = next_chunk(s, 0, s->maxit);
                if (e == cudaSuccess) e = inject_armed_fault(s);
                if (e == cudaSuccess) e = enqueue_chunk<double, double>(s, s->G, s->x, s->p, s->r, s->q, s->z, s->dinv, c);
                s->chunk_done = c;
                s->state = PS_RUN64;
            } else {
                e = enqueue_outer(s);
                s->state = PS_OUTER;
            }
            break;
        case PS_RUN64: {
            const bool fin = h[S_DONE] != 0.0 || h[S_BREAK] != 0.0 || s->chunk_done >= s->maxit;
            if (!fin) {
                const int c = next_chunk(s, s->chunk_done, s->maxit);
                e = enqueue_chunk<double, double>(s, s->G, s->x, s->p, s->r, s->q, s->z, s->dinv, c);
                s->chunk_done += c;
                break;
            }
            s->info.iters += (int)h[S_ITER];
            s->info.outer = 1;
            if (h[S_BREAK] != 0.0 && h[S_DONE] == 0.0)
                s->status = FEM_EBREAKDOWN;
            else if (h[S_DONE] == 0.0)
                s->status = FEM_ENOCONV;
            // true FP64 residual of the returned x; the reduction also sets
            // up a fresh start of the recurrence from it (r = b - A x, z, p
            // = z), used when the recurrence's residual has drifted below
            // the true one
            e = op_apply64(s, s->x, s->q, s->st);
            if (e == cudaSuccess) {
                init_kernel<<<kVecBlocks, kVecThreads, 0, s->st>>>(s->len, s->b, s->q, s->r, s->z, s->dinv, s->part);
                reduce_kernel<<<1, kRedThreads, 0, s->st>>>(R_INIT, kVecBlocks, s->part, s->scal, nullptr,
                                                            s->tol * s->tol);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = end_step(s);
            s->state = PS_FINAL64;
            break;
        }
        case PS_FINAL64: {
            s->info.relres = std::sqrt(h[S_RR] / s->bb);
            const bool met = h[S_RR] <= s->tol * s->tol * s->bb;
            if (s->status == FEM_OK && !met) {
                // residual replacement: the recurrence met the tolerance but
                // the true residual did not.  Restart from the true residual
                // while each restart at least halves it (at most 8 times);
                // otherwise the tolerance is below what FP64 attains here.
                const bool progress = s->restarts == 0 || h[S_RR] <= 0.25 * s->restart_rr;
                if (s->restarts < 8 && progress && s->chunk_done < s->maxit) {
                    s->restarts++;
                    s->restart_rr = h[S_RR];
                    const int c = next_chunk(s, s->chunk_done, s->maxit);
                    e = enqueue_chunk<double, double>(s, s->G, s->x, s->p, s->r, s->q, s->z, s->dinv, c);
                    s->chunk_done += c;
                    s->state = PS_RUN64;
                    break;
                }
                s->status = FEM_ENOCONV;
            }
            s->state = PS_DONE;
            return 1;
        }
        case PS_OUTER: {
            s->info.relres = std::sqrt(h[S_RR_OUTER] / s->bb);
            s->info.outer = s->outer;
            s->info.iters = s->inner_iters;
            if (h[S_RR_OUTER] <= s->tol * s->tol * s->bb) {
                s->state = PS_DONE;
                return 1;
            }
            if (s->outer >= 64 || s->inner_iters >= s->maxit) {
                s->status = FEM_ENOCONV;
                s->state = PS_DONE;
                return 1;
            }
            s->chunk_done = 0;
            const int c = next_chunk(s, 0, s->imaxit);
            e = inject_armed_fault(s);
            if (e == cudaSuccess)
                e = enqueue_chunk<float, float>(s, s->G32, s->d32, s->p32, s->r32, s->q32, s->z32, s->dinv32, c);
            s->chunk_done = c;
            s->state = PS_INNER;
            break;
        }
        case PS_INNER: {
            const bool fin = h[S_DONE] != 0.0 || h[S_BREAK] != 0.0 || s->chunk_done >= s->imaxit;
            if (!fin) {
                const int c = next_chunk(s, s->chunk_done, s->imaxit);
                e = enqueue_chunk<float, float>(s, s->G32, s->d32, s->p32, s->r32, s->q32, s->z32, s->dinv32, c);
                s->chunk_done += c;
                break;
            }
            const int it = (int)h[S_ITER];
            s->inner_iters += it;
            if (it == 0 && h[S_BREAK] != 0.0) {
                s->status = FEM_EBREAKDOWN;
                s->info.iters = s->inner_iters;
                s->state = PS_DONE;
                return 1;
            }
            add_f32_kernel<<<kVecBlocks, kVecThreads, 0, s->st>>>(s->len, s->x, s->d32);
            e = cudaGetLastError();
            s->outer++;
            if (e == cudaSuccess) e = enqueue_outer(s);
            s->state = PS_OUTER;
            break;
        }
        default:
            return 1;
    }
    return e == cudaSuccess ? 0 : -1;
}

int pcg_solve(fem_pcg *s, const double *b, double *x, const fem_pcg_opts *o, fem_pcg_info *info, cudaStream_t st) {
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = pcg_begin(s, b, x, o, st);
    if (e != cudaSuccess) return -2;
    int r;
    while ((r = pcg_advance(s, true)) == 0) {
    }
    if (r < 0) return -2;
    if (info) *info = s->info;
    return s->status;
}

}  // namespace fem

// ---------------------------------------------------------------------- C ABI

extern "C" {

int64_t fem_dot_scratch_size(void) { return fem::dot_scratch_size(); }

int fem_dot(int64_t n, const double *x, const double *y, double *result, double *scratch, void *stream) {
    if (n < 0 || !result || !scratch) return FEM_EINVAL;
    if (n > 0 && (!x || !y)) return FEM_EINVAL;
    cudaError_t e = fem::launch_dot(n, x, y, result, scratch, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : fem::record_cuda_error(e);
}

int fem_bp35_jacobi(const fem_basis *b, int64_t E, const double *G, double lambda, double *dinv, void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G || !dinv) return FEM_EINVAL;
    cudaError_t e = fem::dispatch_degree<fem::DinvLaunch>(b->host.N, b, E, G, lambda, dinv, (float *)nullptr,
                                                          (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : fem::record_cuda_error(e);
}

int fem_bp30_jacobi(const fem_basis *b, int64_t E, const double *G, double lambda, double *dinv, void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G || !dinv) return FEM_EINVAL;
    cudaError_t e = fem::dispatch_degree<fem::Dinv30Launch>(b->host.N, b, E, G, lambda, dinv, (float *)nullptr,
                                                            (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : fem::record_cuda_error(e);
}

}  // extern "C"

namespace fem {

int pcg_new(const fem_basis *b, int op, int64_t E, const double *G, double lambda, int mode, fem_pcg **out) {
    if (!b || !out || E < 1 || !G ||
        (mode != FEM_PCG_FP64 && mode != FEM_PCG_MIXED && mode != FEM_PCG_MIXED16 && mode != FEM_PCG_MIXED_TC))
        return FEM_EINVAL;
    if (op != FEM_OP_BP35 && op != FEM_OP_BP30) return FEM_EINVAL;
    if (mode == FEM_PCG_MIXED_TC && E > (int64_t)0x7fffffff) return FEM_EINVAL;  // one block per element
    if (!(lambda >= 0.0)) return FEM_EINVAL;
    *out = nullptr;
    fem_pcg *s = new (std::nothrow) fem_pcg();
    if (!s) return FEM_ENOMEM;
    std::memset((void *)s, 0, sizeof(*s));
    s->basis = b;
    s->op = op;
    s->gpts = (op == FEM_OP_BP30) ? (int64_t)b->host.m * b->host.m * b->host.m
                                  : (int64_t)b->host.n * b->host.n * b->host.n;
    s->E = E;
    s->len = E * (int64_t)b->host.n * b->host.n * b->host.n;
    s->G = G;
    s->lambda = lambda;
    s->mode = mode;
    s->state = PS_IDLE;
    *out = s;
    return FEM_OK;
}

void pcg_delete(fem_pcg *s) { delete s; }

int pcg_status(const fem_pcg *s, fem_pcg_info *info) {
    if (info) *info = s->info;
    return s->status;
}

void pcg_arm_wait_fault(fem_pcg *s) { s->wait_fault_armed = true; }

int pcg_quiescent(fem_pcg *s) {
    if (!s->pending) return 1;
    const cudaError_t q = cudaEventQuery(s->ev);
    if (q == cudaErrorNotReady) return 0;
    s->pending = false;
    return q == cudaSuccess ? 1 : -1;
}

static_assert(kPcgScalars == S_COUNT, "pinned scalar block size");

}  // namespace fem

extern "C" {

int fem_pcg_create(const fem_basis *b, int op, int64_t E, const double *G, double lambda, int mode, fem_pcg **out) {
    fem_pcg *s = nullptr;
    const int r = fem::pcg_new(b, op, E, G, lambda, mode, &s);
    if (r != FEM_OK) return r;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = fem::pcg_create(s);
    if (e != cudaSuccess) {
        fem::pcg_release(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? FEM_ENOMEM : fem::record_cuda_error(e);
    }
    *out = s;
    return FEM_OK;
}

void fem_pcg_destroy(fem_pcg *s) {
    if (!s) return;
    fem::pcg_release(s);
    delete s;
}

int fem_pcg_inject_fault(fem_pcg *s, int fault) {
    if (!s || fault != FEM_FAULT_WAIT_TIMEOUT) return FEM_EINVAL;
    fem::pcg_arm_wait_fault(s);
    return FEM_OK;
}

int fem_pcg_solve(fem_pcg *s, const double *rhs, double *x, const fem_pcg_opts *opts, fem_pcg_info *info,
                  void *stream) {
    if (!s || !rhs || !x || rhs == x) return FEM_EINVAL;
    const int r = fem::pcg_solve(s, rhs, x, opts, info, (cudaStream_t)stream);
    if (r == -2) return fem::record_cuda_error(cudaGetLastError());
    return r;
}

}  // extern "C"
