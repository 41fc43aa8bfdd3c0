/*
 * fem.h -- C ABI of the GB300 (sm_103a) element-local tensor-product
 * operators of high-order hexahedral spectral elements:
 *
 *   BP1.0  mass matvec                          Mq = I^T J I q
 *   BP3.5  collocated screened-Poisson matvec   Aq = D^T G D q + lambda J q
 *   BP3.0  dealiased screened-Poisson matvec    Aq = I^T (Dt^T G Dt + lambda J) I q
 *
 * after Swirydowicz, Chalmers, Karakus and Warburton, "Acceleration of
 * tensor-product operations for high-order finite element methods"
 * (arXiv:1711.00903), Section 4 (Algorithms 1-5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Degree N in 1..15; n = N+1 Gauss-Lobatto-Legendre (GLL) nodes and
 * m = N+2 Gauss-Legendre points per direction; Np = n^3, NpG = m^3.
 *
 * Vectors are element-local (unassembled, Section 4: the global operator is
 * block diagonal): q[e*Np + i + n*j + n*n*k] is the value at GLL node
 * (r_i, s_j, t_k) of element e, i (the r direction) fastest.
 *
 * Geometric factors are stored per element as planes of points:
 *   BP1.0: wJ[e*NpG + p]                   (wJ = w_a w_b w_c |J| at Gauss point p)
 *   BP3.5: G[(e*7 + g)*Np  + p]            (at GLL node p)
 *   BP3.0: G[(e*7 + g)*NpG + p]            (at Gauss point p)
 * with g = 0..6 = Grr, Grs, Grt, Gss, Gst, Gtt, wJ, each multiplied by the
 * tensor quadrature weight w_a w_b w_c; G = |J| X^{-1} X^{-T} with
 * X = dx/d(r,s,t) (the matrix G^e of Section 4, eq. Gdef).
 *
 * Element vertices: verts[(e*8 + c)*3 + d], corner c = cr + 2*cs + 4*ct with
 * cr, cs, ct in {0,1} meaning r, s, t = -1 or +1; d = x, y, z.  Each element
 * is the trilinear image of the bi-unit cube (Section 4).
 *
 * Memory: every array argument named "device" is a pointer to device memory
 * owned by the caller, 16-byte aligned, not overlapping any output of the
 * same call.  The library owns only what fem_basis_setup allocates.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Apply and geometric-factor calls only enqueue work: they never
 * allocate, never synchronise, and return before the GPU has finished.
 *
 * Errors: every int-returning function returns FEM_OK (0) or a negative
 * code below; fem_strerror() names it.  Argument errors are detected on the
 * host before anything is enqueued.  FEM_ECUDA reports a launch failure
 * (the CUDA error string is available from fem_last_cuda_error()).
 */
#ifndef FEM_H
#define FEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FEM_OK 0
#define FEM_EINVAL (-1)  /* bad degree, size, null or misaligned pointer, aliasing */
#define FEM_ECUDA (-2)   /* CUDA runtime or launch error                         */
#define FEM_ENOMEM (-3)  /* allocation failed (setup calls only)                 */
#define FEM_ENODEV (-4)  /* no usable CUDA device / kernel image for it          */

#define FEM_MAX_N 15

typedef struct fem_basis fem_basis; /* opaque */

typedef enum {
    FEM_GEO_BP1 = 1,  /* wJ at the Gauss points                    */
    FEM_GEO_BP35 = 2, /* 7 factors at the GLL nodes                */
    FEM_GEO_BP30 = 3  /* 7 factors at the Gauss points             */
} fem_geo_kind;

/* Build the degree-N basis (Section 2, Table of notation; Section 4):
 * GLL nodes/weights r, w (n), Gauss nodes/weights rt, wt (m), the
 * interpolation matrix I (m x n, I[a][i] = l_i(rt_a), eq. interpolationOps),
 * the GLL differentiation matrix D (n x n, D[a][i] = l_i'(r_a),
 * eq. derivativeOps) and the Gauss differentiation matrix Dt (m x m,
 * Dt[a][b] = lt_b'(rt_a), Section 4 BP3.0).  Computed on the host in FP64
 * and copied to the current device; prepares the degree-N kernels.
 * *out receives a handle owned by the caller (free with fem_basis_free).
 * Synchronous.  Errors: FEM_EINVAL (N outside 1..15, out NULL),
 * FEM_ENOMEM, FEM_ECUDA, FEM_ENODEV. */
int fem_basis_setup(int N, fem_basis **out);

/* Release a handle (NULL is accepted).  Synchronous. */
void fem_basis_free(fem_basis *b);

/* Degree N of a handle, or FEM_EINVAL for NULL. */
int fem_basis_degree(const fem_basis *b);

/* Copy the host FP64 tables of a handle into caller-owned host arrays of
 * sizes n, n, m, m, m*n, n*n, m*m (row-major); any pointer may be NULL.
 * Errors: FEM_EINVAL for a NULL handle. */
int fem_basis_tables(const fem_basis *b, double *r, double *w, double *rt, double *wt,
                     double *I, double *D, double *Dt);

/* The same FP64 tables computed on the host alone, without a handle or a
 * GPU (same sizes as fem_basis_tables; any pointer may be NULL).
 * Errors: FEM_EINVAL for N outside 1..15. */
int fem_basis_host_tables(int N, double *r, double *w, double *rt, double *wt,
                          double *I, double *D, double *Dt);

/* Geometric factors of E trilinear elements (Section 4: G^e = |J| X^{-1}X^{-T}
 * and J^e, each times the tensor quadrature weight; Algorithms 3-5 take
 * them as data).  kind selects the points and planes as described above.
 *   verts    device, E*8*3 doubles
 *   geo      device, E*NpG (BP1), E*7*Np (BP3.5) or E*7*NpG (BP3.0) doubles
 *   detJ_min device, E doubles or NULL: per-element minimum of |J| over the
 *            points (a value <= 0 flags an inverted element)
 * E == 0 enqueues nothing.  Errors: FEM_EINVAL (NULL handle/pointers when
 * E > 0, E < 0, bad kind, misaligned pointer), FEM_ECUDA. */
int fem_mesh_geofacs(const fem_basis *b, fem_geo_kind kind, int64_t E,
                     const double *verts, double *geo, double *detJ_min, void *stream);

/* BP1.0 mass matvec (Algorithm 3: interpolate GLL -> Gauss with
 * I x I x I (Algorithm 1), scale by wJ, project with I^T x I^T x I^T
 * (Algorithm 2)), six tensor contractions per element, IEEE FP64.
 *   wJ device E*NpG, q device E*Np, Mq device E*Np (must not overlap q, wJ).
 * E == 0 enqueues nothing.  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp1_apply(const fem_basis *b, int64_t E, const double *wJ, const double *q,
                  double *Mq, void *stream);

/* BP3.5 collocated screened-Poisson matvec (Algorithm 4): derivatives
 * along r, s, t with D, the symmetric chain rule with the six G factors,
 * D^T along each direction, plus lambda * wJ * q at the GLL nodes; six
 * tensor contractions per element, IEEE FP64.
 *   G device E*7*Np, q device E*Np, Aq device E*Np (must not overlap q, G).
 * E == 0 enqueues nothing.  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp35_apply(const fem_basis *b, int64_t E, const double *G, double lambda,
                   const double *q, double *Aq, void *stream);

/* BP3.0 dealiased screened-Poisson matvec (Algorithm 5): interpolate to
 * the Gauss points, differentiate there with Dt, apply the chain rule with
 * G, apply Dt^T, add lambda * wJ times the interpolated field, project
 * with I^T; twelve tensor contractions per element, IEEE FP64.
 *   G device E*7*NpG, q device E*Np, Aq device E*Np (must not overlap q, G).
 * E == 0 enqueues nothing.  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp30_apply(const fem_basis *b, int64_t E, const double *G, double lambda,
                   const double *q, double *Aq, void *stream);

/* Static name of an error code. */
const char *fem_strerror(int code);

/* Text of the last CUDA error this thread saw inside the library ("" if none). */
const char *fem_last_cuda_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int fem_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FEM_H */
