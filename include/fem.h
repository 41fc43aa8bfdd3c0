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

/* The factors of all three operators of one mesh in one call: wJ for
 * BP1.0 (E*NpG), G for BP3.5 (E*7*Np) and G for BP3.0 (E*7*NpG), each
 * exactly as fem_mesh_geofacs writes it (same values bit for bit).  Any
 * of the three outputs may be NULL (at least one must not be); outputs
 * must not overlap each other or verts.  When both wJ and the BP3.0
 * factors are asked for, one kernel writes both: BP1.0's wJ is the
 * seventh BP3.0 factor at the same Gauss points (Section 4).  Asynchronous
 * on stream, allocates nothing.  E == 0 enqueues nothing.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_mesh_geofacs_set(const fem_basis *b, int64_t E, const double *verts, double *wJ,
                         double *G35, double *G30, void *stream);

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

/* BP3.5 matvec in FP32 (the inner operator of the mixed-precision solver;
 * same layouts as fem_bp35_apply with float data; FP32 arithmetic).
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp35_apply_f32(const fem_basis *b, int64_t E, const float *G, double lambda,
                       const float *q, float *Aq, void *stream);

/* FP64 issue-rate probe (the FP64 ceiling of the operators is measured, not
 * assumed): fem_fma_probe_threads() threads (8 blocks of 256 per SM of the
 * current device) each run eight independent FP64 FMA chains of iters steps
 * and store one double to out (device, fem_fma_probe_threads() doubles).
 * One launch performs 2 * 8 * iters * threads flops; time it on stream.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int64_t fem_fma_probe_threads(void);
int fem_fma_probe(int64_t iters, double *out, void *stream);

/* Number of bounded device-side waits that gave up on the current device
 * since the library was loaded or last reset (reset != 0 clears it).  The
 * kernels that stage data with TMA bulk copies wait on mbarriers with an
 * iteration limit (about a second) instead of spinning forever; a wait
 * that gives up is counted here and the kernel's output is not to be
 * trusted.  0 in normal operation.  Synchronous.
 * Errors: FEM_EINVAL (count NULL), FEM_ECUDA. */
int fem_wait_timeouts(unsigned long long *count, int reset);

/* Self-test of the bounded device waits: runs one block whose mbarrier
 * wait can never complete (a barrier expecting an arrival that never comes)
 * and reports in *gave_up how many warps gave up after the wait's limit
 * (about a second): 2 when the limit works.  The block also reports the
 * failure through a device status word, as the stream kernels report it to
 * the solver; the call returns FEM_ETIMEDOUT when that report arrived (the
 * expected outcome) and FEM_OK when it did not.  The context stays usable;
 * this self-test's count is not added to fem_wait_timeouts.  Synchronous.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_wait_selftest(unsigned long long *gave_up);

/* Host-side check of the element boxes the operator kernels lay out in
 * shared memory, for every degree: each point of each box (BP3.0's four
 * boxes, BP3.5's n^3 box, in the FP64 and FP32 layouts) must map to a
 * distinct word inside its share of the per-element buffer, and the
 * swizzled FP32 BP3.5 boxes (N = 7 and 15) must serve the lines of every
 * direction, taken by the 32 lanes of a warp, without a shared-memory bank
 * conflict.  Writes the number of violations to *violations (0 when every
 * layout holds).  Runs on the host only: no GPU needed.
 * Errors: FEM_EINVAL (violations NULL). */
int fem_layout_check(int64_t *violations);

/* Roofline calibration stream with a chosen read:write ratio (Section 5
 * calibrates the bandwidth roofline by a copy; the operators read several
 * planes per plane written): dst[i] = sum over p = 0..planes-1, in that
 * order, of src[p*n + i].  src device planes*n values, dst device n values,
 * of word bytes each (8: double, 4: float); both 16-byte aligned, n*word a
 * multiple of 16, 1 <= planes <= 32, no overlap.  Asynchronous on stream,
 * allocates nothing.  Moves (planes + 1) * n * word bytes.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_stream_sum(int planes, int64_t n, const void *src, void *dst, int word, void *stream);

/* BP3.5 and BP3.0 matvecs with half-precision factors: the inner operators
 * of FEM_PCG_MIXED16.  G16: device, the factor layout of fem_bp35_apply /
 * fem_bp30_apply with IEEE binary16 values (uint16_t bits), 16-byte
 * aligned; ginv: device, one double, multiplied into the output (the
 * inverse of the power of two the factors were scaled by; 1.0 for none);
 * q, Aq: device floats.  FP32 arithmetic.  Asynchronous on stream,
 * allocates nothing.  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp35_apply_f16g(const fem_basis *b, int64_t E, const void *G16, const double *ginv, double lambda,
                        const float *q, float *Aq, void *stream);
int fem_bp30_apply_f16g(const fem_basis *b, int64_t E, const void *G16, const double *ginv, double lambda,
                        const float *q, float *Aq, void *stream);

/* Thread layouts of the operator kernels (Section 6 compares both):
 * FEM_LAYOUT_LINES   two-dimensional: one thread per line of an element,
 *                    even-odd folded 1D operators (the default everywhere);
 * FEM_LAYOUT_POINTS  three-dimensional: one thread per quadrature point,
 *                    one element per block, operators in shared memory. */
#define FEM_LAYOUT_LINES 0
#define FEM_LAYOUT_POINTS 1
/* FEM_LAYOUT_WARP    two-dimensional lines as FEM_LAYOUT_LINES, one warp
 *                    (two or four above N = 9) per element and no block
 *                    barrier between the phases (FP32 BP3.0 only). */
#define FEM_LAYOUT_WARP 2
/* FEM_LAYOUT_STREAM  FP32 BP3.0 only: a persistent grid that stages each
 *                    element's field and factors in shared memory with TMA
 *                    bulk copies, the next element's factors in flight
 *                    while the current one finishes (lines as
 *                    FEM_LAYOUT_LINES; degrees whose element fits in
 *                    shared memory). */
#define FEM_LAYOUT_STREAM 3

/* fem_bp30_apply with a chosen thread layout (same arguments, layouts and
 * errors; FEM_EINVAL for an unknown layout).  Both layouts compute the same
 * operator and agree to rounding. */
int fem_bp30_apply_layout(const fem_basis *b, int64_t E, const double *G, double lambda,
                          const double *q, double *Aq, int layout, void *stream);

/* fem_bp35_apply with a chosen thread layout: FEM_LAYOUT_LINES (the
 * default kernels) or FEM_LAYOUT_POINTS (Algorithm 7: one thread per GLL
 * node, one element per block, D in shared memory).  Same arguments,
 * layouts and errors (FEM_EINVAL for another layout); both compute the
 * same operator and agree to rounding. */
int fem_bp35_apply_layout(const fem_basis *b, int64_t E, const double *G, double lambda,
                          const double *q, double *Aq, int layout, void *stream);

/* BP3.0 matvec in FP32 (Algorithm 5 with float data and FP32 arithmetic;
 * the inner operator of the mixed-precision BP3.0 solver).  Same layouts as
 * fem_bp30_apply: G device E*7*m^3 floats, q and Aq device E*n^3 floats,
 * 16-byte aligned, Aq != q.  Asynchronous on stream, allocates nothing.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp30_apply_f32(const fem_basis *b, int64_t E, const float *G, double lambda,
                       const float *q, float *Aq, void *stream);

/* fem_bp30_apply_f32 with a chosen kernel: FEM_LAYOUT_LINES (several
 * elements per block, block barriers between the phases, factors read from
 * global memory), FEM_LAYOUT_STREAM (factors staged by TMA, FEM_EINVAL at a
 * degree where an element does not fit in shared memory) or
 * FEM_LAYOUT_WARP (one warp per element); fem_bp30_apply_f32 takes the
 * fastest measured for the degree.  Same arguments, layouts and errors
 * (FEM_EINVAL for another layout; E <= 2^31 - 1).  All compute the same
 * FP32 operator and agree to FP32 rounding. */
int fem_bp30_apply_f32_layout(const fem_basis *b, int64_t E, const float *G, double lambda,
                              const float *q, float *Aq, int layout, void *stream);

/* BP3.0 matvec (Algorithm 5) with its twelve 1D contractions on the tensor
 * cores: mma.sync m16n8k16 with f16 operands and FP32 accumulation, FP32
 * factors and vectors; the inner operator of FEM_PCG_MIXED_TC.  Every
 * contraction line is scaled by a power of two into the f16 range and
 * split into a high and a low f16 part, and the operator entries likewise,
 * so that three products on one K axis give about 2^-22 relative accuracy
 * (one f16 product gives 2^-11, too coarse for the solver's correction
 * equation).  Layouts as fem_bp30_apply_f32: G device E*7*m^3 floats, q
 * and Aq device E*n^3 floats, 16-byte aligned, Aq != q; E <= 2^31 - 1 (one
 * block per element).  Asynchronous on stream, allocates nothing.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp30_apply_tc(const fem_basis *b, int64_t E, const float *G, double lambda,
                      const float *q, float *Aq, void *stream);

/* BP3.5 matvec (Algorithm 4) with its six 1D derivative contractions (D and
 * D^T at the GLL nodes) on the tensor cores, by the same split-f16 scheme
 * as fem_bp30_apply_tc; the chain rule with the factors and the lambda term
 * in FP32.  The inner operator of FEM_PCG_MIXED_TC for BP3.5.  Layouts as
 * fem_bp35_apply_f32 (G E*7*n^3 floats, q, Aq E*n^3 floats, 16-byte
 * aligned, Aq != q); E <= 2^31 - 1.  Asynchronous on stream, allocates
 * nothing.  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp35_apply_tc(const fem_basis *b, int64_t E, const float *G, double lambda,
                      const float *q, float *Aq, void *stream);

/* BP1.0 and BP3.0 of one field in one pass (Algorithms 3 and 5): the
 * interpolation of q to the Gauss points is computed once for both, and
 * BP1.0's wJ is the seventh plane of G (the same w |J| at the same points,
 * which fem_mesh_geofacs_set writes identically to its wJ output).
 * G: device E*7*m^3 doubles (fem_bp30_apply's layout); q, Mq, Aq: device
 * E*n^3 doubles, 16-byte aligned, Mq, Aq, q pairwise disjoint.  Mq and Aq
 * are bit for bit what fem_bp1_apply (with that wJ) and fem_bp30_apply
 * return.  Asynchronous on stream, allocates nothing.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp1_bp30_apply(const fem_basis *b, int64_t E, const double *G, double lambda,
                       const double *q, double *Mq, double *Aq, void *stream);

/* Precision selectors of the *_apply_ex entry points. */
#define FEM_PREC_F64 0  /* FP64 factors, vectors and arithmetic (fem_bp35_apply, fem_bp30_apply) */
#define FEM_PREC_F32 1  /* FP32 factors, vectors and arithmetic (fem_bp*_apply_f32) */
#define FEM_PREC_F16G 2 /* binary16 factors scaled by a power of two, FP32 vectors and
                         * arithmetic (fem_bp*_apply_f16g) */
#define FEM_PREC_F16TC 3 /* FP32 factors and vectors, contractions on the tensor cores
                          * (fem_bp35_apply_tc, fem_bp30_apply_tc) */

/* BP3.5 and BP3.0 matvecs with the precision chosen at run time: each call
 * is the precision's own entry point above, with G, q and Aq of that
 * precision's types (double; float; uint16_t binary16 bits for G and float
 * for q, Aq).  ginv: device, one double, read by FEM_PREC_F16G only (may be
 * NULL otherwise).  BP1.0 has only its FP64 form.  Layouts, alignment,
 * asynchrony and ownership as for the entry point selected.
 * Errors: FEM_EINVAL (also for an unknown prec), FEM_ECUDA. */
int fem_bp35_apply_ex(const fem_basis *b, int64_t E, int prec, const void *G, const double *ginv,
                      double lambda, const void *q, void *Aq, void *stream);
int fem_bp30_apply_ex(const fem_basis *b, int64_t E, int prec, const void *G, const double *ginv,
                      double lambda, const void *q, void *Aq, void *stream);

/* Inverse of the diagonal of the BP3.5 operator D^T G D + lambda J (the
 * Jacobi preconditioner), in closed form:
 *   diag_ijk = sum_l (D_li^2 Grr_ljk + D_lj^2 Gss_ilk + D_lk^2 Gtt_ijl)
 *            + 2 (D_ii D_jj Grs + D_ii D_kk Grt + D_jj D_kk Gst)_ijk + lambda wJ_ijk.
 *   G device E*7*Np, dinv device E*Np (1/diag).  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp35_jacobi(const fem_basis *b, int64_t E, const double *G, double lambda,
                    double *dinv, void *stream);

/* Inverse of the diagonal of the BP3.0 operator I^T (Dt^T G Dt + lambda J) I:
 * with B = I and C = Dt I the gradient of basis function (i,j,k) at Gauss
 * point (a,b,c) is (C_ai B_bj B_ck, B_ai C_bj B_ck, B_ai B_bj C_ck), and the
 * diagonal sums g^T G g + lambda wJ (B_ai B_bj B_ck)^2 over the points
 * (seven sum-factorised projections).  G device E*7*NpG, dinv device E*Np.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_bp30_jacobi(const fem_basis *b, int64_t E, const double *G, double lambda,
                    double *dinv, void *stream);

/* Deterministic FP64 dot product of two device vectors of n doubles: the
 * result is written to *result (device); scratch is a caller-owned device
 * array of at least fem_dot_scratch_size() doubles (its contents are
 * overwritten).  Two calls with the same inputs give the same bits.
 * Asynchronous on stream.  Errors: FEM_EINVAL, FEM_ECUDA. */
int64_t fem_dot_scratch_size(void);
int fem_dot(int64_t n, const double *x, const double *y, double *result, double *scratch,
            void *stream);

/* The same dot product without any device allocation, for callers that
 * cannot call cudaMalloc where they need the reduction: a serving loop that
 * must not allocate per request (an allocation can synchronise the device
 * or fail under a fixed memory budget), or an application whose device
 * memory is owned by its own allocator, so that a library may not take
 * memory behind its back.  The paper has no counterpart; this is a
 * library convenience.  The caller passes x, y (device, n doubles) and
 * result (device, one double) only.  The partial sums live in a 32 KiB
 * device array inside the library (one partial per 8192 entries), which
 * every GPU that loads the library holds until the process exits, so n is
 * capped at fem_dot_noalloc_max_n() = 33,554,432; larger n returns
 * FEM_ETOOBIG without launching anything.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the rest of the process; make that first call
 * before any stream capture.  cudaDeviceReset of that device after the
 * first call is not supported (the kept address would be stale).  Every call
 * shares the array and overwrites the slots it uses (nothing needs
 * clearing), so calls that overlap on the GPU (different streams, or
 * several host threads) race and must be serialised by the caller.
 * Deterministic; agrees with fem_dot to rounding.  Asynchronous on stream.
 * Errors: FEM_EINVAL, FEM_ETOOBIG, FEM_ECUDA. */
#define FEM_ETOOBIG (-7) /* size beyond a fixed capacity of the library */
int64_t fem_dot_noalloc_max_n(void);
int fem_dot_noalloc(int64_t n, const double *x, const double *y, double *result, void *stream);

/* ---------------------------------------------------------------------
 * Jacobi-preconditioned conjugate gradients for the unassembled BP3.5 or
 * BP3.0 Helmholtz system A x = rhs (Section 4; the solver is the textbook
 * PCG with M = diag A).  Two modes:
 *   FEM_PCG_FP64   all-FP64 PCG;
 *   FEM_PCG_MIXED  FP64 defect correction: the residual rhs - A x, its norm
 *                  and the update of x in FP64; each correction A d = r
 *                  solved to inner_tol by an FP32 PCG (FP32 factors, FP32
 *                  matvec, FP64 dot products).
 *   FEM_PCG_MIXED16  as FEM_PCG_MIXED, with the inner matvec reading the
 *                  factors in IEEE binary16, scaled by a power of two (set
 *                  on the device from the largest factor) and widened to
 *                  FP32 in the kernel: half the factor bytes, same FP32
 *                  arithmetic.  The FP64 outer loop still reaches tol.
 *   FEM_PCG_MIXED_TC  as FEM_PCG_MIXED, with the inner matvec's
 *                  contractions on the tensor cores (fem_bp35_apply_tc,
 *                  fem_bp30_apply_tc: split f16 operands, FP32
 *                  accumulation); E <= 2^31 - 1.
 * A solver context owns its device workspace (about 5 vectors in FP64
 * mode; 7 FP32 (MIXED16: FP16) factor planes and 6 FP32 + 1 FP64 vectors in
 * the mixed modes).
 * --------------------------------------------------------------------- */
#define FEM_EBREAKDOWN (-5) /* p.Ap <= 0 or a non-finite value in the recurrence */
#define FEM_ENOCONV (-6)    /* iteration limit reached; x holds the last iterate */
#define FEM_ETIMEDOUT (-8)  /* a kernel's bounded device wait gave up during the solve
                             * (its staged data may not have landed): x is not to be
                             * trusted.  The solver stops at the end of the step in
                             * which the kernel reported it. */

#define FEM_OP_BP35 2 /* operator selectors of the solver and of batches */
#define FEM_OP_BP30 3

#define FEM_PCG_FP64 0
#define FEM_PCG_MIXED 1
#define FEM_PCG_MIXED16 2
#define FEM_PCG_MIXED_TC 3

typedef struct fem_pcg fem_pcg; /* opaque */

typedef struct {
    double tol;       /* stop when ||rhs - A x||_2 <= tol ||rhs||_2 (default 1e-10) */
    int maxit;        /* iteration limit (default 100000)                          */
    double inner_tol; /* mixed: relative tolerance of each FP32 solve (1e-4); an
                       * FP32 solve also stops once its residual is below
                       * tol/2 * ||rhs|| (the outer target is then in reach) */
    int inner_maxit;  /* mixed: iteration limit of each FP32 solve (100000)        */
    int check_every;  /* host convergence check period (8 FP64, 16 FP32)           */
} fem_pcg_opts;

typedef struct {
    int iters;     /* PCG iterations (FP32 inner iterations in mixed mode) */
    int outer;     /* defect-correction steps (1 in FP64 mode)             */
    double relres; /* ||rhs - A x||_2 / ||rhs||_2 of the returned x, FP64  */
} fem_pcg_info;

/* Creates a solver for E elements of the handle's degree: op FEM_OP_BP35
 * (factors G device E*7*Np) or FEM_OP_BP30 (E*7*NpG), FP64, which must stay
 * valid for the context's life, and lambda >= 0; computes the Jacobi
 * diagonal and, in mixed mode, the FP32 copy of G.  Allocates device memory;
 * synchronous.  Errors: FEM_EINVAL, FEM_ENOMEM, FEM_ECUDA. */
int fem_pcg_create(const fem_basis *b, int op, int64_t E, const double *G, double lambda, int mode,
                   fem_pcg **out);

/* Solves A x = rhs starting from the x passed in (device, E*Np doubles;
 * rhs device, not aliasing x).  opts may be NULL (defaults above); info
 * may be NULL.  Runs on stream and returns after the solve has finished
 * (host convergence checks every check_every iterations; all scalars of
 * the recurrence stay on the device).  The iterate is frozen on the device
 * at the first iteration that meets the tolerance, so the result does not
 * depend on check_every.  FEM_OK means that the true FP64 residual of the
 * returned x meets tol.  FP64 mode: when the recurrence's residual meets tol
 * but the true one does not (rounding drift near FP64's attainable
 * accuracy), the iteration restarts from the true residual, at most 8 times
 * and only while each restart halves it; then FEM_ENOCONV.  Returns FEM_OK,
 * FEM_ENOCONV, FEM_EBREAKDOWN, FEM_ETIMEDOUT (a kernel's bounded device
 * wait gave up), FEM_EINVAL or FEM_ECUDA. */
int fem_pcg_solve(fem_pcg *s, const double *rhs, double *x, const fem_pcg_opts *opts,
                  fem_pcg_info *info, void *stream);

/* Host-side fault injection for tests of the failure path: the solver's
 * next solve reports its first step (FEM_PCG_FP64: its first chunk of
 * iterations; the mixed modes: the first chunk of the first inner solve)
 * exactly as a kernel whose bounded device wait gave up would, so that the
 * solve returns FEM_ETIMEDOUT.  Nothing faults, hangs or waits on the GPU.
 * fault: FEM_FAULT_WAIT_TIMEOUT.  Applies to one solve; synchronous, no GPU
 * work.  Errors: FEM_EINVAL. */
#define FEM_FAULT_WAIT_TIMEOUT 1
int fem_pcg_inject_fault(fem_pcg *s, int fault);

/* Frees a solver (NULL accepted).  Synchronous. */
void fem_pcg_destroy(fem_pcg *s);

/* ---------------------------------------------------------------------
 * Batched matvecs: many independent meshes of mixed degree (1..10), each
 * with its own operator (BP3.5 or BP3.0, FP64), factors, lambda, input and
 * output, applied in ONE persistent launch (Section 4: every element is
 * independent, so meshes are just more elements).  Each element's result is
 * bit-identical to the per-mesh fem_bp35_apply_layout / fem_bp30_apply_layout
 * call with the layout the batch's configuration gives its operator and
 * degree.
 * --------------------------------------------------------------------- */

typedef struct {
    int op;                  /* FEM_OP_BP35 or FEM_OP_BP30                       */
    const fem_basis *basis;  /* degree 1..10 (the handle must outlive the batch) */
    int64_t E;               /* elements (0 allowed)                            */
    const double *geo;       /* device factors, as for the per-mesh call        */
    double lambda;
    const double *q;         /* device input, E*Np doubles                      */
    double *out;             /* device output, E*Np doubles, not aliasing q/geo */
} fem_batch_item;

typedef struct {
    int threads; /* threads per persistent block: 256 or 512              */
    int group;   /* tasks taken per fetch of the shared counter, 1..64    */
    int order;   /* 0: tasks by decreasing cost per element; 1: as given  */
    int layout;  /* thread layout of the tasks, a bit mask (0: lines, the
                  * default): FEM_BATCH_POINTS30 puts BP3.0 tasks up to N = 8,
                  * FEM_BATCH_POINTS35 BP3.5 tasks up to N = 9, in the point
                  * layout (one thread per quadrature point or node)        */
    float ms;    /* measured time of one launch (fem_batch_tune), or 0    */
} fem_batch_config;

#define FEM_BATCH_POINTS30 1 /* = FEM_LAYOUT_POINTS: BP3.0 tasks in the point layout */
#define FEM_BATCH_POINTS35 2 /* BP3.5 tasks in the point layout                    */

typedef struct fem_batch fem_batch; /* opaque */

/* Builds the task list of a batch (device copies of the descriptors; the
 * pointers in the items must stay valid while the batch is used).
 * Allocates device memory; synchronous.  Errors: FEM_EINVAL (bad op, degree
 * above 10, NULL or aliased pointers), FEM_ENOMEM, FEM_ECUDA. */
int fem_batch_create(const fem_batch_item *items, int count, fem_batch **out);

/* One persistent launch over every mesh of the batch with the current
 * configuration (a 4-byte counter reset, then the kernel), asynchronous on
 * stream.  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_batch_apply(fem_batch *b, void *stream);

/* Autotuner: times every configuration (threads 256/512 x group 1/2/4/8 x
 * both task orders x the layout masks that change something: BP3.0 points
 * when the batch has BP3.0 meshes of degree <= 8, BP3.5 points when it has
 * BP3.5 meshes of degree <= 9, and both; reps launches each after a
 * warm-up) on the batch itself,
 * keeps the fastest as the batch's configuration, and writes up to
 * max_results timings to results (may be NULL) and their count to
 * *nresults (may be NULL).  Synchronous.  Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_batch_tune(fem_batch *b, void *stream, int reps, fem_batch_config *results, int max_results,
                   int *nresults);

int fem_batch_get_config(const fem_batch *b, fem_batch_config *cfg);
int fem_batch_set_config(fem_batch *b, const fem_batch_config *cfg);

/* Captures the current configuration's launch (counter reset + kernel) into
 * a CUDA graph on an internal stream the first time (and again after the
 * configuration changes), then launches the graph on stream.
 * Errors: FEM_EINVAL, FEM_ECUDA. */
int fem_batch_graph_launch(fem_batch *b, void *stream);

/* Frees a batch (NULL accepted).  Synchronous. */
void fem_batch_destroy(fem_batch *b);

/* ---------------------------------------------------------------------
 * Continuous-batching server of Helmholtz solves on one GPU.  Each request
 * is a BP3.5 or BP3.0 system on its own mesh (vertices and right-hand side
 * in host memory), solved by the Jacobi-PCG above in FP64 or mixed
 * precision with all of its state on the device.  Requests wait in a queue
 * (FIFO, or least estimated work first) and are admitted while a slot is
 * free and their device footprint fits the HBM budget; admitted solves run
 * on separate streams and
 * overlap on the GPU.  A request's result is bit-identical alone and in
 * the mix (deterministic per-request reductions).
 * --------------------------------------------------------------------- */
typedef struct fem_server fem_server; /* opaque */

/* Admission order of queued requests. */
#define FEM_SERVE_FIFO 0     /* first come, first served (default)                    */
#define FEM_SERVE_SHORTEST 1 /* least estimated work first: E^(4/3) (N+1)^3 N ln(1/tol),
                              * times 2.5 for BP3.0 and 0.15 for the mixed modes (the
                              * per-iteration cost and the growth of Jacobi-PCG's
                              * iteration count with N and the mesh size); ties by
                              * arrival, with aging: a request that has waited
                              * max_wait_s goes first, so a large request is not
                              * starved by a stream of smaller ones.                   */

typedef struct {
    int64_t hbm_budget; /* device bytes admitted requests may hold (default 120 GiB) */
    int max_active;     /* requests in flight at once, 1..256 (default 8)          */
    int check_every;    /* PCG iterations between host checks (default 8)          */
    int policy;         /* FEM_SERVE_FIFO or FEM_SERVE_SHORTEST                     */
    double max_wait_s;  /* FEM_SERVE_SHORTEST aging: once the oldest queued request
                         * has waited this long it is admitted next, ahead of
                         * smaller ones (default 2 s; <= 0 takes the default)   */
} fem_serve_opts;

typedef struct {
    int op;              /* FEM_OP_BP35 or FEM_OP_BP30                              */
    int N;               /* degree 1..15                                            */
    int64_t E;           /* elements                                                */
    const double *verts; /* host, E*8*3; read when the request is admitted          */
    const double *rhs;   /* host, E*Np; read when the request is admitted           */
    double *x;           /* host output, E*Np; written when the request finishes    */
    double lambda;       /* >= 0                                                    */
    int mode;            /* FEM_PCG_FP64, _MIXED, _MIXED16 or _MIXED_TC             */
    double tol;          /* relative residual tolerance                             */
} fem_serve_request;

#define FEM_REQ_QUEUED 0
#define FEM_REQ_RUNNING 1
#define FEM_REQ_DONE 2
#define FEM_REQ_FAILED 3

typedef struct {
    int state;       /* FEM_REQ_*                                               */
    int status;      /* FEM_OK, or why it failed (FEM_ENOMEM: over the budget)   */
    int iters, outer;
    double relres;   /* FP64 ||rhs - A x|| / ||rhs|| of the returned x           */
    double t_submit, t_admit, t_done; /* seconds on the server clock           */
    int64_t bytes;   /* device footprint charged against the budget             */
} fem_serve_result;

/* Creates a server on the current device (prepares every degree, one
 * stream and a pinned scalar block per slot).  opts may be NULL.
 * Errors: FEM_EINVAL, FEM_ENOMEM, FEM_ECUDA. */
int fem_serve_create(const fem_serve_opts *opts, fem_server **out);

/* Queues a request and returns its id; never blocks and never touches the
 * GPU.  The host buffers must stay valid until the request is DONE or
 * FAILED.  Errors: FEM_EINVAL. */
int fem_serve_submit(fem_server *s, const fem_serve_request *req, int64_t *id);

/* Moves the server on without blocking: retires finished solves, moves every
 * solve in flight on by one step when its previous step has finished, and
 * admits queued requests (in the server's policy order) while a slot and the
 * budget allow; a request at the head of that order that does not fit the
 * remaining budget holds back the ones behind it.  Call it in a
 * loop.  *active / *queued (may be NULL) receive the counts afterwards.
 * Errors: FEM_EINVAL. */
int fem_serve_progress(fem_server *s, int *active, int *queued);

/* State and outcome of a request.  Errors: FEM_EINVAL (unknown id). */
int fem_serve_poll(fem_server *s, int64_t id, fem_serve_result *res);

/* Progresses the server (fem_serve_progress) until request id is DONE or
 * FAILED or timeout_s seconds of host time have passed, then writes its
 * result to *res.  Returns FEM_OK when it finished, FEM_ETIMEDOUT when the
 * deadline passed first (the request is untouched and goes on in later
 * calls).  Waits on the host only (it polls the solves' events).
 * Errors: FEM_EINVAL (unknown id, NULL res, negative timeout). */
int fem_serve_wait(fem_server *s, int64_t id, double timeout_s, fem_serve_result *res);

/* Cancels request id.  A queued request is removed at once (FAILED,
 * status FEM_ECANCELED).  A running one is given no further step: it
 * becomes FAILED with FEM_ECANCELED at the first fem_serve_progress after
 * the step in flight on its stream has finished (no kernel is interrupted),
 * and its device memory is released.  A request whose solution is already
 * on its way to the host, or that has finished, is left as it is.  Other
 * requests are not affected.  Errors: FEM_EINVAL (unknown id). */
#define FEM_ECANCELED (-9)
int fem_serve_cancel(fem_server *s, int64_t id);

/* Seconds since the server was created (the clock of fem_serve_result). */
double fem_serve_clock(const fem_server *s);

/* Device bytes currently charged against the budget. */
int64_t fem_serve_in_use(const fem_server *s);

/* Waits for the solves in flight, frees everything (NULL accepted). */
void fem_serve_destroy(fem_server *s);

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
