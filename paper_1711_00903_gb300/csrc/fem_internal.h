// Internal declarations of the GB300 library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/fem.h"

namespace fem {

constexpr int kMaxN = FEM_MAX_N;
constexpr int kMaxQ = kMaxN + 2;

// Layout of the device table of one degree (all FP64, row-major):
//   I  (m x n) at offI, D (n x n) at offD, Dt (m x m) at offDt,
//   then GLL nodes r, Gauss nodes rt, GLL weights w, Gauss weights wt,
//   kMaxQ slots each.
struct OpsLayout {
    int n, m;
    __host__ __device__ constexpr int offI() const { return 0; }
    __host__ __device__ constexpr int offD() const { return m * n; }
    __host__ __device__ constexpr int offDt() const { return m * n + n * n; }
    __host__ __device__ constexpr int total() const { return m * n + n * n + m * m; }
    __host__ __device__ constexpr int offR() const { return total(); }
    __host__ __device__ constexpr int offRt() const { return total() + kMaxQ; }
    __host__ __device__ constexpr int offW() const { return total() + 2 * kMaxQ; }
    __host__ __device__ constexpr int offWt() const { return total() + 3 * kMaxQ; }
    // C = Dt I (m x n): derivatives of the GLL basis at the Gauss points
    __host__ __device__ constexpr int offC() const { return total() + 4 * kMaxQ; }
    __host__ __device__ constexpr int size() const { return total() + 4 * kMaxQ + m * n; }
};

// Host basis: nodes, weights and operator matrices of degree N.
struct HostBasis {
    int N, n, m;
    double r[kMaxQ], w[kMaxQ], rt[kMaxQ], wt[kMaxQ];
    double I[kMaxQ * kMaxQ], D[kMaxQ * kMaxQ], Dt[kMaxQ * kMaxQ];
};

// Computes the host basis (Golub-Welsch-type eigenvalue route + barycentric
// Lagrange formulas).  Returns false on a bad degree.
bool compute_basis(int N, HostBasis *hb);

}  // namespace fem

struct fem_basis {
    fem::HostBasis host;
    double *d_ops;  // device copy of I, D, Dt (fem::OpsLayout)
    void *d_tc;     // device table of the tensor-core operators' B fragments (tc_layout.h)
    int device;
};

namespace fem {

// Launchers (one per operator), dispatching on the degree at run time.
cudaError_t launch_geofacs(const fem_basis *b, int kind, int64_t E, const double *verts,
                           double *geo, double *detJ_min, cudaStream_t s);
cudaError_t launch_bp1(const fem_basis *b, int64_t E, const double *wJ, const double *q,
                       double *Mq, cudaStream_t s);
cudaError_t launch_bp35(const fem_basis *b, int64_t E, const double *G, double lambda,
                        const double *q, double *Aq, cudaStream_t s);
cudaError_t launch_bp1_bp30(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                            double *Mq, double *Aq, cudaStream_t s);
cudaError_t launch_bp30(const fem_basis *b, int64_t E, const double *G, double lambda,
                        const double *q, double *Aq, cudaStream_t s);

// One-time per-degree kernel preparation: uploads the folded operator
// table of every degree (fold_table()) and sets dynamic shared-memory limits.
cudaError_t prepare_bp1(int N, const double *fold_table);
cudaError_t prepare_bp35(int N, const double *fold_table);
cudaError_t prepare_bp30(int N, const double *fold_table);
cudaError_t launch_geofacs_gauss_pair(const fem_basis *b, int64_t E, const double *verts, double *G30, double *wJ,
                                      cudaStream_t s);
cudaError_t prepare_geofacs(int N);

// Host copy of the folded operator table of all degrees 1..15 (built once).
const double *fold_table();

// Records the text of a CUDA error for fem_last_cuda_error() and maps it to
// FEM_ECUDA or FEM_ENODEV.
int record_cuda_error(cudaError_t e);

// BP3.0 launchers for the solver (FP32 plain and both PCG-fused variants).
cudaError_t launch_bp30_point(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                              double *Aq, cudaStream_t s);
cudaError_t prepare_bp30_point(int N);  // and the BP3.5 point kernels
cudaError_t launch_bp35_point(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                              double *Aq, cudaStream_t s);
// FP32 BP3.0 TMA stream kernel (bp30_stream.cu): launch (cudaErrorInvalidValue
// where an element does not fit in shared memory), whether it is the default
// FP32 BP3.0 operator of the degree, its persistent grid (the PCG partials).
cudaError_t launch_bp30_stream(int N, bool pcg, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                               const float *z, float *p, const double *beta, double *partials, cudaStream_t s,
                               double *status);
cudaError_t launch_bp30_stream_f16g(int N, bool pcg, int64_t E, const __half *G, const double *ginv, double lambda,
                                    const float *q, float *Aq, const float *z, float *p, const double *beta,
                                    double *partials, cudaStream_t s, double *status);
bool bp30_stream_default(int N, bool f16, bool pcg);  // pcg: the PCG variant's choice
int64_t bp30_stream_grid(int N, int64_t E, bool f16 = false);
cudaError_t prepare_bp30_stream(int N, const double *fold_table);
// which: 0 the default kernel for the degree, 1 the block kernel, 2 the TMA
// stream kernel (cudaErrorInvalidValue where it does not fit)
cudaError_t launch_bp30_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q,
                            float *Aq, cudaStream_t s, int which = 0);
cudaError_t launch_bp30_pcg(const fem_basis *b, int64_t E, const double *G, double lambda, const double *z,
                            double *p, const double *beta, double *Ap, double *partials, cudaStream_t s);
// half-precision factors (FEM_PCG_MIXED16): binary16 planes scaled by a
// power of two, the inverse scale at ginv (device)
cudaError_t launch_bp35_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                             const float *q, float *Aq, cudaStream_t s);
// status: device word set to 1.0 when a bounded wait of the stream kernel
// gave up (may be NULL)
cudaError_t launch_bp35_pcg_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                                 const float *z, float *p, const double *beta, float *Ap, double *partials,
                                 cudaStream_t s, double *status);
int64_t bp35_f16_blocks(int N, int64_t E);
cudaError_t prepare_bp35_f16(int N, const double *fold_table);
cudaError_t wait_timeouts_bp35_f16(unsigned long long *count, bool reset);
cudaError_t launch_bp30_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                             const float *q, float *Aq, cudaStream_t s);
cudaError_t launch_bp30_pcg_f16g(const fem_basis *b, int64_t E, const __half *G, const double *ginv, double lambda,
                                 const float *z, float *p, const double *beta, float *Ap, double *partials,
                                 cudaStream_t s, double *status);
cudaError_t prepare_bp30_f16(int N, const double *fold_table);
cudaError_t launch_bp30_pcg_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                float *p, const double *beta, float *Ap, double *partials, cudaStream_t s,
                                double *status);
int64_t bp30_f16_blocks(int N, int64_t E);
// tensor-core BP3.0 (FEM_PCG_MIXED_TC): FP32 data, f16 split contractions
int64_t tc_table_words(int N);
void build_tc_table(const HostBasis &h, uint32_t *words);
cudaError_t prepare_bp30_tc(int N);
cudaError_t launch_bp30_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                           cudaStream_t s);
cudaError_t launch_bp30_pcg_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                               float *p, const double *beta, float *Ap, double *partials, cudaStream_t s);
cudaError_t prepare_bp35_tc(int N);
cudaError_t launch_bp35_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                           cudaStream_t s);
cudaError_t launch_bp35_pcg_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                               float *p, const double *beta, float *Ap, double *partials, cudaStream_t s);
// FP32 BP3.0 with one warp per element (bp30_warp.cu)
cudaError_t prepare_bp30_warp(int N, const double *fold_table);
cudaError_t launch_bp30_warp(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                             cudaStream_t s);
cudaError_t launch_bp30_pcg_warp(const fem_basis *b, int64_t E, const float *G, double lambda, const float *z,
                                 float *p, const double *beta, float *Ap, double *partials, cudaStream_t s);
int64_t bp30_blocks(int N, int64_t E, bool f32);

// FP32 BP3.5 matvec (the inner operator of the mixed-precision solver).
cudaError_t wait_timeouts_bp35(unsigned long long *count, bool reset);
// Host checks of the element-box layouts in shared memory: the number of
// violations (points mapped outside their buffer or onto another point's
// word; bank conflicts of the swizzled boxes), 0 when the layouts hold.
int layout_violations_bp30();
int layout_violations_bp35();
// The same count for the BP3.0 stream kernels (FP32 and FP16 factors).
cudaError_t wait_timeouts_bp30_stream(unsigned long long *count, bool reset);
cudaError_t launch_stream_sum(int planes, int64_t n, const void *src, void *dst, int word, cudaStream_t s);
int stream_max_planes();
int64_t fma_probe_threads();
cudaError_t run_wait_selftest(unsigned long long *gave_up, bool *reported);
cudaError_t launch_fma_probe(int64_t iters, double *out, cudaStream_t s);
cudaError_t launch_bp35_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q,
                            float *Aq, cudaStream_t s);
cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *result, double *scratch,
                       cudaStream_t s);
int64_t dot_scratch_size();

// PCG solver internals (pcg.cu).  A solve is resumable: pcg_begin enqueues
// its first step on a stream, pcg_advance moves it on by one step when the
// previous one has finished (1 = finished, 0 = in flight, -1 = CUDA error).
int pcg_new(const fem_basis *b, int op, int64_t E, const double *G, double lambda, int mode, fem_pcg **out);
void pcg_delete(fem_pcg *s);
cudaError_t pcg_create(fem_pcg *s);
cudaError_t pcg_create_on(fem_pcg *s, cudaStream_t st, double *lent_hscal);
void pcg_release(fem_pcg *s);
void pcg_release_on(fem_pcg *s, cudaStream_t st);
cudaError_t pcg_begin(fem_pcg *s, const double *b, double *x, const fem_pcg_opts *o, cudaStream_t st);
int pcg_advance(fem_pcg *s, bool blocking);
int pcg_solve(fem_pcg *s, const double *b, double *x, const fem_pcg_opts *o, fem_pcg_info *info, cudaStream_t st);
int pcg_status(const fem_pcg *s, fem_pcg_info *info);
// Host-side fault injection: the solver's next solve reports its first
// inner step (FP64 mode: its first chunk) as if a device wait had given up.
void pcg_arm_wait_fault(fem_pcg *s);
// 1 when no step of the solve is in flight on its stream, 0 while one is,
// -1 on a CUDA error (non-blocking).
int pcg_quiescent(fem_pcg *s);
constexpr int kPcgScalars = 14;  // doubles of pinned host memory a solver context needs

}  // namespace fem
