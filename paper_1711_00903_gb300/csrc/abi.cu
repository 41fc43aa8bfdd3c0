// C ABI entry points (include/fem.h): argument checks, basis handles and
// dispatch to the kernels.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "fem_internal.h"

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
    std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return (e == cudaErrorNoDevice || e == cudaErrorNoKernelImageForDevice || e == cudaErrorInsufficientDriver)
               ? FEM_ENODEV
               : FEM_ECUDA;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// True when [a, a+na) and [b, b+nb) (in doubles) overlap.
bool overlap(const double *a, int64_t na, const double *b, int64_t nb) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), a1 = a0 + (uintptr_t)na * 8;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(b), b1 = b0 + (uintptr_t)nb * 8;
    return a0 < b1 && b0 < a1;
}

int64_t cube(int x) { return (int64_t)x * x * x; }

// Common checks of an apply call; returns FEM_OK or FEM_EINVAL.
int check_apply(const fem_basis *b, int64_t E, const double *geo, int64_t geo_per_elem,
                const double *q, const double *out) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!geo || !q || !out) return FEM_EINVAL;
    if (!aligned16(geo) || !aligned16(q) || !aligned16(out)) return FEM_EINVAL;
    const int64_t np = cube(b->host.n);
    if (E > (INT64_MAX / 8) / (geo_per_elem > np ? geo_per_elem : np)) return FEM_EINVAL;
    if (overlap(out, E * np, q, E * np) || overlap(out, E * np, geo, E * geo_per_elem)) return FEM_EINVAL;
    if ((E + 1) > (int64_t)0x7fffffff) return FEM_EINVAL;  // grid size limit
    return FEM_OK;
}

}  // namespace

namespace fem {
int record_cuda_error(cudaError_t e) { return cuda_fail(e); }
}  // namespace fem

extern "C" {

int fem_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char *fem_strerror(int code) {
    switch (code) {
        case FEM_OK: return "FEM_OK";
        case FEM_EINVAL: return "FEM_EINVAL: invalid argument";
        case FEM_ECUDA: return "FEM_ECUDA: CUDA runtime or launch error";
        case FEM_ENOMEM: return "FEM_ENOMEM: allocation failed";
        case FEM_ENODEV: return "FEM_ENODEV: no usable CUDA device";
        case FEM_EBREAKDOWN: return "FEM_EBREAKDOWN: conjugate-gradient breakdown";
        case FEM_ENOCONV: return "FEM_ENOCONV: iteration limit reached";
        case FEM_ETOOBIG: return "FEM_ETOOBIG: size beyond the fixed capacity of the call";
        case FEM_ECANCELED: return "FEM_ECANCELED: the request was cancelled";
        case FEM_ETIMEDOUT: return "FEM_ETIMEDOUT: a bounded device wait gave up; the result is not to be trusted";
        default: return "unknown fem error code";
    }
}

const char *fem_last_cuda_error(void) { return g_cuda_err; }

int fem_basis_setup(int N, fem_basis **out) {
    if (!out || N < 1 || N > FEM_MAX_N) return FEM_EINVAL;
    *out = nullptr;
    fem_basis *b = new (std::nothrow) fem_basis();
    if (!b) return FEM_ENOMEM;
    if (!fem::compute_basis(N, &b->host)) {
        delete b;
        return FEM_EINVAL;
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e);
    }
    const fem::HostBasis &h = b->host;
    const fem::OpsLayout L{h.n, h.m};
    double table[fem::OpsLayout{fem::kMaxQ - 1, fem::kMaxQ}.size() + 64];
    std::memset(table, 0, sizeof table);
    std::memcpy(table + L.offI(), h.I, sizeof(double) * h.m * h.n);
    std::memcpy(table + L.offD(), h.D, sizeof(double) * h.n * h.n);
    std::memcpy(table + L.offDt(), h.Dt, sizeof(double) * h.m * h.m);
    std::memcpy(table + L.offR(), h.r, sizeof(double) * h.n);
    std::memcpy(table + L.offRt(), h.rt, sizeof(double) * h.m);
    std::memcpy(table + L.offW(), h.w, sizeof(double) * h.n);
    std::memcpy(table + L.offWt(), h.wt, sizeof(double) * h.m);
    for (int a2 = 0; a2 < h.m; a2++)  // C = Dt I
        for (int i = 0; i < h.n; i++) {
            double s = 0.0;
            for (int c = 0; c < h.m; c++) s += h.Dt[a2 * h.m + c] * h.I[c * h.n + i];
            table[L.offC() + a2 * h.n + i] = s;
        }
    e = cudaMalloc(&b->d_ops, sizeof(double) * L.size());
    if (e != cudaSuccess) {
        delete b;
        return e == cudaErrorMemoryAllocation ? FEM_ENOMEM : cuda_fail(e);
    }
    e = cudaMemcpy(b->d_ops, table, sizeof(double) * L.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {  // B fragments of the tensor-core operators
        const int64_t words = fem::tc_table_words(N);
        uint32_t *tc = new (std::nothrow) uint32_t[words];
        if (!tc) {
            cudaFree(b->d_ops);
            delete b;
            return FEM_ENOMEM;
        }
        fem::build_tc_table(h, tc);
        e = cudaMalloc(&b->d_tc, sizeof(uint32_t) * words);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_tc, tc, sizeof(uint32_t) * words, cudaMemcpyHostToDevice);
        delete[] tc;
    }
    if (e == cudaSuccess) e = fem::prepare_bp1(N, fem::fold_table());
    if (e == cudaSuccess) e = fem::prepare_bp35(N, fem::fold_table());
    if (e == cudaSuccess) e = fem::prepare_bp30(N, fem::fold_table());
    if (e == cudaSuccess) e = fem::prepare_geofacs(N);
    if (e == cudaSuccess) e = fem::prepare_bp30_point(N);
    if (e == cudaSuccess) e = fem::prepare_bp35_f16(N, fem::fold_table());
    if (e == cudaSuccess) e = fem::prepare_bp30_f16(N, fem::fold_table());
    if (e == cudaSuccess) e = fem::prepare_bp30_tc(N);
    if (e == cudaSuccess) e = fem::prepare_bp35_tc(N);
    if (e == cudaSuccess) e = fem::prepare_bp30_warp(N, fem::fold_table());
    if (e != cudaSuccess) {
        cudaFree(b->d_ops);
        if (b->d_tc) cudaFree(b->d_tc);
        delete b;
        return cuda_fail(e);
    }
    *out = b;
    return FEM_OK;
}

void fem_basis_free(fem_basis *b) {
    if (!b) return;
    if (b->d_ops) cudaFree(b->d_ops);
    if (b->d_tc) cudaFree(b->d_tc);
    delete b;
}

int fem_basis_degree(const fem_basis *b) { return b ? b->host.N : FEM_EINVAL; }

static void copy_tables(const fem::HostBasis &h, double *r, double *w, double *rt, double *wt,
                        double *I, double *D, double *Dt) {
    if (r) std::memcpy(r, h.r, sizeof(double) * h.n);
    if (w) std::memcpy(w, h.w, sizeof(double) * h.n);
    if (rt) std::memcpy(rt, h.rt, sizeof(double) * h.m);
    if (wt) std::memcpy(wt, h.wt, sizeof(double) * h.m);
    if (I) std::memcpy(I, h.I, sizeof(double) * h.m * h.n);
    if (D) std::memcpy(D, h.D, sizeof(double) * h.n * h.n);
    if (Dt) std::memcpy(Dt, h.Dt, sizeof(double) * h.m * h.m);
}

int fem_basis_tables(const fem_basis *b, double *r, double *w, double *rt, double *wt, double *I,
                     double *D, double *Dt) {
    if (!b) return FEM_EINVAL;
    copy_tables(b->host, r, w, rt, wt, I, D, Dt);
    return FEM_OK;
}

int fem_basis_host_tables(int N, double *r, double *w, double *rt, double *wt, double *I, double *D,
                          double *Dt) {
    fem::HostBasis h;
    if (!fem::compute_basis(N, &h)) return FEM_EINVAL;
    copy_tables(h, r, w, rt, wt, I, D, Dt);
    return FEM_OK;
}

int fem_mesh_geofacs(const fem_basis *b, fem_geo_kind kind, int64_t E, const double *verts, double *geo,
                     double *detJ_min, void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (kind != FEM_GEO_BP1 && kind != FEM_GEO_BP35 && kind != FEM_GEO_BP30) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!verts || !geo || !aligned16(verts) || !aligned16(geo)) return FEM_EINVAL;
    if (detJ_min && !aligned16(detJ_min)) return FEM_EINVAL;
    if (E + 1 > (int64_t)0x7fffffff) return FEM_EINVAL;
    const int q = (kind == FEM_GEO_BP35) ? b->host.n : b->host.m;
    const int64_t per = (kind == FEM_GEO_BP1 ? 1 : 7) * cube(q);
    if (overlap(geo, E * per, verts, E * 24)) return FEM_EINVAL;
    if (detJ_min && (overlap(detJ_min, E, verts, E * 24) || overlap(detJ_min, E, geo, E * per)))
        return FEM_EINVAL;
    cudaError_t e = fem::launch_geofacs(b, kind, E, verts, geo, detJ_min, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_mesh_geofacs_set(const fem_basis *b, int64_t E, const double *verts, double *wJ, double *G35, double *G30,
                         void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (!wJ && !G35 && !G30) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!verts || !aligned16(verts) || E + 1 > (int64_t)0x7fffffff) return FEM_EINVAL;
    const int64_t nw = E * cube(b->host.m), n35 = E * 7 * cube(b->host.n), n30 = E * 7 * cube(b->host.m);
    const double *outs[3] = {wJ, G35, G30};
    const int64_t sizes[3] = {nw, n35, n30};
    for (int i = 0; i < 3; i++) {
        if (!outs[i]) continue;
        if (!aligned16(outs[i]) || overlap(outs[i], sizes[i], verts, E * 24)) return FEM_EINVAL;
        for (int j = 0; j < i; j++)
            if (outs[j] && overlap(outs[i], sizes[i], outs[j], sizes[j])) return FEM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (G35) e = fem::launch_geofacs(b, FEM_GEO_BP35, E, verts, G35, nullptr, s);
    if (e == cudaSuccess) {
        if (G30 && wJ)
            e = fem::launch_geofacs_gauss_pair(b, E, verts, G30, wJ, s);
        else if (G30)
            e = fem::launch_geofacs(b, FEM_GEO_BP30, E, verts, G30, nullptr, s);
        else if (wJ)
            e = fem::launch_geofacs(b, FEM_GEO_BP1, E, verts, wJ, nullptr, s);
    }
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp1_apply(const fem_basis *b, int64_t E, const double *wJ, const double *q, double *Mq,
                  void *stream) {
    const int c = check_apply(b, E, wJ, b ? cube(b->host.m) : 0, q, Mq);
    if (c != FEM_OK || E == 0) return c;
    cudaError_t e = fem::launch_bp1(b, E, wJ, q, Mq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp35_apply(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                   double *Aq, void *stream) {
    const int c = check_apply(b, E, G, b ? 7 * cube(b->host.n) : 0, q, Aq);
    if (c != FEM_OK || E == 0) return c;
    cudaError_t e = fem::launch_bp35(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp35_apply_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                       void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G || !q || !Aq || !aligned16(G) || !aligned16(q) || !aligned16(Aq)) return FEM_EINVAL;
    if ((const void *)Aq == (const void *)q || (E + 1) > (int64_t)0x7fffffff) return FEM_EINVAL;
    cudaError_t e = fem::launch_bp35_f32(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_wait_timeouts(unsigned long long *count, int reset) {
    if (!count) return FEM_EINVAL;
    unsigned long long a = 0, b = 0, c = 0;
    cudaError_t e = fem::wait_timeouts_bp35(&a, reset != 0);
    if (e == cudaSuccess) e = fem::wait_timeouts_bp35_f16(&b, reset != 0);
    if (e == cudaSuccess) e = fem::wait_timeouts_bp30_stream(&c, reset != 0);
    *count = a + b + c;
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_layout_check(int64_t *violations) {
    if (!violations) return FEM_EINVAL;
    *violations = (int64_t)fem::layout_violations_bp30() + (int64_t)fem::layout_violations_bp35();
    return FEM_OK;
}

int fem_wait_selftest(unsigned long long *gave_up) {
    if (!gave_up) return FEM_EINVAL;
    bool reported = false;
    cudaError_t e = fem::run_wait_selftest(gave_up, &reported);
    if (e != cudaSuccess) return cuda_fail(e);
    return reported ? FEM_ETIMEDOUT : FEM_OK;
}

int64_t fem_fma_probe_threads(void) { return fem::fma_probe_threads(); }

int fem_fma_probe(int64_t iters, double *out, void *stream) {
    if (iters < 1 || !out || !aligned16(out)) return FEM_EINVAL;
    cudaError_t e = fem::launch_fma_probe(iters, out, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_stream_sum(int planes, int64_t n, const void *src, void *dst, int word, void *stream) {
    if (planes < 1 || planes > fem::stream_max_planes() || n < 0 || (word != 4 && word != 8)) return FEM_EINVAL;
    if (n == 0) return FEM_OK;
    if (!src || !dst || !aligned16(src) || !aligned16(dst) || (n * word) % 16 != 0) return FEM_EINVAL;
    const char *s0 = (const char *)src, *d0 = (const char *)dst;
    const int64_t sb = (int64_t)planes * n * word, db = n * word;
    if (d0 < s0 + sb && s0 < d0 + db) return FEM_EINVAL;  // overlapping buffers
    cudaError_t e = fem::launch_stream_sum(planes, n, src, dst, word, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp35_apply_f16g(const fem_basis *b, int64_t E, const void *G16, const double *ginv, double lambda,
                        const float *q, float *Aq, void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G16 || !ginv || !q || !Aq || !aligned16(G16) || !aligned16(q) || !aligned16(Aq)) return FEM_EINVAL;
    if ((const void *)Aq == (const void *)q || (E + 1) > (int64_t)0x7fffffff) return FEM_EINVAL;
    cudaError_t e = fem::launch_bp35_f16g(b, E, (const __half *)G16, ginv, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp30_apply_f16g(const fem_basis *b, int64_t E, const void *G16, const double *ginv, double lambda,
                        const float *q, float *Aq, void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G16 || !ginv || !q || !Aq || !aligned16(G16) || !aligned16(q) || !aligned16(Aq)) return FEM_EINVAL;
    if ((const void *)Aq == (const void *)q || (E + 1) > (int64_t)0x7fffffff) return FEM_EINVAL;
    cudaError_t e = fem::launch_bp30_f16g(b, E, (const __half *)G16, ginv, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp30_apply_layout(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                          double *Aq, int layout, void *stream) {
    if (layout != FEM_LAYOUT_LINES && layout != FEM_LAYOUT_POINTS) return FEM_EINVAL;
    if (layout == FEM_LAYOUT_LINES) return fem_bp30_apply(b, E, G, lambda, q, Aq, stream);
    const int c = check_apply(b, E, G, b ? 7 * cube(b->host.m) : 0, q, Aq);
    if (c != FEM_OK || E == 0) return c;
    cudaError_t e = fem::launch_bp30_point(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp35_apply_layout(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                          double *Aq, int layout, void *stream) {
    if (layout != FEM_LAYOUT_LINES && layout != FEM_LAYOUT_POINTS) return FEM_EINVAL;
    if (layout == FEM_LAYOUT_LINES) return fem_bp35_apply(b, E, G, lambda, q, Aq, stream);
    const int c = check_apply(b, E, G, b ? 7 * cube(b->host.n) : 0, q, Aq);
    if (c != FEM_OK || E == 0) return c;
    cudaError_t e = fem::launch_bp35_point(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp30_apply_f32(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                       void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G || !q || !Aq || !aligned16(G) || !aligned16(q) || !aligned16(Aq)) return FEM_EINVAL;
    if ((const void *)Aq == (const void *)q || (E + 1) > (int64_t)0x7fffffff) return FEM_EINVAL;
    cudaError_t e = fem::launch_bp30_f32(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp30_apply_f32_layout(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q,
                              float *Aq, int layout, void *stream) {
    if (layout != FEM_LAYOUT_LINES && layout != FEM_LAYOUT_WARP && layout != FEM_LAYOUT_STREAM) return FEM_EINVAL;
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G || !q || !Aq || !aligned16(G) || !aligned16(q) || !aligned16(Aq)) return FEM_EINVAL;
    if ((const void *)Aq == (const void *)q || E > (int64_t)0x7fffffff) return FEM_EINVAL;
    cudaError_t e = layout == FEM_LAYOUT_WARP
                        ? fem::launch_bp30_warp(b, E, G, lambda, q, Aq, (cudaStream_t)stream)
                        : fem::launch_bp30_f32(b, E, G, lambda, q, Aq, (cudaStream_t)stream,
                                               layout == FEM_LAYOUT_STREAM ? 2 : 1);
    if (e == cudaErrorInvalidValue && layout == FEM_LAYOUT_STREAM) return FEM_EINVAL;  // does not fit at this degree
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp35_apply_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                      void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G || !q || !Aq || !aligned16(G) || !aligned16(q) || !aligned16(Aq)) return FEM_EINVAL;
    if ((const void *)Aq == (const void *)q || E > (int64_t)0x7fffffff) return FEM_EINVAL;
    cudaError_t e = fem::launch_bp35_tc(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp30_apply_tc(const fem_basis *b, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                      void *stream) {
    if (!b || E < 0) return FEM_EINVAL;
    if (E == 0) return FEM_OK;
    if (!G || !q || !Aq || !aligned16(G) || !aligned16(q) || !aligned16(Aq)) return FEM_EINVAL;
    if ((const void *)Aq == (const void *)q || E > (int64_t)0x7fffffff) return FEM_EINVAL;
    cudaError_t e = fem::launch_bp30_tc(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp30_apply(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                   double *Aq, void *stream) {
    const int c = check_apply(b, E, G, b ? 7 * cube(b->host.m) : 0, q, Aq);
    if (c != FEM_OK || E == 0) return c;
    cudaError_t e = fem::launch_bp30(b, E, G, lambda, q, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp1_bp30_apply(const fem_basis *b, int64_t E, const double *G, double lambda, const double *q,
                       double *Mq, double *Aq, void *stream) {
    int c = check_apply(b, E, G, b ? 7 * cube(b->host.m) : 0, q, Aq);
    if (c == FEM_OK) c = check_apply(b, E, G, b ? 7 * cube(b->host.m) : 0, q, Mq);
    if (c != FEM_OK || E == 0) return c;
    const int64_t np = cube(b->host.n);
    if (overlap(Mq, E * np, Aq, E * np)) return FEM_EINVAL;
    cudaError_t e = fem::launch_bp1_bp30(b, E, G, lambda, q, Mq, Aq, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : cuda_fail(e);
}

int fem_bp35_apply_ex(const fem_basis *b, int64_t E, int prec, const void *G, const double *ginv, double lambda,
                      const void *q, void *Aq, void *stream) {
    switch (prec) {
        case FEM_PREC_F64:
            return fem_bp35_apply(b, E, (const double *)G, lambda, (const double *)q, (double *)Aq, stream);
        case FEM_PREC_F32:
            return fem_bp35_apply_f32(b, E, (const float *)G, lambda, (const float *)q, (float *)Aq, stream);
        case FEM_PREC_F16G:
            return fem_bp35_apply_f16g(b, E, G, ginv, lambda, (const float *)q, (float *)Aq, stream);
        case FEM_PREC_F16TC:
            return fem_bp35_apply_tc(b, E, (const float *)G, lambda, (const float *)q, (float *)Aq, stream);
        default:
            return FEM_EINVAL;
    }
}

int fem_bp30_apply_ex(const fem_basis *b, int64_t E, int prec, const void *G, const double *ginv, double lambda,
                      const void *q, void *Aq, void *stream) {
    switch (prec) {
        case FEM_PREC_F64:
            return fem_bp30_apply(b, E, (const double *)G, lambda, (const double *)q, (double *)Aq, stream);
        case FEM_PREC_F32:
            return fem_bp30_apply_f32(b, E, (const float *)G, lambda, (const float *)q, (float *)Aq, stream);
        case FEM_PREC_F16G:
            return fem_bp30_apply_f16g(b, E, G, ginv, lambda, (const float *)q, (float *)Aq, stream);
        case FEM_PREC_F16TC:
            return fem_bp30_apply_tc(b, E, (const float *)G, lambda, (const float *)q, (float *)Aq, stream);
        default:
            return FEM_EINVAL;
    }
}

}  // extern "C"
