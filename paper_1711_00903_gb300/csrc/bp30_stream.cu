// Instantiations and launchers of the FP32 / FP16-factor BP3.0 stream
// kernels of bp30_stream.cuh (a translation unit of their own, compiled in
// parallel with the block kernels).
#include "bp30_stream.cuh"

namespace fem {
namespace {

// The stream kernel's choice as the default BP3.0 operator of a degree, from
// the sweep on the 32^3 mesh (GB300, fraction of the copy rate against the
// block kernel).  FP32 factors: 0.63 / 0.57 at N = 3, 0.72 / 0.67 at 6,
// 0.66 / 0.64 at 7, 0.38 / 0.37 at 14 and 0.39 / 0.35 at 15; at the other
// degrees the block kernel was as fast or faster (0.62 / 0.34 at N = 1).
// With the packed FMA and the searched box strides the plain operator
// (not the PCG variant, which reads the old p in its staging loop) also
// gains at N = 8, 10 and 11 (GDOF/s: 94 / 90, 77 / 76, 89 / 87; 59 / 87 at
// N = 12 and 69 / 78 at 13 stay with the block kernel).  FP16 factors
// (GDOF/s): 92 / 85 at N = 7, 88 / 81 at 8, 95 / 81 at 9, 87 / 74 at 10,
// 76 / 70 at 12, 75 / 68 at 13; ties or losses elsewhere (50 / 64 at N = 4).
template <int N, typename TG, bool PCG>
constexpr bool stream30_default() {
    if constexpr (!Bp30Stream<N, true, TG>::fits) {
        return false;
    } else if constexpr (sizeof(TG) == 4) {
        return N == 3 || N == 6 || N == 7 || N == 14 || N == 15 || (!PCG && (N == 8 || N == 10 || N == 11));
    } else {
        return (N >= 7 && N <= 10) || N == 12 || N == 13;
    }
}

template <typename TG>
struct Stream30 {
    template <int N>
    struct Launch {
        static cudaError_t run(bool pcg, int64_t E, const TG *G, const double *ginv, double lambda, const float *q,
                               float *Aq, const float *z, float *p, const double *beta, double *partials,
                               cudaStream_t s, double *status) {
            if constexpr (Bp30Stream<N, true, TG>::fits) {
                if (pcg)
                    return launch_stream30<N, true, TG, 1>(E, G, lambda, q, Aq, z, p, beta, partials, s, ginv,
                                                           status);
                return launch_stream30<N, false, TG, 1>(E, G, lambda, q, Aq, z, p, beta, partials, s, ginv, status);
            } else {
                return cudaErrorInvalidValue;
            }
        }
    };
    template <int N>
    struct Info {
        static cudaError_t run(int64_t E, bool pcg, int64_t *grid, bool *def) {
            *def = pcg ? stream30_default<N, TG, true>() : stream30_default<N, TG, false>();
            *grid = stream_grid30(E, Bp30Stream<N, true, TG>::blocks_per_sm);
            return cudaSuccess;
        }
    };
    template <int N>
    struct Prepare {
        static cudaError_t run() { return prepare_stream30<N, TG, 1>(); }
    };
};

FEM_DEFINE_FOLD_UPLOAD(upload_fold_bp30_stream_tu)

}  // namespace

FEM_DEFINE_WAIT_COUNTER(wait_timeouts_bp30_stream)

cudaError_t launch_bp30_stream(int N, bool pcg, int64_t E, const float *G, double lambda, const float *q, float *Aq,
                               const float *z, float *p, const double *beta, double *partials, cudaStream_t s,
                               double *status) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<Stream30<float>::Launch>(N, pcg, E, G, (const double *)nullptr, lambda, q, Aq, z, p, beta,
                                                    partials, s, status);
}

cudaError_t launch_bp30_stream_f16g(int N, bool pcg, int64_t E, const __half *G, const double *ginv, double lambda,
                                    const float *q, float *Aq, const float *z, float *p, const double *beta,
                                    double *partials, cudaStream_t s, double *status) {
    if (E <= 0) return cudaSuccess;
    return dispatch_degree<Stream30<__half>::Launch>(N, pcg, E, G, ginv, lambda, q, Aq, z, p, beta, partials, s,
                                                     status);
}

bool bp30_stream_default(int N, bool f16, bool pcg) {
    int64_t g = 0;
    bool d = false;
    if (f16)
        dispatch_degree<Stream30<__half>::Info>(N, (int64_t)1, pcg, &g, &d);
    else
        dispatch_degree<Stream30<float>::Info>(N, (int64_t)1, pcg, &g, &d);
    return d;
}

int64_t bp30_stream_grid(int N, int64_t E, bool f16) {
    int64_t g = 0;
    bool d = false;
    if (f16)
        dispatch_degree<Stream30<__half>::Info>(N, E, true, &g, &d);
    else
        dispatch_degree<Stream30<float>::Info>(N, E, true, &g, &d);
    return g;
}

cudaError_t prepare_bp30_stream(int N, const double *fold_table) {
    cudaError_t e = upload_fold_bp30_stream_tu(fold_table);
    if (e == cudaSuccess) e = dispatch_degree<Stream30<float>::Prepare>(N);
    if (e == cudaSuccess) e = dispatch_degree<Stream30<__half>::Prepare>(N);
    return e;
}

}  // namespace fem
