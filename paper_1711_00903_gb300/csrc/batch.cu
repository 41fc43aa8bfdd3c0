// Batched application of BP3.5 and BP3.0 (FP64) to many independent meshes of
// mixed degree in one persistent launch.
//
// The batch is flattened into tasks of up to EPB(N) consecutive elements of
// one mesh (EPB chosen per degree for the launch's block size).  A grid of
// (resident blocks per SM x SMs) persistent blocks pulls groups of tasks
// from a global counter (one atomicAdd per group) and runs each task with
// the same device functions as the stand-alone kernels (bp35_body.cuh,
// bp30_body.cuh), so every element's result is bit-identical to the
// per-mesh calls.  Tasks are ordered by decreasing cost per element by
// default, so that the expensive high-degree work starts first and the tail
// is made of cheap tasks.
//
// The launch shape (threads per block, tasks per counter fetch, task order,
// and the thread layout per operator: lines, or one thread per point for
// BP3.0 tasks up to N = 8 (bp30_point.cuh) and BP3.5 tasks up to N = 9
// (bp35_point.cuh, Algorithm 7)) is chosen by a small autotuner that times
// every candidate on the batch itself; the chosen configuration can be
// replayed from a CUDA graph that contains the counter reset and the kernel.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "bp30_body.cuh"
#include "bp30_point.cuh"
#include "bp35_body.cuh"
#include "bp35_point.cuh"

namespace fem {
namespace {

constexpr int kBatchMaxN = 10;
constexpr int kBatchMaxPointN = 8;    // BP3.0 point layout: m^3 <= 1000 points, 4 m^3 doubles of shared memory
constexpr int kBatchMaxPointN35 = 9;  // BP3.5 point layout: n^3 <= 1000 nodes
constexpr int kBatchSmemBudget = 96 * 1024;

struct BatchMesh {
    const double *ops;  // basis table of the mesh's degree (point layout)
    const double *G;
    const double *q;
    double *out;
    double lambda;
    int64_t E;
    int op;
    int N;
};

struct BatchTask {
    int64_t e0;
    int mesh;
    int nel;
};

template <int THREADS, int N>
struct Epb35 {
    static constexpr int n = N + 1;
    static constexpr int per = 3 * Box<n, n, n>::size * 8;
    static constexpr int a = THREADS / (n * n), b = kBatchSmemBudget / per;
    static constexpr int v = (a < b ? a : b) > 0 ? (a < b ? a : b) : 1;
};
template <int THREADS, int N>
struct Epb30 {
    static constexpr int m = N + 2;
    static constexpr int per = 3 * Box<m, m, m>::size * 8;
    static constexpr int a = THREADS / (m * m), b = kBatchSmemBudget / per;
    static constexpr int v = (a < b ? a : b) > 0 ? (a < b ? a : b) : 1;
};

template <int THREADS, int N>
constexpr int batch_smem_n() {
    constexpr int s35 = Bp35Layout<double, N, Epb35<THREADS, N>::v>::smem;
    constexpr int s30 = Bp30Layout<N, Epb30<THREADS, N>::v>::smem;
    constexpr int sp = N <= kBatchMaxPointN ? Bp30Point<N>::smem : 0;
    constexpr int sp35 = N <= kBatchMaxPointN35 ? Bp35Point<N>::smem : 0;
    constexpr int s = s35 > s30 ? s35 : s30;
    constexpr int t = s > sp ? s : sp;
    return t > sp35 ? t : sp35;
}

template <int THREADS>
constexpr int batch_smem() {
    int s = 0;
    const int v[kBatchMaxN] = {batch_smem_n<THREADS, 1>(), batch_smem_n<THREADS, 2>(), batch_smem_n<THREADS, 3>(),
                               batch_smem_n<THREADS, 4>(), batch_smem_n<THREADS, 5>(), batch_smem_n<THREADS, 6>(),
                               batch_smem_n<THREADS, 7>(), batch_smem_n<THREADS, 8>(), batch_smem_n<THREADS, 9>(),
                               batch_smem_n<THREADS, 10>()};
    for (int i = 0; i < kBatchMaxN; i++) s = v[i] > s ? v[i] : s;
    return s;
}

template <int THREADS>
int epb_for(int op, int N) {
    switch (op * 16 + N) {
#define FEM_EPB(K)                                   \
    case FEM_OP_BP35 * 16 + K:                       \
        return Epb35<THREADS, K>::v;                 \
    case FEM_OP_BP30 * 16 + K:                       \
        return Epb30<THREADS, K>::v;
        FEM_EPB(1) FEM_EPB(2) FEM_EPB(3) FEM_EPB(4) FEM_EPB(5)
        FEM_EPB(6) FEM_EPB(7) FEM_EPB(8) FEM_EPB(9) FEM_EPB(10)
#undef FEM_EPB
        default:
            return 1;
    }
}

// One task, as a separate (not inlined) function per operator and degree so
// that each body gets its own register allocation.
template <int THREADS, int K>
__device__ __noinline__ void task35(unsigned char *smem, const BatchTask tk, const BatchMesh M) {
    bp35_block<double, K, Epb35<THREADS, K>::v, false>(smem, tk.e0, tk.nel, M.G, M.lambda, M.q, M.out, nullptr,
                                                       nullptr, nullptr, nullptr);
}
template <int THREADS, int K>
__device__ __noinline__ void task30(unsigned char *smem, const BatchTask tk, const BatchMesh M) {
    bp30_block<K, Epb30<THREADS, K>::v>(reinterpret_cast<double *>(smem), tk.e0, tk.nel, M.G, M.lambda, M.q, M.out);
}
// the same tasks in the point layouts: their elements one after the other
template <int THREADS, int K>
__device__ __noinline__ void task30_point(unsigned char *smem, const BatchTask tk, const BatchMesh M) {
    for (int el = 0; el < tk.nel; el++) {
        if (el > 0) __syncthreads();
        bp30_point_block<K, THREADS>(reinterpret_cast<double *>(smem), M.ops, tk.e0 + el, M.G, M.lambda, M.q, M.out);
    }
}
template <int THREADS, int K>
__device__ __noinline__ void task35_point(unsigned char *smem, const BatchTask tk, const BatchMesh M) {
    for (int el = 0; el < tk.nel; el++) {
        if (el > 0) __syncthreads();
        bp35_point_block<K, THREADS>(reinterpret_cast<double *>(smem), M.ops, tk.e0 + el, M.G, M.lambda, M.q, M.out);
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
batch_kernel(const BatchMesh *__restrict__ meshes, const BatchTask *__restrict__ tasks, int ntasks, int group,
             int layout, int *__restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_t;
    for (;;) {
        __syncthreads();  // the previous task is finished with shared memory and s_t
        if (threadIdx.x == 0) s_t = atomicAdd(counter, group);
        __syncthreads();
        const int t0 = s_t;
        if (t0 >= ntasks) return;
        const int t1 = (t0 + group < ntasks) ? t0 + group : ntasks;
        for (int t = t0; t < t1; t++) {
            if (t > t0) __syncthreads();
            const BatchTask tk = tasks[t];
            const BatchMesh M = meshes[tk.mesh];
            switch (M.op * 16 + M.N) {
#define FEM_TASK(K)                                           \
    case FEM_OP_BP35 * 16 + K:                                \
        if (K <= kBatchMaxPointN35 && (layout & FEM_BATCH_POINTS35)) \
            task35_point<THREADS, (K <= kBatchMaxPointN35 ? K : 1)>(smem, tk, M); \
        else                                                  \
            task35<THREADS, K>(smem, tk, M);                  \
        break;                                                \
    case FEM_OP_BP30 * 16 + K:                                \
        if (K <= kBatchMaxPointN && (layout & FEM_BATCH_POINTS30)) \
            task30_point<THREADS, (K <= kBatchMaxPointN ? K : 1)>(smem, tk, M); \
        else                                                  \
            task30<THREADS, K>(smem, tk, M);                  \
        break;
                FEM_TASK(1) FEM_TASK(2) FEM_TASK(3) FEM_TASK(4) FEM_TASK(5)
                FEM_TASK(6) FEM_TASK(7) FEM_TASK(8) FEM_TASK(9) FEM_TASK(10)
#undef FEM_TASK
                default:
                    break;
            }
        }
    }
}

FEM_DEFINE_FOLD_UPLOAD(upload_fold_batch_tu)

// FP64 instructions per element (even-odd lines; used to order tasks).
double cost_per_element(int op, int N) {
    const int n = N + 1, m = N + 2;
    return op == FEM_OP_BP30 ? (double)m * m * m * (2.0 * m + 30) + 4.0 * n * n * n * m
                             : (double)n * n * n * (3.0 * n + 15);
}

}  // namespace
}  // namespace fem

struct fem_batch {
    int nmeshes;
    std::vector<fem::BatchMesh> host_meshes;
    fem::BatchMesh *d_meshes;
    fem::BatchTask *d_tasks[2][2];  // [variant][order]
    int ntasks[2][2];
    int *d_counter;
    int blocks[2];  // persistent grid per variant
    fem_batch_config cfg;
    cudaStream_t capture_stream;
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    fem_batch_config graph_cfg;
    int device;
};

namespace fem {
namespace {

template <int THREADS>
cudaError_t prepare_variant(int *blocks) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         batch_smem<THREADS>());
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<THREADS>, THREADS, batch_smem<THREADS>());
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *blocks = (per_sm > 0 ? per_sm : 1) * sms;
    return cudaSuccess;
}

std::vector<BatchTask> build_tasks(const std::vector<BatchMesh> &ms, int variant, int order) {
    std::vector<int> idx(ms.size());
    for (size_t i = 0; i < ms.size(); i++) idx[i] = (int)i;
    if (order == 0)
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return cost_per_element(ms[a].op, ms[a].N) > cost_per_element(ms[b].op, ms[b].N);
        });
    std::vector<BatchTask> t;
    for (int i : idx) {
        const int epb = variant == 0 ? epb_for<256>(ms[i].op, ms[i].N) : epb_for<512>(ms[i].op, ms[i].N);
        for (int64_t e = 0; e < ms[i].E; e += epb) {
            BatchTask k;
            k.e0 = e;
            k.mesh = i;
            k.nel = (int)std::min<int64_t>(epb, ms[i].E - e);
            t.push_back(k);
        }
    }
    return t;
}

cudaError_t launch(fem_batch *b, const fem_batch_config &c, cudaStream_t s) {
    const int v = c.threads == 512 ? 1 : 0, o = c.order ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (b->ntasks[v][o] == 0) return cudaSuccess;
    if (v == 0)
        batch_kernel<256><<<b->blocks[0], 256, batch_smem<256>(), s>>>(b->d_meshes, b->d_tasks[0][o], b->ntasks[0][o],
                                                                       c.group, c.layout, b->d_counter);
    else
        batch_kernel<512><<<b->blocks[1], 512, batch_smem<512>(), s>>>(b->d_meshes, b->d_tasks[1][o], b->ntasks[1][o],
                                                                       c.group, c.layout, b->d_counter);
    return cudaGetLastError();
}

void release(fem_batch *b) {
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (int v = 0; v < 2; v++)
        for (int o = 0; o < 2; o++)
            if (b->d_tasks[v][o]) cudaFree(b->d_tasks[v][o]);
    if (b->d_meshes) cudaFree(b->d_meshes);
    if (b->d_counter) cudaFree(b->d_counter);
}

bool valid_config(const fem_batch_config *c) {
    return c && (c->threads == 256 || c->threads == 512) && c->group >= 1 && c->group <= 64 &&
           (c->order == 0 || c->order == 1) && c->layout >= 0 &&
           c->layout <= (FEM_BATCH_POINTS30 | FEM_BATCH_POINTS35);
}

}  // namespace
}  // namespace fem

extern "C" {

int fem_batch_create(const fem_batch_item *items, int count, fem_batch **out) {
    if (!out || count < 0 || (count > 0 && !items)) return FEM_EINVAL;
    *out = nullptr;
    std::vector<fem::BatchMesh> ms;
    for (int i = 0; i < count; i++) {
        const fem_batch_item &it = items[i];
        if (!it.basis || (it.op != FEM_OP_BP35 && it.op != FEM_OP_BP30) || it.E < 0) return FEM_EINVAL;
        const int N = it.basis->host.N;
        if (N > fem::kBatchMaxN || !(it.lambda == it.lambda)) return FEM_EINVAL;
        if (it.E > 0 && (!it.geo || !it.q || !it.out)) return FEM_EINVAL;
        if (it.E > 0 && (it.out == it.q || it.out == it.geo)) return FEM_EINVAL;
        fem::BatchMesh m;
        m.ops = it.basis->d_ops;
        m.G = it.geo;
        m.q = it.q;
        m.out = it.out;
        m.lambda = it.lambda;
        m.E = it.E;
        m.op = it.op;
        m.N = N;
        ms.push_back(m);
    }
    fem_batch *b = new (std::nothrow) fem_batch();
    if (!b) return FEM_ENOMEM;
    b->nmeshes = count;
    b->host_meshes = ms;
    b->cfg.threads = 256;
    b->cfg.group = 1;
    b->cfg.order = 0;
    b->cfg.layout = FEM_LAYOUT_LINES;
    b->cfg.ms = 0.0f;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = fem::upload_fold_batch_tu(fem::fold_table());
    if (e == cudaSuccess) e = fem::prepare_variant<256>(&b->blocks[0]);
    if (e == cudaSuccess) e = fem::prepare_variant<512>(&b->blocks[1]);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_meshes, sizeof(fem::BatchMesh) * (ms.size() + 1));
    if (e == cudaSuccess && !ms.empty())
        e = cudaMemcpy(b->d_meshes, ms.data(), sizeof(fem::BatchMesh) * ms.size(), cudaMemcpyHostToDevice);
    for (int v = 0; v < 2 && e == cudaSuccess; v++)
        for (int o = 0; o < 2 && e == cudaSuccess; o++) {
            std::vector<fem::BatchTask> t = fem::build_tasks(ms, v, o);
            b->ntasks[v][o] = (int)t.size();
            e = cudaMalloc((void **)&b->d_tasks[v][o], sizeof(fem::BatchTask) * (t.size() + 1));
            if (e == cudaSuccess && !t.empty())
                e = cudaMemcpy(b->d_tasks[v][o], t.data(), sizeof(fem::BatchTask) * t.size(), cudaMemcpyHostToDevice);
        }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        fem::release(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? FEM_ENOMEM : fem::record_cuda_error(e);
    }
    *out = b;
    return FEM_OK;
}

void fem_batch_destroy(fem_batch *b) {
    if (!b) return;
    fem::release(b);
    delete b;
}

int fem_batch_apply(fem_batch *b, void *stream) {
    if (!b) return FEM_EINVAL;
    cudaError_t e = fem::launch(b, b->cfg, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : fem::record_cuda_error(e);
}

int fem_batch_get_config(const fem_batch *b, fem_batch_config *cfg) {
    if (!b || !cfg) return FEM_EINVAL;
    *cfg = b->cfg;
    return FEM_OK;
}

int fem_batch_set_config(fem_batch *b, const fem_batch_config *cfg) {
    if (!b || !fem::valid_config(cfg)) return FEM_EINVAL;
    b->cfg = *cfg;
    return FEM_OK;
}

int fem_batch_tune(fem_batch *b, void *stream, int reps, fem_batch_config *results, int max_results,
                   int *nresults) {
    if (!b || reps < 1) return FEM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads[2] = {256, 512}, groups[4] = {1, 2, 4, 8};
    // a point layout is a candidate only when the batch has meshes it applies to
    bool p30 = false, p35 = false;
    for (const fem::BatchMesh &m : b->host_meshes) {
        p30 = p30 || (m.op == FEM_OP_BP30 && m.N <= fem::kBatchMaxPointN && m.E > 0);
        p35 = p35 || (m.op == FEM_OP_BP35 && m.N <= fem::kBatchMaxPointN35 && m.E > 0);
    }
    int layouts[4], nlayouts = 0;
    for (int l = 0; l <= (FEM_BATCH_POINTS30 | FEM_BATCH_POINTS35); l++)
        if ((!(l & FEM_BATCH_POINTS30) || p30) && (!(l & FEM_BATCH_POINTS35) || p35)) layouts[nlayouts++] = l;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return fem::record_cuda_error(e);
    fem_batch_config best = b->cfg;
    best.ms = 1e30f;
    int k = 0;
    for (int li = 0; li < nlayouts && e == cudaSuccess; li++)
    for (int ti = 0; ti < 2 && e == cudaSuccess; ti++)
        for (int gi = 0; gi < 4 && e == cudaSuccess; gi++)
            for (int order = 0; order < 2 && e == cudaSuccess; order++) {
                fem_batch_config c;
                c.threads = threads[ti];
                c.group = groups[gi];
                c.order = order;
                c.layout = layouts[li];
                e = fem::launch(b, c, s);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                for (int r = 0; r < reps && e == cudaSuccess; r++) e = fem::launch(b, c, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                c.ms = ms / reps;
                if (results && k < max_results) results[k] = c;
                k++;
                if (e == cudaSuccess && c.ms < best.ms) best = c;
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (nresults) *nresults = k;
    if (e != cudaSuccess) return fem::record_cuda_error(e);
    b->cfg = best;
    return FEM_OK;
}

int fem_batch_graph_launch(fem_batch *b, void *stream) {
    if (!b) return FEM_EINVAL;
    cudaError_t e = cudaSuccess;
    const bool stale = !b->graph_exec || b->graph_cfg.threads != b->cfg.threads || b->graph_cfg.group != b->cfg.group ||
                       b->graph_cfg.order != b->cfg.order || b->graph_cfg.layout != b->cfg.layout;
    if (stale) {
        if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->graph_exec = nullptr;
        b->graph = nullptr;
        e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = fem::launch(b, b->cfg, b->capture_stream);
            e = cudaStreamEndCapture(b->capture_stream, &b->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
        if (e != cudaSuccess) return fem::record_cuda_error(e);
        b->graph_cfg = b->cfg;
    }
    e = cudaGraphLaunch(b->graph_exec, (cudaStream_t)stream);
    return e == cudaSuccess ? FEM_OK : fem::record_cuda_error(e);
}

}  // extern "C"
