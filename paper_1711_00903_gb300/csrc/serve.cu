// Continuous-batching server of Helmholtz solves (BP3.5 or BP3.0 operator,
// FP64 or mixed-precision Jacobi-PCG) on one GPU.
//
// Requests arrive at any time (fem_serve_submit) and wait in a queue, served
// first come first served or least estimated work first.
// fem_serve_progress, called in the caller's loop, never blocks: it admits
// queued requests while a slot is free and their device footprint fits the
// HBM budget, moves every admitted solve on by one step when its previous
// step has finished (each slot has its own stream, so the GPU works on
// several solves at once), and retires finished solves (copy of x to the
// caller's host buffer, stream-ordered release of their device memory).
//
// A solve in the mix executes exactly the kernels, on exactly the data, that
// it executes alone (every reduction is deterministic and per request, and
// the iterate freezes on the device at convergence), so its result is
// bit-identical alone and in the mix.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "fem_internal.h"

namespace {

struct Request {
    fem_serve_request req;
    fem_serve_result res;
    double work;  // est_work(req)
    // device state while running
    int slot;
    fem_pcg *pcg;
    double *verts_d, *G, *rhs_d, *x_d;
    bool finishing;  // solve finished, x on its way to the host
    bool cancel;     // cancelled while running: retire once no step is in flight
    cudaEvent_t done_ev;
};

struct Slot {
    cudaStream_t stream;
    double *hscal;  // pinned scalars lent to the slot's solver
    bool busy;
};

int64_t footprint(const fem_serve_request &r) {
    const int64_t n = r.N + 1, m = r.N + 2;
    const int64_t np = n * n * n, gpts = (r.op == FEM_OP_BP30) ? m * m * m : np;
    const int64_t len = r.E * np;
    int64_t bytes = 8 * (24 * r.E + 7 * r.E * gpts + 2 * len);  // vertices, factors, rhs, x
    bytes += 8 * 3 * (r.E + 3 * 152 * 8);                        // partial sums (upper bound)
    if (r.mode == FEM_PCG_FP64)
        bytes += 8 * 5 * len;  // q, r, z, p, 1/diag
    else  // q (FP64); FP32 (or FP16) factors and 6 FP32 vectors
        bytes += 8 * len + (r.mode == FEM_PCG_MIXED16 ? 2 : 4) * 7 * r.E * gpts + 4 * 6 * len;
    return bytes + 64 * 1024;
}

// Estimated device work of a solve, for FEM_SERVE_SHORTEST: the per-iteration
// cost (E (N+1)^3, 2.5 times more for BP3.0, about 0.15 of it for the FP32
// inner iterations of the mixed modes) times the Jacobi-PCG iteration count,
// which grows like the square root of the condition number, roughly
// N E^(1/3) on these meshes, and like ln(1/tol).
double est_work(const fem_serve_request &r) {
    const double n = r.N + 1.0;
    double w = std::pow((double)r.E, 4.0 / 3.0) * n * n * n * r.N * std::log(1.0 / r.tol);
    if (r.op == FEM_OP_BP30) w *= 2.5;
    if (r.mode == FEM_PCG_MIXED_TC)
        w *= 0.3;  // the tensor-core inner operator measured about twice the FP32 one's time
    else if (r.mode != FEM_PCG_FP64)
        w *= 0.15;
    return w;
}

double now_s(const std::chrono::steady_clock::time_point &t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct fem_server {
    fem_serve_opts opts;
    std::chrono::steady_clock::time_point t0;
    fem_basis *bases[FEM_MAX_N + 1];
    std::vector<Slot> slots;
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    std::vector<int64_t> running;
    int64_t next_id;
    int64_t in_use;
    int device;
};

namespace {

cudaError_t admit(fem_server *s, Request &R, int slot) {
    const fem_serve_request &q = R.req;
    Slot &S = s->slots[slot];
    cudaStream_t st = S.stream;
    const fem_basis *b = s->bases[q.N];
    const int64_t n = q.N + 1, m = q.N + 2, np = n * n * n;
    const int64_t gpts = (q.op == FEM_OP_BP30) ? m * m * m : np;
    const int64_t len = q.E * np;
    cudaError_t e = cudaMallocAsync((void **)&R.verts_d, sizeof(double) * 24 * q.E, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&R.G, sizeof(double) * 7 * q.E * gpts, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&R.rhs_d, sizeof(double) * len, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&R.x_d, sizeof(double) * len, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.verts_d, q.verts, sizeof(double) * 24 * q.E, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.rhs_d, q.rhs, sizeof(double) * len, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.x_d, 0, sizeof(double) * len, st);
    if (e == cudaSuccess)
        e = fem::launch_geofacs(b, q.op == FEM_OP_BP30 ? FEM_GEO_BP30 : FEM_GEO_BP35, q.E, R.verts_d, R.G, nullptr, st);
    if (e != cudaSuccess) return e;
    int r = fem::pcg_new(b, q.op, q.E, R.G, q.lambda, q.mode, &R.pcg);
    if (r != FEM_OK) return cudaErrorInvalidValue;
    e = fem::pcg_create_on(R.pcg, st, S.hscal);
    if (e != cudaSuccess) return e;
    fem_pcg_opts o;
    std::memset(&o, 0, sizeof o);
    o.tol = q.tol;
    o.check_every = s->opts.check_every;
    e = fem::pcg_begin(R.pcg, R.rhs_d, R.x_d, &o, st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R.done_ev, cudaEventDisableTiming);
    return e;
}

void release(fem_server *s, Request &R) {
    if (R.slot < 0) return;
    cudaStream_t st = s->slots[R.slot].stream;
    if (R.pcg) {
        fem::pcg_release_on(R.pcg, st);
        fem::pcg_delete(R.pcg);
        R.pcg = nullptr;
    }
    double *bufs[] = {R.verts_d, R.G, R.rhs_d, R.x_d};
    for (double *p : bufs)
        if (p) cudaFreeAsync(p, st);
    R.verts_d = R.G = R.rhs_d = R.x_d = nullptr;
    if (R.done_ev) cudaEventDestroy(R.done_ev);
    R.done_ev = nullptr;
    s->slots[R.slot].busy = false;
    R.slot = -1;
    s->in_use -= R.res.bytes;
}

}  // namespace

extern "C" {

int fem_serve_create(const fem_serve_opts *opts, fem_server **out) {
    if (!out) return FEM_EINVAL;
    *out = nullptr;
    fem_serve_opts o;
    o.hbm_budget = (opts && opts->hbm_budget > 0) ? opts->hbm_budget : (int64_t)120 << 30;
    o.max_active = (opts && opts->max_active > 0) ? opts->max_active : 8;
    o.check_every = (opts && opts->check_every > 0) ? opts->check_every : 8;
    o.policy = opts ? opts->policy : FEM_SERVE_FIFO;
    o.max_wait_s = (opts && opts->max_wait_s > 0.0) ? opts->max_wait_s : 2.0;
    if (o.max_active > 256 || (o.policy != FEM_SERVE_FIFO && o.policy != FEM_SERVE_SHORTEST)) return FEM_EINVAL;
    fem_server *s = new (std::nothrow) fem_server();
    if (!s) return FEM_ENOMEM;
    s->opts = o;
    s->t0 = std::chrono::steady_clock::now();
    s->next_id = 1;
    s->in_use = 0;
    std::memset(s->bases, 0, sizeof s->bases);
    cudaError_t e = cudaGetDevice(&s->device);
    int r = FEM_OK;
    for (int N = 1; N <= FEM_MAX_N && r == FEM_OK && e == cudaSuccess; N++) r = fem_basis_setup(N, &s->bases[N]);
    s->slots.resize(o.max_active);
    for (int i = 0; i < o.max_active && e == cudaSuccess && r == FEM_OK; i++) {
        s->slots[i].busy = false;
        e = cudaStreamCreateWithFlags(&s->slots[i].stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&s->slots[i].hscal, sizeof(double) * fem::kPcgScalars);
    }
    if (e != cudaSuccess || r != FEM_OK) {
        fem_serve_destroy(s);
        return r != FEM_OK ? r : fem::record_cuda_error(e);
    }
    *out = s;
    return FEM_OK;
}

double fem_serve_clock(const fem_server *s) { return s ? now_s(s->t0) : 0.0; }

int fem_serve_submit(fem_server *s, const fem_serve_request *req, int64_t *id) {
    if (!s || !req || !id) return FEM_EINVAL;
    const fem_serve_request &q = *req;
    if ((q.op != FEM_OP_BP35 && q.op != FEM_OP_BP30) || q.N < 1 || q.N > FEM_MAX_N || q.E < 1) return FEM_EINVAL;
    if (!q.verts || !q.rhs || !q.x || (q.mode != FEM_PCG_FP64 && q.mode != FEM_PCG_MIXED && q.mode != FEM_PCG_MIXED16 &&
                                     q.mode != FEM_PCG_MIXED_TC))
        return FEM_EINVAL;
    if (!(q.lambda >= 0.0) || !(q.tol > 0.0)) return FEM_EINVAL;
    Request R;
    std::memset((void *)&R, 0, sizeof R);
    R.req = q;
    R.slot = -1;
    R.res.state = FEM_REQ_QUEUED;
    R.res.status = FEM_OK;
    R.res.t_submit = now_s(s->t0);
    R.res.bytes = footprint(q);
    R.work = est_work(q);
    *id = s->next_id++;
    s->reqs[*id] = R;
    s->queue.push_back(*id);
    return FEM_OK;
}

int fem_serve_progress(fem_server *s, int *active, int *queued) {
    if (!s) return FEM_EINVAL;
    cudaSetDevice(s->device);
    // 1. advance or retire the requests in flight
    for (size_t k = 0; k < s->running.size();) {
        Request &R = s->reqs[s->running[k]];
        bool retire = false;
        if (R.cancel && !R.finishing) {
            // no further step is enqueued; the request retires once the step
            // in flight (if any) has finished on its stream
            const int q = fem::pcg_quiescent(R.pcg);
            if (q != 0) {
                R.res.state = FEM_REQ_FAILED;
                R.res.status = q > 0 ? FEM_ECANCELED : fem::record_cuda_error(cudaGetLastError());
                R.res.t_done = now_s(s->t0);
                release(s, R);
                s->running.erase(s->running.begin() + k);
            } else {
                k++;
            }
            continue;
        }
        if (!R.finishing) {
            const int r = fem::pcg_advance(R.pcg, false);
            if (r < 0) {
                R.res.state = FEM_REQ_FAILED;
                R.res.status = fem::record_cuda_error(cudaGetLastError());
                retire = true;
            } else if (r == 1) {
                fem_pcg_info info;
                R.res.status = fem::pcg_status(R.pcg, &info);
                R.res.iters = info.iters;
                R.res.outer = info.outer;
                R.res.relres = info.relres;
                const int64_t np = (int64_t)(R.req.N + 1) * (R.req.N + 1) * (R.req.N + 1);
                cudaStream_t st = s->slots[R.slot].stream;
                cudaError_t e = cudaMemcpyAsync(R.req.x, R.x_d, sizeof(double) * R.req.E * np,
                                                cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaEventRecord(R.done_ev, st);
                if (e != cudaSuccess) {
                    R.res.state = FEM_REQ_FAILED;
                    R.res.status = fem::record_cuda_error(e);
                    retire = true;
                } else {
                    R.finishing = true;
                }
            }
        }
        if (R.finishing && !retire) {
            const cudaError_t q = cudaEventQuery(R.done_ev);
            if (q == cudaSuccess) {
                R.res.t_done = now_s(s->t0);
                R.res.state = (R.res.status == FEM_OK) ? FEM_REQ_DONE : FEM_REQ_FAILED;
                retire = true;
            } else if (q != cudaErrorNotReady) {
                R.res.state = FEM_REQ_FAILED;
                R.res.status = fem::record_cuda_error(q);
                retire = true;
            }
        }
        if (retire) {
            release(s, R);
            s->running.erase(s->running.begin() + k);
        } else {
            k++;
        }
    }
    // 2. admit from the head of the queue (first come, first served), or
    // the least estimated work first (ties by arrival) among the requests
    // that have waited less than max_wait_s: once the oldest request has
    // waited that long it goes first (aging), so a large request is not
    // starved by a stream of smaller ones
    while (!s->queue.empty()) {
        if (s->opts.policy == FEM_SERVE_SHORTEST &&
            now_s(s->t0) - s->reqs[s->queue.front()].res.t_submit < s->opts.max_wait_s) {
            auto best = s->queue.begin();
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
                if (s->reqs[*it].work < s->reqs[*best].work) best = it;
            if (best != s->queue.begin()) {
                const int64_t id = *best;
                s->queue.erase(best);
                s->queue.push_front(id);
            }
        }
        Request &R = s->reqs[s->queue.front()];
        if (R.res.bytes > s->opts.hbm_budget) {  // can never fit
            R.res.state = FEM_REQ_FAILED;
            R.res.status = FEM_ENOMEM;
            R.res.t_done = now_s(s->t0);
            s->queue.pop_front();
            continue;
        }
        int slot = -1;
        for (size_t i = 0; i < s->slots.size(); i++)
            if (!s->slots[i].busy) {
                slot = (int)i;
                break;
            }
        if (slot < 0 || s->in_use + R.res.bytes > s->opts.hbm_budget) break;
        s->slots[slot].busy = true;
        R.slot = slot;
        s->in_use += R.res.bytes;
        R.res.t_admit = now_s(s->t0);
        R.res.state = FEM_REQ_RUNNING;
        const int64_t id = s->queue.front();
        s->queue.pop_front();
        const cudaError_t e = admit(s, R, slot);
        if (e != cudaSuccess) {
            R.res.state = FEM_REQ_FAILED;
            R.res.status = (e == cudaErrorMemoryAllocation) ? FEM_ENOMEM : fem::record_cuda_error(e);
            R.res.t_done = now_s(s->t0);
            release(s, R);
            continue;
        }
        s->running.push_back(id);
    }
    if (active) *active = (int)s->running.size();
    if (queued) *queued = (int)s->queue.size();
    return FEM_OK;
}

int fem_serve_poll(fem_server *s, int64_t id, fem_serve_result *res) {
    if (!s || !res) return FEM_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return FEM_EINVAL;
    *res = it->second.res;
    return FEM_OK;
}

int fem_serve_wait(fem_server *s, int64_t id, double timeout_s, fem_serve_result *res) {
    if (!s || !res || !(timeout_s >= 0.0)) return FEM_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return FEM_EINVAL;
    const double deadline = now_s(s->t0) + timeout_s;
    for (;;) {
        const int st = it->second.res.state;
        if (st == FEM_REQ_DONE || st == FEM_REQ_FAILED) break;
        if (now_s(s->t0) >= deadline) {
            *res = it->second.res;
            return FEM_ETIMEDOUT;
        }
        const int r = fem_serve_progress(s, nullptr, nullptr);
        if (r != FEM_OK) return r;
    }
    *res = it->second.res;
    return FEM_OK;
}

int fem_serve_cancel(fem_server *s, int64_t id) {
    if (!s) return FEM_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return FEM_EINVAL;
    Request &R = it->second;
    if (R.res.state == FEM_REQ_QUEUED) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == id) {
                s->queue.erase(q);
                break;
            }
        R.res.state = FEM_REQ_FAILED;
        R.res.status = FEM_ECANCELED;
        R.res.t_done = now_s(s->t0);
        return FEM_OK;
    }
    if (R.res.state == FEM_REQ_RUNNING && !R.finishing) R.cancel = true;
    return FEM_OK;  // finishing, done or failed: nothing to cancel
}

int64_t fem_serve_in_use(const fem_server *s) { return s ? s->in_use : 0; }

void fem_serve_destroy(fem_server *s) {
    if (!s) return;
    for (int64_t id : s->running) {
        Request &R = s->reqs[id];
        if (R.slot >= 0) cudaStreamSynchronize(s->slots[R.slot].stream);
        release(s, R);
    }
    for (Slot &S : s->slots) {
        if (S.stream) {
            cudaStreamSynchronize(S.stream);
            cudaStreamDestroy(S.stream);
        }
        if (S.hscal) cudaFreeHost(S.hscal);
    }
    for (int N = 1; N <= FEM_MAX_N; N++) fem_basis_free(s->bases[N]);
    delete s;
}

}  // extern "C"
