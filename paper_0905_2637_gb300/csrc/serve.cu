// serve.cu -- request loop with continuous batching.
//
// A request is a short run of the vortex method of Sec. 3: blobs move with
// their own velocity (Eq. 6) and keep their circulation, here with n_steps
// midpoint-RK2 steps, i.e. 2 * n_steps velocity evaluations (Eq. 9 by the
// FMM).  The scheduler thread works in rounds.  Every round it admits queued
// requests while slots and the HBM budget allow (the per-request estimate
// adapts the memory model of Table 1), runs ONE evaluation for every resident
// request in a single batched pass (petfmm_evaluate_batch: all stages launch
// once for the whole mix), applies each request's RK2 stage on the device,
// and retires requests whose last step is done.  Requests that arrive while
// others are on the GPU join at the next round; their state (positions,
// circulations, RK2 copy) stays resident on the device until retirement.
// An instance's arithmetic does not depend on the rest of the batch, so a
// request's result is the same alone and in the mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/petfmm.h"
#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// RK2 stage update: stage 0 saves x_n and moves to the midpoint, stage 1
// completes the step from x_n with the midpoint velocity.
__global__ void k_rk2(int64_t n, int stage, double dt, double *x, double *y, double *xn,
                      double *yn, const double *u, const double *v) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (stage == 0) {
        const double x0 = x[i], y0 = y[i];
        xn[i] = x0;
        yn[i] = y0;
        x[i] = x0 + 0.5 * dt * u[i];
        y[i] = y0 + 0.5 * dt * v[i];
    } else {
        x[i] = xn[i] + dt * u[i];
        y[i] = yn[i] + dt * v[i];
    }
}

constexpr int BBOX_BLOCKS = 64;

// Bounding box of the positions (min x, min y, max x, max y): each block
// reduces a grid-stride share into out[4 * blockIdx.x + 0..3].
__global__ void k_bbox(int64_t n, const double *x, const double *y, double *out) {
    __shared__ double s[4][256];
    double a = INFINITY, b = INFINITY, c = -INFINITY, d = -INFINITY;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        a = fmin(a, x[i]);
        b = fmin(b, y[i]);
        c = fmax(c, x[i]);
        d = fmax(d, y[i]);
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    s[3][threadIdx.x] = d;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + o]);
            s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + o]);
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) out[4 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

// Combines the BBOX_BLOCKS partial boxes of request blockIdx.x.
__global__ void k_bbox_final(const double *part, double *out) {
    if (threadIdx.x != 0) return;
    const double *p = part + size_t(blockIdx.x) * 4 * BBOX_BLOCKS;
    double a = p[0], b = p[1], c = p[2], d = p[3];
    for (int k = 1; k < BBOX_BLOCKS; ++k) {
        a = fmin(a, p[4 * k]);
        b = fmin(b, p[4 * k + 1]);
        c = fmax(c, p[4 * k + 2]);
        d = fmax(d, p[4 * k + 3]);
    }
    out[4 * blockIdx.x] = a;
    out[4 * blockIdx.x + 1] = b;
    out[4 * blockIdx.x + 2] = c;
    out[4 * blockIdx.x + 3] = d;
}

struct Req {
    uint64_t ticket = 0;
    petfmm_request spec{};
    std::vector<double> hx, hy, hg;  // host copies (initial state, then result)
    Clock::time_point t_submit, t_admit, t_done;
    int status = PETFMM_OK;
    bool done = false;
    // resident state
    double *x = nullptr, *y = nullptr, *g = nullptr, *u = nullptr, *v = nullptr, *xn = nullptr,
           *yn = nullptr;
    int levels = 1;
    petfmm_domain dom{};
    int evals_done = 0;
    size_t bytes = 0;
    int rounds = 0;      // rounds this request took part in
    int max_shared = 0;  // most requests resident in one of those rounds (itself included)
};

struct TraceSample {
    double t_ms;  // since the server was created
    int32_t queued, active;
};

}  // namespace

struct petfmm_server {
    size_t budget = 0;
    int max_slots = 0, max_queue = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::map<uint64_t, Req *> all;
    uint64_t next_ticket = 1;
    size_t used = 0;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;
    petfmm_ctx *ctx64 = nullptr, *ctxmx = nullptr;
    double *dbox = nullptr, *hbox = nullptr;
    int box_cap = 0;
    cudaMemPool_t pool = nullptr;  // request state (see free_state)
    // admissions run on their own stream while a round computes; the next
    // round waits for their copies through ev_copy
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_copy = nullptr;
    bool copies_pending = false;
    // timing events around each round's work on the stream (device time)
    cudaEvent_t ev_r0 = nullptr, ev_r1 = nullptr;
    double gpu_ms = 0.0;
    // counters (under mu)
    Clock::time_point t_create;
    uint64_t rounds = 0, submitted = 0, admitted = 0, completed = 0;
    int max_active = 0;
    double sum_active = 0.0, busy_ms = 0.0;
    // host time of the worker by phase: admissions (allocation, copies to
    // the device, domain), launching a round, waiting for it, and the work
    // after it (statuses, domains, completions with their copies back)
    double admit_ms = 0.0, launch_ms = 0.0, wait_ms = 0.0, post_ms = 0.0;
    std::vector<TraceSample> trace;  // one sample per round (its start)
};

namespace {

size_t estimate(int64_t n, int L, int p, int precision) {
    const double lam = (std::ldexp(1.0, 2 * (L + 1)) - 1.0) / 3.0;
    const double leaves = std::ldexp(1.0, 2 * L);
    const size_t per_particle = 56 /* resident x, y, g, u, v, RK2 copy */ + 16 /* sort keys/vals */ +
                                (precision == PETFMM_FP64 ? 24 : 16) /* sorted particles */ + 8;
    const size_t coef = precision == PETFMM_FP64 ? 16 : 8;
    return size_t(n) * per_particle + size_t(2.0 * lam * p * coef) + size_t(leaves * 12.0) +
           size_t((n / 32 + leaves) * 16.0) + (1u << 20);
}

// Request state comes from the server's own stream-ordered memory pool:
// allocating and freeing it does not synchronise the device (cudaMalloc and
// cudaFree would wait for the round in flight), and freed blocks stay in the
// pool for the next admissions.
void free_state(petfmm_server *s, Req *r) {
    double *bufs[] = {r->x, r->y, r->g, r->u, r->v, r->xn, r->yn};
    for (double *b : bufs)
        if (b) cudaFreeAsync(b, s->stream);
    r->x = r->y = r->g = r->u = r->v = r->xn = r->yn = nullptr;
}

// Square domain around the bounding box, with a margin so that blobs can move.
petfmm_domain fit_domain(double x0, double y0, double x1, double y1) {
    double w = std::max(x1 - x0, y1 - y0);
    if (!(w > 0.0)) w = 1.0;
    w *= 1.25;
    petfmm_domain d;
    d.x0 = 0.5 * (x0 + x1) - 0.5 * w;
    d.y0 = 0.5 * (y0 + y1) - 0.5 * w;
    d.width = w;
    return d;
}

bool inside(const petfmm_domain &d, const double *b) {
    return b[0] >= d.x0 && b[1] >= d.y0 && b[2] <= d.x0 + d.width && b[3] <= d.y0 + d.width;
}

// Device state of an admitted request, from the server's pool, and its
// initial positions and strengths copied in on the admission stream (the
// host arrays live in the request until it finishes; the next round waits
// for the copies).  The domain was fitted at submit time.
int admit(petfmm_server *s, Req *r) {
    const int64_t n = r->spec.n;
    const size_t bytes = size_t(n > 0 ? n : 1) * sizeof(double);
    double **bufs[] = {&r->x, &r->y, &r->g, &r->u, &r->v, &r->xn, &r->yn};
    for (double **b : bufs) {
        if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(b), bytes, s->pool, s->cstream) !=
            cudaSuccess) {
            cudaGetLastError();
            free_state(s, r);
            return PETFMM_ENOMEM;
        }
    }
    if (n > 0) {
        if (cudaMemcpyAsync(r->x, r->hx.data(), bytes, cudaMemcpyHostToDevice, s->cstream) != cudaSuccess ||
            cudaMemcpyAsync(r->y, r->hy.data(), bytes, cudaMemcpyHostToDevice, s->cstream) != cudaSuccess ||
            cudaMemcpyAsync(r->g, r->hg.data(), bytes, cudaMemcpyHostToDevice, s->cstream) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize(s->cstream);  // no copy in flight into what is freed
            free_state(s, r);
            return PETFMM_ECUDA;
        }
    }
    s->copies_pending = true;
    r->levels = r->spec.levels > 0 ? r->spec.levels
                                   : petfmm_choose_levels(n, r->spec.order, r->spec.sigma, &r->dom);
    if (r->levels < 1) {
        free_state(s, r);
        return PETFMM_EINVAL;
    }
    return PETFMM_OK;
}

void finish(petfmm_server *s, Req *r, int status) {
    const int64_t n = r->spec.n;
    if (status == PETFMM_OK && n > 0) {
        if (cudaMemcpy(r->hx.data(), r->x, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(r->hy.data(), r->y, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            status = PETFMM_ECUDA;
    }
    free_state(s, r);
    r->hg.clear();
    r->hg.shrink_to_fit();
    std::lock_guard<std::mutex> lk(s->mu);
    s->completed++;
    r->status = status;
    r->t_done = Clock::now();
    r->done = true;
    s->used -= r->bytes;
}

// One round: one evaluation for every resident request, then its RK2 stage.
// launch_round enqueues it (the scheduler then admits new requests while the
// GPU computes); complete_round waits for it and handles its results.
struct Round {
    Clock::time_point t0, t1;
    int rc64 = 0, rcmx = 0;
    bool any64 = false, anymx = false;
};

void launch_round(petfmm_server *s, std::vector<Req *> &act, Round &rd) {
    const Clock::time_point t0 = Clock::now();
    rd.t0 = t0;
    if (s->copies_pending) {  // the copies of the requests admitted last time
        cudaEventRecord(s->ev_copy, s->cstream);
        cudaStreamWaitEvent(s->stream, s->ev_copy, 0);
        s->copies_pending = false;
    }
    cudaEventRecord(s->ev_r0, s->stream);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->rounds++;
        s->max_active = std::max(s->max_active, int(act.size()));
        s->sum_active += double(act.size());
        s->trace.push_back(TraceSample{std::chrono::duration<double, std::milli>(t0 - s->t_create).count(),
                                       int32_t(s->queue.size()), int32_t(act.size())});
        for (Req *r : act) {
            r->rounds++;
            r->max_shared = std::max(r->max_shared, int(act.size()));
        }
    }
    std::vector<petfmm_instance> in64, inmx;
    std::vector<Req *> r64, rmx;
    for (Req *r : act) {
        petfmm_instance it;
        it.domain = r->dom;
        it.levels = r->levels;
        it.order = r->spec.order;
        it.sigma = r->spec.sigma;
        it.n = r->spec.n;
        it.x = r->x; it.y = r->y; it.gamma = r->g; it.u = r->u; it.v = r->v;
        if (r->spec.precision == PETFMM_FP64) { in64.push_back(it); r64.push_back(r); }
        else { inmx.push_back(it); rmx.push_back(r); }
    }
    rd.any64 = !in64.empty();
    rd.anymx = !inmx.empty();
    rd.rc64 = in64.empty() ? 0 : petfmm_evaluate_batch(s->ctx64, int(in64.size()), in64.data());
    rd.rcmx = inmx.empty() ? 0 : petfmm_evaluate_batch(s->ctxmx, int(inmx.size()), inmx.data());
    if ((int)act.size() > s->box_cap) {
        cudaFree(s->dbox);
        cudaFreeHost(s->hbox);
        s->box_cap = std::max<int>(int(act.size()), 2 * s->box_cap);
        // final boxes, then BBOX_BLOCKS partial boxes per request
        cudaMalloc(&s->dbox, size_t(s->box_cap) * 4 * (BBOX_BLOCKS + 1) * sizeof(double));
        cudaMallocHost(&s->hbox, size_t(s->box_cap) * 4 * sizeof(double));
    }
    double *dpart = s->dbox + size_t(s->box_cap) * 4;
    for (size_t i = 0; i < act.size(); ++i) {
        Req *r = act[i];
        const int64_t n = r->spec.n;
        if (n > 0) {
            const int stage = r->evals_done & 1;
            k_rk2<<<unsigned((n + 255) / 256), 256, 0, s->stream>>>(n, stage, r->spec.dt, r->x, r->y,
                                                                    r->xn, r->yn, r->u, r->v);
            k_bbox<<<BBOX_BLOCKS, 256, 0, s->stream>>>(n, r->x, r->y, dpart + i * 4 * BBOX_BLOCKS);
        }
    }
    if (!act.empty())
        k_bbox_final<<<unsigned(act.size()), 32, 0, s->stream>>>(dpart, s->dbox);
    cudaMemcpyAsync(s->hbox, s->dbox, act.size() * 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    cudaEventRecord(s->ev_r1, s->stream);
    rd.t1 = Clock::now();
}

// Requests a round finished, with their statuses: the worker completes them
// (copies back, frees) once the next round is on the GPU.
using Finished = std::vector<std::pair<Req *, int>>;

void complete_round(petfmm_server *s, std::vector<Req *> &act, Round &rd, Finished &fin) {
    const int rc64 = rd.rc64, rcmx = rd.rcmx;
    const Clock::time_point t0 = rd.t0, t1 = Clock::now();
    int st64 = rd.any64 ? petfmm_sync(s->ctx64) : 0;
    int stmx = rd.anymx ? petfmm_sync(s->ctxmx) : 0;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    const Clock::time_point t2 = Clock::now();
    float round_ms = 0.f;
    if (e == cudaSuccess && cudaEventElapsedTime(&round_ms, s->ev_r0, s->ev_r1) != cudaSuccess) {
        cudaGetLastError();
        round_ms = 0.f;
    }
    // A finished request belongs to the caller from the moment finish() marks
    // it done (a poll may release it at once), so it is dropped from the
    // active list here, handed to the worker through fin, and never touched
    // by a round again.
    std::vector<Req *> keep;
    keep.reserve(act.size());
    for (size_t i = 0; i < act.size(); ++i) {
        Req *r = act[i];
        const bool is64 = r->spec.precision == PETFMM_FP64;
        int st = is64 ? (rc64 ? rc64 : st64) : (rcmx ? rcmx : stmx);
        if (e != cudaSuccess) st = PETFMM_ECUDA;
        r->evals_done++;
        if (st != PETFMM_OK) {
            fin.emplace_back(r, st);
            continue;
        }
        if (r->spec.n > 0 && !inside(r->dom, s->hbox + 4 * i)) {
            const double *b = s->hbox + 4 * i;
            if (!(std::isfinite(b[0]) && std::isfinite(b[1]) && std::isfinite(b[2]) && std::isfinite(b[3]))) {
                fin.emplace_back(r, PETFMM_EDOMAIN);
                continue;
            }
            r->dom = fit_domain(b[0], b[1], b[2], b[3]);
        }
        if (r->evals_done >= 2 * r->spec.n_steps) {
            fin.emplace_back(r, PETFMM_OK);
            continue;
        }
        keep.push_back(r);
    }
    act.swap(keep);
    const Clock::time_point t3 = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->busy_ms += std::chrono::duration<double, std::milli>(t3 - t0).count();
    s->gpu_ms += round_ms;
    s->launch_ms += std::chrono::duration<double, std::milli>(rd.t1 - t0).count();
    s->wait_ms += std::chrono::duration<double, std::milli>(t2 - t1).count();
    s->post_ms += std::chrono::duration<double, std::milli>(t3 - t2).count();
}

void worker_main(petfmm_server *s) {
    cudaSetDevice(s->device);
    std::vector<Req *> act;
    // completions of the last round: their copies back to the host (which
    // block this thread) run while the next round computes
    Finished fin;
    auto complete = [&]() {
        if (fin.empty()) return;
        const Clock::time_point tf = Clock::now();
        for (auto &f : fin) finish(s, f.first, f.second);
        fin.clear();
        std::lock_guard<std::mutex> lk(s->mu);
        s->post_ms += std::chrono::duration<double, std::milli>(Clock::now() - tf).count();
    };
    for (;;) {
        if (act.empty()) complete();  // no round to overlap them with
        std::vector<Req *> newly;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            while (!s->stop && act.empty() && s->queue.empty()) s->cv.wait(lk);
            if (s->stop) {
                for (Req *r : s->queue) {
                    r->status = PETFMM_EBUSY;
                    r->done = true;
                    r->t_done = Clock::now();
                }
                s->queue.clear();
                if (act.empty()) break;
            }
            while (!s->queue.empty() && int(act.size() + newly.size()) < s->max_slots &&
                   s->used + s->queue.front()->bytes <= s->budget) {
                Req *r = s->queue.front();
                s->queue.pop_front();
                s->used += r->bytes;
                s->admitted++;
                newly.push_back(r);
            }
        }
        // the resident requests' round goes to the GPU first; the new ones are
        // admitted (device state, copies on the admission stream) while it
        // computes, and join the next round
        Round rd;
        if (!act.empty()) launch_round(s, act, rd);
        complete();
        const Clock::time_point ta = Clock::now();
        std::vector<Req *> joined;
        for (Req *r : newly) {
            int rc = admit(s, r);
            r->t_admit = Clock::now();
            if (rc != PETFMM_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                r->status = rc;
                r->done = true;
                r->t_done = Clock::now();
                s->used -= r->bytes;
                continue;
            }
            if (r->spec.n == 0 || r->spec.n_steps == 0) {
                finish(s, r, PETFMM_OK);
                continue;
            }
            joined.push_back(r);
        }
        if (!newly.empty()) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->admit_ms += std::chrono::duration<double, std::milli>(Clock::now() - ta).count();
        }
        if (!act.empty()) complete_round(s, act, rd, fin);
        act.insert(act.end(), joined.begin(), joined.end());
    }
}

}  // namespace

extern "C" {

size_t petfmm_serve_estimate_bytes(int64_t n, int levels, int order, int precision) {
    if (n < 0 || levels < 1 || levels > petfmm::MAX_L || order < 1 || order > petfmm::MAX_P) return 0;
    return estimate(n, levels, order, precision);
}

int petfmm_serve_create(size_t hbm_budget_bytes, int max_slots, int max_queue, petfmm_server **out) {
    if (!out || max_slots < 1 || max_queue < 1 || hbm_budget_bytes == 0) return PETFMM_EINVAL;
    *out = nullptr;
    petfmm_server *s = new (std::nothrow) petfmm_server();
    if (s) s->t_create = Clock::now();
    if (!s) return PETFMM_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->max_queue = max_queue;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_copy, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&s->ev_r0) != cudaSuccess || cudaEventCreate(&s->ev_r1) != cudaSuccess) {
        cudaGetLastError();
        if (s->ev_r1) cudaEventDestroy(s->ev_r1);
        if (s->ev_r0) cudaEventDestroy(s->ev_r0);
        if (s->ev_copy) cudaEventDestroy(s->ev_copy);
        if (s->cstream) cudaStreamDestroy(s->cstream);
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return PETFMM_ECUDA;
    }
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        uint64_t keep = UINT64_MAX;  // hold freed blocks for reuse
        if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            if (s->pool) cudaMemPoolDestroy(s->pool);
            cudaEventDestroy(s->ev_r0);
            cudaEventDestroy(s->ev_r1);
            cudaEventDestroy(s->ev_copy);
            cudaStreamDestroy(s->cstream);
            cudaStreamDestroy(s->stream);
            delete s;
            return PETFMM_ECUDA;
        }
    }
    const petfmm_domain unit{0.0, 0.0, 1.0};
    int rc = petfmm_create(&unit, 2, 8, 0.01, PETFMM_FP64, PETFMM_F64, s->stream, &s->ctx64);
    if (rc == PETFMM_OK)
        rc = petfmm_create(&unit, 2, 8, 0.01, PETFMM_MIXED, PETFMM_F64, s->stream, &s->ctxmx);
    if (rc != PETFMM_OK) {
        if (s->ctx64) petfmm_destroy(s->ctx64);
        cudaMemPoolDestroy(s->pool);
        cudaEventDestroy(s->ev_r0);
        cudaEventDestroy(s->ev_r1);
        cudaEventDestroy(s->ev_copy);
        cudaStreamDestroy(s->cstream);
        cudaStreamDestroy(s->stream);
        delete s;
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PETFMM_OK;
}

int petfmm_serve_submit(petfmm_server *s, const petfmm_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return PETFMM_EINVAL;
    const petfmm_request &q = *req;
    if (q.n < 0 || (q.n > 0 && (!q.x || !q.y || !q.gamma)) || q.order < 1 || q.order > petfmm::MAX_P ||
        !(q.sigma > 0.0) || !std::isfinite(q.dt) || q.n_steps < 0 || q.levels > petfmm::MAX_L ||
        (q.precision != PETFMM_FP64 && q.precision != PETFMM_MIXED))
        return PETFMM_EINVAL;
    Req *r = new (std::nothrow) Req();
    if (!r) return PETFMM_ENOMEM;
    r->spec = q;
    r->spec.x = r->spec.y = r->spec.gamma = nullptr;
    try {
        r->hx.assign(q.x, q.x + q.n);
        r->hy.assign(q.y, q.y + q.n);
        r->hg.assign(q.gamma, q.gamma + q.n);
    } catch (...) {
        delete r;
        return PETFMM_ENOMEM;
    }
    // the initial domain, here in the caller's thread rather than in the
    // scheduler's: a square 1.25 times the bounding box
    if (q.n > 0) {
        double bx0 = r->hx[0], by0 = r->hy[0], bx1 = bx0, by1 = by0;
        for (int64_t i = 1; i < q.n; ++i) {
            bx0 = std::min(bx0, r->hx[size_t(i)]);
            bx1 = std::max(bx1, r->hx[size_t(i)]);
            by0 = std::min(by0, r->hy[size_t(i)]);
            by1 = std::max(by1, r->hy[size_t(i)]);
        }
        if (!(std::isfinite(bx0) && std::isfinite(bx1) && std::isfinite(by0) && std::isfinite(by1))) {
            delete r;
            return PETFMM_EDOMAIN;
        }
        r->dom = fit_domain(bx0, by0, bx1, by1);
    } else {
        r->dom = petfmm_domain{0.0, 0.0, 1.0};
    }
    // admission estimate with the level the request will use (worst case 10)
    int L = q.levels > 0 ? q.levels : 10;
    if (q.levels <= 0 && q.n > 0) {
        L = std::min(12, std::max(1, int(std::ceil(std::log(double(q.n) / 8.0) / std::log(4.0)))));
    }
    r->bytes = estimate(q.n, L, q.order, q.precision);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r->bytes > s->budget) {
            delete r;
            return PETFMM_ENOMEM;
        }
        if (int(s->queue.size()) >= s->max_queue || s->stop) {
            delete r;
            return PETFMM_EBUSY;
        }
        r->ticket = s->next_ticket++;
        s->submitted++;
        s->queue.push_back(r);
        s->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    s->cv.notify_one();
    return PETFMM_OK;
}

int petfmm_serve_poll(petfmm_server *s, uint64_t ticket, petfmm_result *out) {
    if (!s || !out) return PETFMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return PETFMM_EINVAL;
    Req *r = it->second;
    if (!r->done) return PETFMM_ENOTREADY;
    out->status = r->status;
    out->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    const auto adm = r->t_admit.time_since_epoch().count() ? r->t_admit : r->t_done;
    out->queue_ms = std::chrono::duration<double, std::milli>(adm - r->t_submit).count();
    out->rounds = r->rounds;
    out->max_shared = r->max_shared;
    out->n = r->status == PETFMM_OK ? r->spec.n : 0;
    out->x = r->status == PETFMM_OK ? r->hx.data() : nullptr;
    out->y = r->status == PETFMM_OK ? r->hy.data() : nullptr;
    return PETFMM_OK;
}

int petfmm_serve_release(petfmm_server *s, uint64_t ticket) {
    if (!s) return PETFMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return PETFMM_EINVAL;
    if (!it->second->done) return PETFMM_ENOTREADY;
    delete it->second;
    s->all.erase(it);
    return PETFMM_OK;
}

int petfmm_serve_stats(petfmm_server *s, petfmm_serve_counters *out) {
    if (!s || !out) return PETFMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->rounds = s->rounds;
    out->submitted = s->submitted;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->queued = int32_t(s->queue.size());
    out->max_active = s->max_active;
    out->mean_active = s->rounds ? s->sum_active / double(s->rounds) : 0.0;
    out->busy_ms = s->busy_ms;
    out->gpu_ms = s->gpu_ms;
    out->admit_ms = s->admit_ms;
    out->launch_ms = s->launch_ms;
    out->wait_ms = s->wait_ms;
    out->post_ms = s->post_ms;
    out->up_ms = std::chrono::duration<double, std::milli>(Clock::now() - s->t_create).count();
    return PETFMM_OK;
}

int petfmm_serve_trace(petfmm_server *s, double *t_ms, int32_t *queued, int32_t *active, int cap) {
    if (!s || cap < 0 || (cap > 0 && (!t_ms || !queued || !active))) return PETFMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const int n = int(std::min<size_t>(s->trace.size(), size_t(INT32_MAX)));
    for (int i = 0; i < std::min(n, cap); ++i) {
        t_ms[i] = s->trace[size_t(i)].t_ms;
        queued[i] = s->trace[size_t(i)].queued;
        active[i] = s->trace[size_t(i)].active;
    }
    return n;
}

int petfmm_serve_destroy(petfmm_server *s) {
    if (!s) return PETFMM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->all) {
        free_state(s, kv.second);
        delete kv.second;
    }
    if (s->cstream) cudaStreamSynchronize(s->cstream);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->ev_copy) cudaEventDestroy(s->ev_copy);
    if (s->ev_r0) cudaEventDestroy(s->ev_r0);
    if (s->ev_r1) cudaEventDestroy(s->ev_r1);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    if (s->ctx64) petfmm_destroy(s->ctx64);
    if (s->ctxmx) petfmm_destroy(s->ctxmx);
    if (s->dbox) cudaFree(s->dbox);
    if (s->hbox) cudaFreeHost(s->hbox);
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaGetLastError();
    delete s;
    return PETFMM_OK;
}

}  // extern "C"
