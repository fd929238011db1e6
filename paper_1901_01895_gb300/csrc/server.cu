// Request server: continuous batching of RK4IP propagation requests on one GPU.
//
// A design sweep submits many independent link simulations (launch power, length, mode
// count, N_t).  Each is the RK4IP of Eq. 4a-4f on its own fields; they share nothing but
// the fiber description.  The server keeps, per shape (fiber type, N_t, step size h,
// propagator sharing between polarisations), a pool of B request slots on the device:
//
//   fields  [P][B][N_t]   slot b of field f is row f*B + b, so the B slots sit side by
//                         side on the time axis of each field; the Kerr kernels (pointwise
//                         in t) see one problem of B*N_t samples, and the linear-step
//                         kernel one row per (field, slot) with that slot's propagator row;
//   E       [P>>s][B][N_t] per-slot propagator exp(h/2 D) (each request has its own betas,
//                         loss and dt);
//   steps   [B]           steps left per slot, in device memory.
//
// One graph per pool holds K RK4IP steps, each followed by a tick that decrements the
// positive step counters.  Every kernel of a step skips the rows (linear step) and sample
// tiles (Kerr) whose slot has no steps left, so a slot that finishes inside a graph stays
// untouched for the rest of it, and the same graph serves any set of occupied slots.
//
// A worker thread drives the pools: it admits pending requests into free slots (copies
// the fields in, builds the slot's propagator rows, then sets its step counter on the
// pool's compute stream, between graphs), keeps up to two graphs in flight per pool,
// reads back the step counters after each graph, and copies finished slots out on a
// second stream while the next graph runs.  Pools are created when a request of a new
// shape arrives and the HBM budget allows; idle pools are freed to make room.  Requests
// admitted while others run join the next graph of their pool: their work overlaps
// with the requests already on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mmf.h"
#include "ctx.h"
#include "kernels.h"

using namespace mmf;

namespace {

using Clock = std::chrono::steady_clock;

struct FiberType {
    int n_modes = 0, n_pol = 0;
    std::vector<double> S;
    std::vector<int32_t> parity;
    bool has_parity = false;
    double gamma = 0;
    unsigned flags = 0;
};

enum { RQ_PENDING = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Req {
    uint64_t id = 0;
    int fiber = 0;
    std::vector<double> betas;   // [P][4]
    double alpha = 0, dt = 0, h = 0;
    int n_steps = 0;
    int64_t N_t = 0;
    int e_shift = 0;
    const void* in = nullptr;
    void* out = nullptr;
    int state = RQ_PENDING;      // guarded by the server mutex
    int err = MMF_OK;
    std::string msg;
    Clock::time_point t_submit, t_admit, t_done;
};

struct Pool;

}  // namespace

struct mmf_server {
    int device = 0;
    size_t budget = 0;           // bytes the pools may hold
    int max_slots = 0;           // running requests over all pools (0 = no limit)
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    // guarded by mu
    std::vector<FiberType> fibers;
    std::deque<Req*> pending;
    std::unordered_map<uint64_t, Req*> reqs;
    uint64_t next_id = 1;
    uint64_t n_done = 0, n_failed = 0;
    double fs_steps = 0;         // field-sample steps of completed requests
    uint64_t graph_launches = 0, kernel_launches = 0;
    int n_pools = 0, running = 0, peak_running = 0;
    size_t used = 0;
    int fatal = MMF_OK;
    std::string fatal_msg;
    // worker only
    std::vector<Pool*> pools;
};

namespace {

struct Chunk {
    cudaEvent_t ev = nullptr;
    int* snap = nullptr;          // pinned [B + 1]: steps left, then the device status word
    uint64_t seq = 0;
};

enum { SL_FREE = 0, SL_RUNNING = 1, SL_DRAINING = 2 };

struct Pool {
    int fiber = 0;
    int64_t N_t = 0;
    double h = 0;
    int e_shift = 0;
    int B = 0, P = 0, K = 1, e_rows = 0;
    mmf_ctx* ctx = nullptr;
    float2* A = nullptr;          // [P][B][N_t]
    int* d_steps = nullptr;       // [B]
    int* h_steps = nullptr;       // pinned [B] admission values
    double* h_betas = nullptr;    // pinned [B][P][4]
    cudaStream_t stream = nullptr;    // graphs and step counters
    cudaStream_t cstream = nullptr;   // admission and drain copies
    cudaGraphExec_t graph = nullptr;
    std::vector<Req*> slot;
    std::vector<int> state;
    std::vector<uint64_t> admit_seq;  // chunks launched before the slot's step counter was set
    std::vector<int> left_est;        // steps not yet covered by launched graphs
    std::vector<cudaEvent_t> ev_admit, ev_drain;
    Chunk chunk[2];
    int head = 0, inflight = 0;
    uint64_t launched = 0;
    int running = 0, draining = 0;
    size_t bytes = 0;
    Clock::time_point last_used;
};

constexpr int FIELD_COPIES = 7;   // fields + six scratch copies per slot

size_t slot_bytes(int P, int e_rows, int64_t N) {
    // plus the linear step's scratch copy above N_t = 2^14
    const int copies = FIELD_COPIES + (lin_needs_scratch(N) ? 1 : 0);
    return (size_t)copies * P * N * sizeof(float2) + (size_t)e_rows * N * sizeof(float4) + (size_t)P * 32 + 64;
}

// Slots per pool: enough requests side by side for ~2^23 field samples per launch
// (a full GPU for the linear-step and Kerr kernels), at least 2, at most 64.
int pool_slots(const mmf_server* s, int P, int64_t N) {
    int64_t b = ((int64_t)1 << 23) / ((int64_t)P * N);
    b = std::max<int64_t>(2, std::min<int64_t>(64, b));
    if (s->max_slots > 0) b = std::min<int64_t>(b, s->max_slots);
    return (int)b;
}

// RK4IP steps per graph: about 2^25 field-sample steps per graph, 1 to 16.
int pool_graph_steps(int P, int B, int64_t N) {
    int64_t k = ((int64_t)1 << 25) / ((int64_t)P * B * N);
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, k));
}

void free_pool(Pool* p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->cstream) cudaStreamSynchronize(p->cstream);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    for (auto& c : p->chunk) {
        if (c.ev) cudaEventDestroy(c.ev);
        if (c.snap) cudaFreeHost(c.snap);
    }
    for (auto e : p->ev_admit)
        if (e) cudaEventDestroy(e);
    for (auto e : p->ev_drain)
        if (e) cudaEventDestroy(e);
    if (p->ctx) ctx_free(p->ctx);
    cudaFree(p->A);
    cudaFree(p->d_steps);
    if (p->h_steps) cudaFreeHost(p->h_steps);
    if (p->h_betas) cudaFreeHost(p->h_betas);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (p->cstream) cudaStreamDestroy(p->cstream);
    delete p;
}

// Builds a pool for r's shape; returns nullptr with a message on failure.
Pool* make_pool(mmf_server* s, const FiberType& ft, const Req* r, std::string* why) {
    Pool* p = new (std::nothrow) Pool();
    if (!p) {
        *why = "host allocation failed";
        return nullptr;
    }
    const int P = ft.n_modes * ft.n_pol;
    p->fiber = r->fiber;
    p->N_t = r->N_t;
    p->h = r->h;
    p->e_shift = r->e_shift;
    p->P = P;
    p->B = pool_slots(s, P, r->N_t);
    p->K = pool_graph_steps(P, p->B, r->N_t);
    auto bail = [&](const std::string& m) -> Pool* {
        *why = m;
        free_pool(p);
        return nullptr;
    };
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking) != cudaSuccess)
        return bail("stream creation failed");
    int rc = ctx_create(&p->ctx, ft.n_modes, ft.n_pol, ft.S.data(), ft.has_parity ? ft.parity.data() : nullptr, nullptr,
                        0.0, ft.gamma, r->N_t, r->dt, ft.flags, p->stream, p->B, r->e_shift);
    if (rc != MMF_OK) return bail(std::string("pool: ") + mmf_last_error());
    p->e_rows = p->ctx->e_rows;
    const size_t fbytes = sizeof(float2) * (size_t)P * p->B * r->N_t;
    if (cudaMalloc(&p->A, fbytes) != cudaSuccess || cudaMalloc(&p->d_steps, sizeof(int) * p->B) != cudaSuccess)
        return bail("pool field allocation failed");
    if (cudaMemset(p->A, 0, fbytes) != cudaSuccess || cudaMemset(p->d_steps, 0, sizeof(int) * p->B) != cudaSuccess)
        return bail("pool clear failed");
    if (cudaMallocHost(&p->h_steps, sizeof(int) * p->B) != cudaSuccess ||
        cudaMallocHost(&p->h_betas, sizeof(double) * 4 * P * p->B) != cudaSuccess)
        return bail("pinned allocation failed");
    for (auto& c : p->chunk) {
        if (cudaEventCreateWithFlags(&c.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&c.snap, sizeof(int) * (p->B + 1)) != cudaSuccess)
            return bail("pinned allocation failed");
    }
    p->ev_admit.assign(p->B, nullptr);
    p->ev_drain.assign(p->B, nullptr);
    for (int b = 0; b < p->B; ++b)
        if (cudaEventCreateWithFlags(&p->ev_admit[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_drain[b], cudaEventDisableTiming) != cudaSuccess)
            return bail("event creation failed");
    p->slot.assign(p->B, nullptr);
    p->state.assign(p->B, SL_FREE);
    p->admit_seq.assign(p->B, 0);
    p->left_est.assign(p->B, 0);
    p->ctx->d_slot_steps = p->d_steps;
    // the graph: K x (RK4IP step + tick)
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(p->ctx->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bail("begin capture failed");
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < p->K && e == cudaSuccess; ++k) {
        e = ctx_enqueue_step(p->ctx, p->A, p->h, p->ctx->cap);
        if (e == cudaSuccess) e = slot_tick_launch(p->d_steps, p->B, p->ctx->cap);
    }
    cudaError_t e2 = cudaStreamEndCapture(p->ctx->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bail(std::string("capture pool graph: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&p->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        p->graph = nullptr;
        return bail(std::string("instantiate pool graph: ") + cudaGetErrorString(e));
    }
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return bail("pool set-up failed");
    p->bytes = p->ctx->scratch_bytes + fbytes + sizeof(int) * p->B;
    p->last_used = Clock::now();
    return p;
}

void finish(mmf_server* s, Req* r, int err, const std::string& msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_done = Clock::now();
    r->err = err;
    r->msg = msg;
    r->state = err == MMF_OK ? RQ_DONE : RQ_FAILED;
    if (err == MMF_OK) {
        ++s->n_done;
        const FiberType& ft = s->fibers[r->fiber];
        s->fs_steps += (double)ft.n_modes * ft.n_pol * (double)r->N_t * r->n_steps;
    } else {
        ++s->n_failed;
    }
    s->cv.notify_all();
}

void set_fatal(mmf_server* s, cudaError_t e, const char* what) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal == MMF_OK) {
        s->fatal = MMF_ECUDA;
        s->fatal_msg = std::string(what) + ": " + cudaGetErrorString(e);
    }
}

bool pool_matches(const Pool* p, const Req* r) {
    return p->fiber == r->fiber && p->N_t == r->N_t && p->h == r->h && p->e_shift == r->e_shift;
}

int first_free(const Pool* p) {
    for (int b = 0; b < p->B; ++b)
        if (p->state[b] == SL_FREE) return b;
    return -1;
}

// Admission: place pending requests into free slots of their pool, creating pools as the
// HBM budget allows (freeing idle pools of other shapes when it does not).
bool admit(mmf_server* s) {
    std::vector<Req*> cand;
    int running;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        cand.assign(s->pending.begin(), s->pending.end());
        running = s->running;
    }
    bool progress = false;
    std::vector<Req*> admitted;
    for (Req* r : cand) {
        if (s->max_slots > 0 && running >= s->max_slots) break;
        // a request that waits for memory holds back every later one (first come, first
        // served), so that a busy shape cannot keep its pool alive and starve it
        Pool* p = nullptr;
        bool have_shape = false;
        for (Pool* q : s->pools)
            if (pool_matches(q, r)) {
                have_shape = true;
                if (first_free(q) >= 0) {
                    p = q;
                    break;
                }
            }
        if (!p && have_shape) continue;   // wait for a slot of this shape
        if (!p) {
            FiberType ft;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                ft = s->fibers[r->fiber];
            }
            const int P = ft.n_modes * ft.n_pol;
            const int B = pool_slots(s, P, r->N_t);
            // slots + twiddles + a bound on the Kerr tables (M^4 bytes covers the FP32 pair
            // blocks and the BF16 hi/lo tensor-core tiles) + 1 MiB of small tables
            const size_t M4 = (size_t)ft.n_modes * ft.n_modes * ft.n_modes * ft.n_modes;
            const size_t need = (size_t)B * slot_bytes(P, P >> r->e_shift, r->N_t) + sizeof(float4) * r->N_t + M4 +
                                ((size_t)1 << 20);
            if (need > s->budget) {
                // can never fit: fail it rather than wait forever
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->pending.erase(std::find(s->pending.begin(), s->pending.end(), r));
                }
                finish(s, r, MMF_EBUSY, "request shape does not fit in the server's HBM budget");
                progress = true;
                continue;
            }
            // free idle pools (least recently used first) until the new one fits
            while (s->used + need > s->budget) {
                Pool* victim = nullptr;
                for (Pool* q : s->pools)
                    if (q->running == 0 && q->draining == 0 && q->inflight == 0 &&
                        (!victim || q->last_used < victim->last_used))
                        victim = q;
                if (!victim) break;
                s->pools.erase(std::find(s->pools.begin(), s->pools.end(), victim));
                const size_t vb = victim->bytes;
                free_pool(victim);
                std::lock_guard<std::mutex> lk(s->mu);
                s->used -= vb;
                s->n_pools = (int)s->pools.size();
            }
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            if (s->used + need > s->budget || need + ((size_t)256 << 20) > free_b) break;
            std::string why;
            p = make_pool(s, ft, r, &why);
            if (!p) {
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->pending.erase(std::find(s->pending.begin(), s->pending.end(), r));
                }
                finish(s, r, MMF_ENOMEM, why);
                progress = true;
                continue;
            }
            s->pools.push_back(p);
            std::lock_guard<std::mutex> lk(s->mu);
            s->used += p->bytes;
            s->n_pools = (int)s->pools.size();
        }
        const int b = first_free(p);
        const int P = p->P;
        const int64_t N = p->N_t;
        // slot inputs on the copy stream: betas, propagator rows, fields
        double* hb = p->h_betas + (size_t)b * P * 4;
        std::memcpy(hb, r->betas.data(), sizeof(double) * 4 * P);
        double* db = p->ctx->d_betas + (size_t)b * P * 4;
        cudaError_t e = cudaMemcpyAsync(db, hb, sizeof(double) * 4 * P, cudaMemcpyHostToDevice, p->cstream);
        if (e == cudaSuccess)
            e = propagator_table_launch(p->ctx->d_E + (size_t)b * N, db, p->e_rows, 1 << p->e_shift, (int)N, r->dt,
                                        r->alpha, r->h / 2, (size_t)p->B * N, p->cstream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(p->A + (size_t)b * N, sizeof(float2) * p->B * N, r->in, sizeof(float2) * N,
                                  sizeof(float2) * N, P, cudaMemcpyDefault, p->cstream);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_admit[b], p->cstream);
        // the step counter on the compute stream, between graphs
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->ev_admit[b], 0);
        p->h_steps[b] = r->n_steps;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_steps + b, p->h_steps + b, sizeof(int), cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) {
            set_fatal(s, e, "admission");
            return true;
        }
        p->slot[b] = r;
        p->state[b] = SL_RUNNING;
        p->admit_seq[b] = p->launched;
        p->left_est[b] = r->n_steps;
        ++p->running;
        p->last_used = Clock::now();
        ++running;
        admitted.push_back(r);
        progress = true;
    }
    if (!admitted.empty()) {
        std::lock_guard<std::mutex> lk(s->mu);
        const Clock::time_point now = Clock::now();
        for (Req* r : admitted) {
            s->pending.erase(std::find(s->pending.begin(), s->pending.end(), r));
            r->state = RQ_RUNNING;
            r->t_admit = now;
            ++s->kernel_launches;   // propagator rows of the slot
        }
        s->running += (int)admitted.size();
        s->peak_running = std::max(s->peak_running, s->running);
    }
    return progress;
}

// Keep up to two graphs in flight per pool while any slot has steps not yet launched.
bool launch(mmf_server* s) {
    bool progress = false;
    for (Pool* p : s->pools) {
        while (p->inflight < 2) {
            bool need = false;
            for (int b = 0; b < p->B; ++b) need |= p->state[b] == SL_RUNNING && p->left_est[b] > 0;
            if (!need) break;
            Chunk& c = p->chunk[(p->head + p->inflight) % 2];
            cudaError_t e = cudaGraphLaunch(p->graph, p->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c.snap, p->d_steps, sizeof(int) * p->B, cudaMemcpyDeviceToHost, p->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c.snap + p->B, p->ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
            if (e == cudaSuccess) e = cudaEventRecord(c.ev, p->stream);
            if (e != cudaSuccess) {
                set_fatal(s, e, "graph launch");
                return true;
            }
            c.seq = p->launched++;
            ++p->inflight;
            for (int b = 0; b < p->B; ++b)
                if (p->state[b] == SL_RUNNING) p->left_est[b] -= p->K;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                ++s->graph_launches;
                // per step: four Kerr evaluations and four linear steps (three launches each at
                // N_t above 2^14), then the slot tick
                const uint64_t per_step = 4 + 4 * (lin_needs_scratch(p->N_t) ? 3 : 1) + 1;
                s->kernel_launches += (uint64_t)p->K * per_step;
            }
            progress = true;
        }
    }
    return progress;
}

// Completed graphs: slots whose counter reached zero are copied out; completed copies
// finish their requests and free the slot.
bool harvest(mmf_server* s) {
    bool progress = false;
    for (Pool* p : s->pools) {
        while (p->inflight > 0) {
            Chunk& c = p->chunk[p->head];
            cudaError_t q = cudaEventQuery(c.ev);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) {
                set_fatal(s, q, "graph");
                return true;
            }
            p->head = (p->head + 1) % 2;
            --p->inflight;
            progress = true;
            const int status = c.snap[p->B];
            if (status != 0) {
                // a bounded device-side wait of a Kerr kernel gave up: no result of the pool
                // is trusted and its step counters are not reliable, so the server stops
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->fatal == MMF_OK) {
                    s->fatal = MMF_ETIMEOUT;
                    s->fatal_msg = "a bounded device-side wait gave up (code " + std::to_string(status) + ")";
                }
                return true;
            }
            for (int b = 0; b < p->B; ++b) {
                if (p->state[b] != SL_RUNNING || c.seq < p->admit_seq[b]) continue;
                if (c.snap[b] > 0) continue;
                Req* r = p->slot[b];
                cudaError_t e = cudaMemcpy2DAsync(r->out, sizeof(float2) * p->N_t, p->A + (size_t)b * p->N_t,
                                                  sizeof(float2) * p->B * p->N_t, sizeof(float2) * p->N_t, p->P,
                                                  cudaMemcpyDefault, p->cstream);
                if (e == cudaSuccess) e = cudaEventRecord(p->ev_drain[b], p->cstream);
                if (e != cudaSuccess) {
                    set_fatal(s, e, "drain");
                    return true;
                }
                p->state[b] = SL_DRAINING;
                --p->running;
                ++p->draining;
            }
        }
        for (int b = 0; b < p->B; ++b) {
            if (p->state[b] != SL_DRAINING) continue;
            cudaError_t q = cudaEventQuery(p->ev_drain[b]);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                set_fatal(s, q, "drain copy");
                return true;
            }
            Req* r = p->slot[b];
            p->slot[b] = nullptr;
            p->state[b] = SL_FREE;
            --p->draining;
            p->last_used = Clock::now();
            {
                std::lock_guard<std::mutex> lk(s->mu);
                --s->running;
            }
            finish(s, r, MMF_OK, "");
            progress = true;
        }
    }
    return progress;
}

void fail_all(mmf_server* s) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->reqs) {
        Req* r = kv.second;
        if (r->state == RQ_PENDING || r->state == RQ_RUNNING) {
            r->state = RQ_FAILED;
            r->err = s->fatal;
            r->msg = s->fatal_msg;
            r->t_done = Clock::now();
            ++s->n_failed;
        }
    }
    s->pending.clear();
    s->running = 0;
    s->cv.notify_all();
}

void worker_main(mmf_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            if (s->fatal != MMF_OK) {
                lk.unlock();
                fail_all(s);
                lk.lock();
                s->cv.wait(lk, [&] { return s->stop; });
                break;
            }
            bool busy = !s->pending.empty();
            for (Pool* p : s->pools) busy |= p->running > 0 || p->draining > 0 || p->inflight > 0;
            if (!busy) {
                s->cv.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->stop || !s->pending.empty(); });
                continue;
            }
        }
        bool progress = harvest(s);
        progress |= admit(s);
        progress |= launch(s);
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (Pool* p : s->pools) free_pool(p);
    s->pools.clear();
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" {

int mmf_server_create(mmf_server_handle* out, size_t hbm_budget_bytes, int max_slots) {
    if (!out) return ctx_fail(MMF_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 0) return ctx_fail(MMF_EINVAL, "max_slots must be >= 0");
    mmf_server* s = new (std::nothrow) mmf_server();
    if (!s) return ctx_fail(MMF_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return ctx_fail(MMF_ECUDA, "no CUDA device");
    }
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete s;
        return ctx_fail(MMF_ECUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
    }
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : free_b / 10 * 9;
    s->max_slots = max_slots;
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        delete s;
        return ctx_fail(MMF_ENOMEM, "could not start the server thread");
    }
    *out = s;
    return MMF_OK;
}

int mmf_server_add_fiber(mmf_server_handle s, int n_modes, int n_pol, const double* S_plmn,
                         const int32_t* parity_class, double gamma, unsigned flags, int* fiber_id) {
    if (!s || !S_plmn || !fiber_id) return ctx_fail(MMF_EINVAL, "NULL argument");
    if (n_modes < 1 || (n_pol != 1 && n_pol != 2)) return ctx_fail(MMF_EINVAL, "bad mode or polarisation count");
    if (n_modes * n_pol > 1023) return ctx_fail(MMF_EINVAL, "at most 1023 fields");
    if (!std::isfinite(gamma)) return ctx_fail(MMF_EINVAL, "gamma must be finite");
    FiberType ft;
    ft.n_modes = n_modes;
    ft.n_pol = n_pol;
    const size_t M4 = (size_t)n_modes * n_modes * n_modes * n_modes;
    ft.S.assign(S_plmn, S_plmn + M4);
    for (double v : ft.S)
        if (!std::isfinite(v)) return ctx_fail(MMF_EINVAL, "S_plmn has a non-finite entry");
    if (parity_class) {
        ft.parity.assign(parity_class, parity_class + n_modes);
        ft.has_parity = true;
    }
    ft.gamma = gamma;
    ft.flags = flags;
    std::lock_guard<std::mutex> lk(s->mu);
    s->fibers.push_back(std::move(ft));
    *fiber_id = (int)s->fibers.size() - 1;
    return MMF_OK;
}

int mmf_server_submit(mmf_server_handle s, const mmf_request* req, uint64_t* id) {
    if (!s || !req || !id) return ctx_fail(MMF_EINVAL, "NULL argument");
    if (!req->fields_in || !req->fields_out || !req->betas) return ctx_fail(MMF_EINVAL, "NULL request pointer");
    if (!pow2(req->N_t) || req->N_t < 16 || req->N_t > (1 << 17))
        return ctx_fail(MMF_EINVAL, "N_t must be a power of two in [16, 131072]");
    if (req->n_steps < 1) return ctx_fail(MMF_EINVAL, "n_steps must be >= 1");
    if (!(req->dt > 0) || !std::isfinite(req->dt) || !std::isfinite(req->L) || !std::isfinite(req->alpha))
        return ctx_fail(MMF_EINVAL, "dt, L and alpha must be finite (dt > 0)");
    Req* r = new (std::nothrow) Req();
    if (!r) return ctx_fail(MMF_ENOMEM, "host allocation failed");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != MMF_OK) {
        delete r;
        return ctx_fail(s->fatal, s->fatal_msg);
    }
    if (req->fiber < 0 || req->fiber >= (int)s->fibers.size()) {
        delete r;
        return ctx_fail(MMF_EINVAL, "unknown fiber id");
    }
    const FiberType& ft = s->fibers[req->fiber];
    const int P = ft.n_modes * ft.n_pol;
    r->fiber = req->fiber;
    r->betas.assign(req->betas, req->betas + 4 * P);
    for (double v : r->betas)
        if (!std::isfinite(v)) {
            delete r;
            return ctx_fail(MMF_EINVAL, "betas has a non-finite entry");
        }
    r->alpha = req->alpha;
    r->dt = req->dt;
    r->n_steps = req->n_steps;
    r->h = req->L / req->n_steps;
    r->N_t = req->N_t;
    r->e_shift = 0;
    if (ft.n_pol == 2) {
        bool same = true;
        for (int m = 0; m < ft.n_modes && same; ++m)
            same = std::memcmp(&r->betas[8 * m], &r->betas[8 * m + 4], 4 * sizeof(double)) == 0;
        r->e_shift = same ? 1 : 0;
    }
    r->in = req->fields_in;
    r->out = req->fields_out;
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    *id = r->id;
    s->cv.notify_all();
    return MMF_OK;
}

int mmf_server_poll(mmf_server_handle s, uint64_t id, int* state, double* latency_ms) {
    if (!s || !state) return ctx_fail(MMF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return ctx_fail(MMF_EINVAL, "unknown request id");
    const Req* r = it->second;
    *state = r->state;
    if (latency_ms)
        *latency_ms = r->state >= RQ_DONE ? std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count() : -1.0;
    if (r->state == RQ_FAILED) return ctx_fail(r->err, r->msg);
    return MMF_OK;
}

int mmf_server_wait(mmf_server_handle s, uint64_t id, double timeout_s, double* latency_ms) {
    if (!s) return ctx_fail(MMF_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return ctx_fail(MMF_EINVAL, "unknown request id");
    Req* r = it->second;
    const auto done = [&] { return r->state >= RQ_DONE; };
    if (timeout_s < 0) {
        s->cv.wait(lk, done);
    } else if (!s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        return ctx_fail(MMF_ETIMEOUT, "request not finished within the timeout");
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (r->state == RQ_FAILED) return ctx_fail(r->err, r->msg);
    return MMF_OK;
}

int mmf_server_release(mmf_server_handle s, uint64_t id) {
    if (!s) return ctx_fail(MMF_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return ctx_fail(MMF_EINVAL, "unknown request id");
    if (it->second->state < RQ_DONE) return ctx_fail(MMF_EBUSY, "request still pending or running");
    delete it->second;
    s->reqs.erase(it);
    return MMF_OK;
}

int mmf_server_stats(mmf_server_handle s, mmf_server_stats_t* out) {
    if (!s || !out) return ctx_fail(MMF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->completed = s->n_done;
    out->failed = s->n_failed;
    out->pending = s->pending.size();
    out->running = s->running;
    out->peak_running = s->peak_running;
    out->pools = s->n_pools;
    out->bytes_in_use = s->used;
    out->field_sample_steps = s->fs_steps;
    out->graph_launches = s->graph_launches;
    out->kernel_launches = s->kernel_launches;
    return s->fatal;
}

int mmf_server_destroy(mmf_server_handle s) {
    if (!s) return MMF_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return MMF_OK;
}

}  // extern "C"
