// serve.cu -- the serving loop: simulations submitted as requests, admitted
// against a device-memory budget, kept resident and advanced step by step,
// their final state copied back when done.
//
// Continuous batching without lockstep: every resident simulation has a
// CUDA stream of its own, and a server step launches the next step of each
// simulation whose previous step has finished (read from a CUDA event on its
// stream), so a small job takes many steps while a large one takes one, and
// requests that arrive are admitted between steps as memory and slots free
// up.  Small jobs run on high-priority streams, whose thread blocks the GPU
// schedules first as SMs free up.  A step's latency is its own CUDA-event
// time on its stream, including any time its kernels queued behind other
// jobs' work.
//
// Device memory comes from one caller-allocated arena (the budget) that the
// server sub-allocates first-fit; each resident simulation owns its state
// arrays and its context workspace inside the arena.  Every computation is
// the same sequence of library calls a lone simulation makes
// (sph_rhs_initial, sph_step), so a job's result does not depend on what else
// is resident.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over [0, size) with 256-byte granularity.
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    void init(size_t bytes) {
        size = bytes & ~size_t(255);
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = up256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up256(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t free_bytes() const {
        size_t s = 0;
        for (auto &kv : free_) s += kv.second;
        return s;
    }
};

enum { JOB_QUEUED = 0, JOB_RUNNING = 1, JOB_DONE = 2, JOB_FAILED = 3 };

struct Job {
    uint64_t id = 0;
    int state = JOB_QUEUED;
    int error = SPH_OK;
    int n = 0, n_gas = 0, n_steps = 0, steps_done = 0;
    double dt = 0.0;
    std::vector<double> r, v, e;     // IC on submit, final state when done
    std::vector<float> m, h;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<float> step_ms;
    // device side
    size_t state_off = 0, state_bytes = 0, ws_off = 0, ws_bytes = 0;
    bool has_state = false, has_ws = false;
    SphState st{};
    sph_ctx *ctx = nullptr;
    long long capacity = 0;
    int log2_M = 10;
    int stream_slot = -1;         // the job's own stream while resident
    bool rhs_done = false;
    bool in_flight = false;       // a launched step has not been harvested
    bool step_in_launch = false;  // ... and it included a step (not the RHS alone)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the launched step
};

// Jobs below this many particles take the high-priority streams.
constexpr int kSmallJob = 131072;

// Scratch of the pair-once gravity kernel for jobs it applies to (0 if none).
size_t pairs_bytes(const SphParams &p, int n) {
    return pp_gravity_pairs_eligible(n, p.eps, 0) ? pp_gravity_pairs_workspace_bytes(n) : 0;
}

size_t state_bytes(int n, int ng, size_t grav_work) {
    size_t b = up256(grav_work);
    b += up256(3 * sizeof(double) * n) * 3;            // r, v, v_save
    b += up256(sizeof(double) * ng) * 2;               // e, e_save
    b += up256(sizeof(float) * n) + up256(sizeof(float) * ng);   // mass, h
    b += up256(16ull * n) * 2;                          // pos_m, grav
    b += up256(16ull * ng) * 3;                         // pos_h, vel_e, acc_hyd
    b += up256(sizeof(float) * ng);                     // rho
    return b;
}

void carve_state(Job &j, char *base, size_t grav_work) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *p = base + o;
        o += up256(bytes);
        return p;
    };
    const int n = j.n, ng = j.n_gas;
    j.st.n = n;
    j.st.n_gas = ng;
    j.st.r = (double *)take(3 * sizeof(double) * n);
    j.st.v = (double *)take(3 * sizeof(double) * n);
    j.st.v_save = (double *)take(3 * sizeof(double) * n);
    j.st.e = (double *)take(sizeof(double) * ng);
    j.st.e_save = (double *)take(sizeof(double) * ng);
    j.st.mass = (float *)take(sizeof(float) * n);
    j.st.h = (float *)take(sizeof(float) * ng);
    j.st.pos_m = (float *)take(16ull * n);
    j.st.grav = (float *)take(16ull * n);
    j.st.pos_h = (float *)take(16ull * ng);
    j.st.vel_e = (float *)take(16ull * ng);
    j.st.acc_hyd = (float *)take(16ull * ng);
    j.st.rho = (float *)take(sizeof(float) * ng);
    j.st.fresh = 0;
    j.st.grav_flags = 0;
    j.st.events = nullptr;
    j.st.grav_work = grav_work ? take(grav_work) : nullptr;
    j.st.grav_work_bytes = grav_work;
}

int log2_buckets(int ng) {
    int m = 10;
    while ((1ll << m) < 2ll * std::max(1, ng) && m < 30) ++m;
    return m;
}

}  // namespace

struct sph_server {
    SphParams params;
    char *arena_base = nullptr;
    Arena arena;
    int max_resident = 8;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;   // the resident job on each stream (1) or none (0)
    int n_high = 0;                 // streams [0, n_high) have the higher priority
    std::vector<float> step_ms_all; // latency of every step taken, in completion order
    int policy = SPH_SERVE_FIFO;    // order in which queued requests are admitted
    std::map<uint64_t, Job> jobs;
    std::deque<uint64_t> queue;
    std::vector<uint64_t> resident;
    uint64_t next_id = 1;
    std::mutex mu;
};

namespace {

// Give the job's memory back to the arena.  Kernels of the job may still be
// queued on its stream (the list build of size_lists, a step that failed on
// the host side after launching work), and the arena may hand the same bytes
// to another job on another stream at once, so the stream is drained first.
void free_device(sph_server *s, Job &j) {
    if (j.stream_slot >= 0 && (j.has_ws || j.has_state || j.in_flight))
        cudaStreamSynchronize(s->streams[j.stream_slot]);
    if (j.ev0) cudaEventDestroy(j.ev0);
    if (j.ev1) cudaEventDestroy(j.ev1);
    j.ev0 = j.ev1 = nullptr;
    j.in_flight = false;
    if (j.stream_slot >= 0) {
        s->stream_busy[j.stream_slot] = 0;
        j.stream_slot = -1;
    }
    if (j.ctx) {
        sph_ctx_destroy(j.ctx);
        j.ctx = nullptr;
    }
    if (j.has_ws) {
        s->arena.release(j.ws_off, j.ws_bytes);
        j.has_ws = false;
    }
    if (j.has_state) {
        s->arena.release(j.state_off, j.state_bytes);
        j.has_state = false;
    }
}

// (Re)create the job's context with room for `capacity` list entries.
int make_ctx(sph_server *s, Job &j, long long capacity, cudaStream_t st) {
    const int ng = std::max(1, j.n_gas);
    size_t need = sph_ctx_workspace_bytes(ng, j.log2_M, capacity);
    if (need == 0) return SPH_ERR_INVALID_ARG;
    size_t off = 0;
    if (!s->arena.alloc(need, &off)) return SPH_ERR_BUDGET;
    sph_ctx *c = nullptr;
    int rc = sph_ctx_create(&s->params, ng, j.log2_M, capacity, s->arena_base + off, need,
                            (sph_stream_t)st, &c);
    if (rc) {
        s->arena.release(off, need);
        return rc;
    }
    if (j.ctx) sph_ctx_destroy(j.ctx);
    if (j.has_ws) {
        // the old workspace may still be read by work queued on st
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            sph_ctx_destroy(c);
            s->arena.release(off, need);
            j.ctx = nullptr;
            return SPH_ERR_CUDA;
        }
        s->arena.release(j.ws_off, j.ws_bytes);
    }
    j.ctx = c;
    j.ws_off = off;
    j.ws_bytes = need;
    j.has_ws = true;
    j.capacity = capacity;
    return SPH_OK;
}

// Sort and count lists at the current working copies; grow the context until
// the lists fit with 30% headroom.
int size_lists(sph_server *s, Job &j, cudaStream_t st) {
    if (j.n_gas == 0) return SPH_OK;
    for (int tries = 0; tries < 8; ++tries) {
        int rc = sph_bin_and_sort(j.ctx, j.st.pos_h, j.n_gas, nullptr, nullptr, nullptr, nullptr,
                                  (sph_stream_t)st);
        if (rc) return rc;
        int64_t needed = 0;
        rc = sph_build_neighbors(j.ctx, j.n_gas, nullptr, nullptr, 0, &needed, (sph_stream_t)st);
        if (rc && rc != SPH_ERR_NB_OVERFLOW) return rc;
        if (rc == SPH_OK && needed <= 0.7 * (double)j.capacity) return SPH_OK;
        if ((rc = make_ctx(s, j, (long long)(needed * 1.6) + 1024, st))) return rc;
    }
    return SPH_ERR_NB_OVERFLOW;
}

// Admit job j: state + context out of the arena, upload the IC, size lists.
int admit(sph_server *s, Job &j, cudaStream_t st) {
    const size_t gw = pairs_bytes(s->params, j.n);
    j.state_bytes = state_bytes(j.n, j.n_gas, gw);
    if (!s->arena.alloc(j.state_bytes, &j.state_off)) return SPH_ERR_BUDGET;
    j.has_state = true;
    carve_state(j, s->arena_base + j.state_off, gw);
    j.log2_M = log2_buckets(j.n_gas);
    int rc = make_ctx(s, j, std::max<long long>(1024, (long long)j.n_gas * 120), st);
    if (rc) {
        free_device(s, j);
        return rc;
    }
    const size_t n = j.n, ng = j.n_gas;
    SPH_CUDA_TRY(cudaMemcpyAsync(j.st.r, j.r.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    SPH_CUDA_TRY(cudaMemcpyAsync(j.st.v, j.v.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    SPH_CUDA_TRY(cudaMemcpyAsync(j.st.mass, j.m.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
    if (ng) {
        SPH_CUDA_TRY(cudaMemcpyAsync(j.st.e, j.e.data(), ng * sizeof(double), cudaMemcpyHostToDevice, st));
        SPH_CUDA_TRY(cudaMemcpyAsync(j.st.h, j.h.data(), ng * sizeof(float), cudaMemcpyHostToDevice, st));
    }
    rc = integrate_step(SPH_EMIT, 0.0, j.n, j.n_gas, j.st.r, j.st.v, j.st.e, nullptr, nullptr, nullptr,
                        nullptr, j.st.mass, j.st.h, j.st.pos_m, j.st.pos_h, j.st.vel_e,
                        (sph_stream_t)st);
    if (rc == SPH_OK) rc = size_lists(s, j, st);
    if (rc) {
        free_device(s, j);
        return rc;
    }
    if (cudaEventCreate(&j.ev0) != cudaSuccess || cudaEventCreate(&j.ev1) != cudaSuccess) {
        free_device(s, j);
        return SPH_ERR_CUDA;
    }
    j.state = JOB_RUNNING;
    j.t_admit = now_s();
    return SPH_OK;
}

// A free stream for a job of n particles: a high-priority one for small jobs
// (normal if none is free), a normal one for the others (high if none is).
int pick_stream(sph_server *s, int n) {
    const int ns = (int)s->streams.size();
    const bool small = n < kSmallJob;
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < ns; ++k) {
            const bool high = k < s->n_high;
            if (!s->stream_busy[k] && (pass == 1 || high == small)) return k;
        }
    return -1;
}

// Estimated seconds of GPU work a request still needs: its steps times the
// cost of one (direct gravity ~ N^2 at ~3.9e12 pair terms per second, the SPH
// stages ~ 4 ns per particle, ~0.5 ms of launches per step).
double work_left(const Job &j) {
    const double n = (double)j.n;
    return (double)(j.n_steps - j.steps_done + 1) * (n * n / 3.9e12 + n * 4e-9 + 5e-4);
}

void admit_queued(sph_server *s) {
    if (s->policy == SPH_SERVE_SHORTEST_FIRST)
        std::stable_sort(s->queue.begin(), s->queue.end(), [&](uint64_t a, uint64_t b) {
            return work_left(s->jobs[a]) < work_left(s->jobs[b]);
        });
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)s->resident.size() < s->max_resident;) {
        Job &j = s->jobs[*it];
        const int slot = pick_stream(s, j.n);
        if (slot < 0) break;   // every stream holds a resident job
        j.stream_slot = slot;
        s->stream_busy[slot] = 1;
        int rc = admit(s, j, s->streams[slot]);
        if (rc == SPH_OK) {
            s->resident.push_back(j.id);
            it = s->queue.erase(it);
        } else {
            free_device(s, j);   // whatever the failed admission holds, its stream included
            if (rc == SPH_ERR_BUDGET && !s->resident.empty()) {
                ++it;   // does not fit now; smaller ones behind it may
            } else {    // failed, or does not fit even into an empty arena
                j.state = JOB_FAILED;
                j.error = rc;
                it = s->queue.erase(it);
            }
        }
    }
}

}  // namespace

extern "C" int sph_server_create(const SphParams *params, void *d_arena, size_t arena_bytes,
                                 int32_t max_resident, int32_t n_streams, sph_server **out) {
    if (!params || !out || !d_arena || (reinterpret_cast<uintptr_t>(d_arena) & 255u) ||
        arena_bytes < 4096 || max_resident < 1 || n_streams < 1 || n_streams > 64)
        return SPH_ERR_INVALID_ARG;
    sph_server *s = new (std::nothrow) sph_server;
    if (!s) return SPH_ERR_INVALID_ARG;
    s->params = *params;
    s->arena_base = static_cast<char *>(d_arena);
    s->arena.init(arena_bytes);
    s->max_resident = max_resident;
    int lo = 0, hi = 0;   // numerically lower is the higher priority
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
        delete s;
        return SPH_ERR_CUDA;
    }
    const int ns = std::max(n_streams, max_resident);
    s->n_high = ns >= 2 ? ns / 2 : 0;
    for (int i = 0; i < ns; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, i < s->n_high ? hi : lo) !=
            cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            delete s;
            return SPH_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    s->stream_busy.assign(ns, 0);
    *out = s;
    return SPH_OK;
}

extern "C" int sph_server_destroy(sph_server *s) {
    if (!s) return SPH_ERR_INVALID_ARG;
    for (auto st : s->streams) cudaStreamSynchronize(st);
    for (auto &kv : s->jobs) free_device(s, kv.second);
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
    return SPH_OK;
}

extern "C" int sim_submit(sph_server *s, const SimRequest *req, uint64_t *job_id) {
    if (!s || !req || !job_id || req->n < 1 || req->n_gas < 0 || req->n_gas > req->n ||
        req->n_steps < 0 || !(req->dt == req->dt) || !req->h_r || !req->h_v || !req->h_m ||
        (req->n_gas > 0 && (!req->h_e || !req->h_h)))
        return SPH_ERR_INVALID_ARG;
    // a request that can never fit the budget is refused at once
    const size_t est = state_bytes(req->n, req->n_gas, pairs_bytes(s->params, req->n)) +
                       sph_ctx_workspace_bytes(std::max(1, req->n_gas), log2_buckets(req->n_gas),
                                               std::max<long long>(1024, (long long)req->n_gas * 120));
    std::lock_guard<std::mutex> lock(s->mu);
    if (est > s->arena.size) return SPH_ERR_BUDGET;
    Job j;
    j.id = s->next_id++;
    j.n = req->n;
    j.n_gas = req->n_gas;
    j.n_steps = req->n_steps;
    j.dt = req->dt;
    j.r.assign(req->h_r, req->h_r + 3 * (size_t)req->n);
    j.v.assign(req->h_v, req->h_v + 3 * (size_t)req->n);
    j.m.assign(req->h_m, req->h_m + req->n);
    if (req->n_gas) {
        j.e.assign(req->h_e, req->h_e + req->n_gas);
        j.h.assign(req->h_h, req->h_h + req->n_gas);
    }
    j.t_submit = now_s();
    *job_id = j.id;
    s->queue.push_back(j.id);
    s->jobs.emplace(j.id, std::move(j));
    return SPH_OK;
}

namespace {

// Launch the next step of resident job j on its stream (the initial RHS
// first, on its first launch), between its two events.
void launch_step(sph_server *s, Job &j) {
    cudaStream_t st = s->streams[j.stream_slot];
    int rc = SPH_OK;
    if (cudaEventRecord(j.ev0, st) != cudaSuccess) rc = SPH_ERR_CUDA;
    if (rc == SPH_OK && !j.rhs_done) {
        rc = sph_rhs_initial(j.ctx, &j.st, (sph_stream_t)st);
        j.rhs_done = true;
    }
    j.step_in_launch = rc == SPH_OK && j.steps_done < j.n_steps;
    if (j.step_in_launch) rc = sph_step(j.ctx, &j.st, j.dt, (sph_stream_t)st);
    if (rc == SPH_OK && cudaEventRecord(j.ev1, st) != cudaSuccess) rc = SPH_ERR_CUDA;
    if (rc) {
        j.state = JOB_FAILED;
        j.error = rc;
        return;
    }
    j.in_flight = true;
}

// Job j's launched step has finished: count it, check its device status and
// list capacity (growing the context between steps), and copy the final
// state back when the job is done.
void harvest(sph_server *s, Job &j) {
    cudaStream_t st = s->streams[j.stream_slot];
    j.in_flight = false;
    if (j.step_in_launch) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, j.ev0, j.ev1);
        j.steps_done += 1;
        j.step_ms.push_back(ms);
        s->step_ms_all.push_back(ms);
    }
    if (j.state == JOB_RUNNING && j.n_gas > 0) {
        int32_t flags = 0;
        int rc = sph_ctx_device_status(j.ctx, (sph_stream_t)st, &flags);
        if (flags & SPH_FLAG_NB_OVERFLOW) {
            j.state = JOB_FAILED;
            j.error = SPH_ERR_NB_OVERFLOW;
        } else if (rc != SPH_OK && rc != SPH_ERR_DEVICE) {
            j.state = JOB_FAILED;
            j.error = rc;
        } else if (j.steps_done < j.n_steps) {
            int64_t used = 0;
            if (sph_ctx_nb_total(j.ctx, (sph_stream_t)st, &used) == SPH_OK &&
                used > 0.7 * (double)j.capacity) {
                // grow between steps: re-sort the same working copies into
                // a larger context (the lists are a function of pos_h)
                int rc2 = make_ctx(s, j, (long long)(used * 1.6) + 1024, st);
                if (rc2 == SPH_OK) rc2 = size_lists(s, j, st);
                if (rc2 != SPH_OK) {
                    j.state = JOB_FAILED;
                    j.error = rc2;
                }
            }
        }
    }
    if (j.state == JOB_RUNNING && j.steps_done >= j.n_steps) {
        const size_t n = j.n, ng = j.n_gas;
        bool ok = cudaMemcpyAsync(j.r.data(), j.st.r, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaMemcpyAsync(j.v.data(), j.st.v, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  (ng == 0 || cudaMemcpyAsync(j.e.data(), j.st.e, ng * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess) &&
                  cudaStreamSynchronize(st) == cudaSuccess;
        j.state = ok ? JOB_DONE : JOB_FAILED;
        if (!ok) j.error = SPH_ERR_CUDA;
        j.t_done = now_s();
    }
}

}  // namespace

extern "C" int sph_server_step(sph_server *s, int32_t *h_resident, double *h_step_ms) {
    if (!s) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    const double t0 = now_s();
    admit_queued(s);
    bool progressed = false;
    for (int pass = 0; pass < 2; ++pass) {
        // harvest the steps that have finished
        for (uint64_t id : s->resident) {
            Job &j = s->jobs[id];
            if (!j.in_flight) continue;
            const cudaError_t q = cudaEventQuery(j.ev1);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                j.state = JOB_FAILED;
                j.error = SPH_ERR_CUDA;
                j.in_flight = false;
                continue;
            }
            harvest(s, j);
            progressed = true;
        }
        // retire the jobs that finished or failed, then launch the next step
        // of every idle resident job
        std::vector<uint64_t> still;
        for (uint64_t id : s->resident) {
            Job &j = s->jobs[id];
            if (j.state == JOB_RUNNING) still.push_back(id);
            else free_device(s, j);
        }
        s->resident.swap(still);
        for (uint64_t id : s->resident) {
            Job &j = s->jobs[id];
            if (!j.in_flight) launch_step(s, j);
        }
        bool any = false;
        for (uint64_t id : s->resident) any |= s->jobs[id].in_flight;
        if (progressed || !any) break;
        // nothing finished yet: wait for the first step that does (bounded)
        const double tw = now_s();
        bool done = false;
        while (!done) {
            for (uint64_t id : s->resident) {
                const Job &j = s->jobs[id];
                if (j.in_flight && cudaEventQuery(j.ev1) != cudaErrorNotReady) done = true;
            }
            if (!done) {
                if (now_s() - tw > 3600.0) return SPH_ERR_TIMEOUT;
                std::this_thread::sleep_for(std::chrono::microseconds(50));
            }
        }
    }
    // memory and slots freed by retired jobs take queued requests at once
    admit_queued(s);
    for (uint64_t id : s->resident) {
        Job &j = s->jobs[id];
        if (!j.in_flight && j.state == JOB_RUNNING) launch_step(s, j);
    }
    if (h_resident) *h_resident = (int32_t)s->resident.size();
    if (h_step_ms) *h_step_ms = (now_s() - t0) * 1e3;
    return SPH_OK;
}

extern "C" int sph_server_set_policy(sph_server *s, int32_t policy) {
    if (!s || (policy != SPH_SERVE_FIFO && policy != SPH_SERVE_SHORTEST_FIRST))
        return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->policy = policy;
    return SPH_OK;
}

extern "C" int sph_server_step_times(sph_server *s, float *h_ms, int32_t cap, int32_t *h_count) {
    if (!s || !h_count || cap < 0 || (cap > 0 && !h_ms)) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    const int32_t n = (int32_t)s->step_ms_all.size();
    *h_count = n;
    if (cap > 0 && n > 0)
        std::memcpy(h_ms, s->step_ms_all.data(), sizeof(float) * (size_t)std::min(n, cap));
    return SPH_OK;
}

extern "C" int sim_poll(sph_server *s, uint64_t job_id, SimStatus *out) {
    if (!s || !out) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return SPH_ERR_NOT_FOUND;
    const Job &j = it->second;
    std::memset(out, 0, sizeof(*out));
    out->state = j.state;
    out->error = j.error;
    out->n = j.n;
    out->n_gas = j.n_gas;
    out->n_steps = j.n_steps;
    out->steps_done = j.steps_done;
    out->submit_s = j.t_submit;
    out->admit_s = j.t_admit;
    out->done_s = j.t_done;
    if (!j.step_ms.empty()) {
        std::vector<float> v = j.step_ms;
        std::sort(v.begin(), v.end());
        out->step_ms_p50 = v[(v.size() - 1) / 2];
        out->step_ms_p99 = v[std::min(v.size() - 1, (size_t)(0.99 * (v.size() - 1) + 0.5))];
    }
    if (j.state == JOB_DONE) {
        out->h_r = j.r.data();
        out->h_v = j.v.data();
        out->h_e = j.n_gas ? j.e.data() : nullptr;
    }
    return SPH_OK;
}

extern "C" int sim_checkpoint(sph_server *s, uint64_t job_id, double *h_r, double *h_v, double *h_e,
                              float *h_h, int32_t *h_steps_done) {
    if (!s || !h_r || !h_v || !h_steps_done) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return SPH_ERR_NOT_FOUND;
    Job &j = it->second;
    if (j.n_gas > 0 && (!h_e || !h_h)) return SPH_ERR_INVALID_ARG;
    if (j.state != JOB_RUNNING || !j.rhs_done) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = s->streams[j.stream_slot];
    if (j.in_flight) {
        // let the launched step finish and count it, as a server step would
        SPH_CUDA_TRY(cudaEventSynchronize(j.ev1));
        harvest(s, j);
        if (j.state == JOB_DONE) {   // that was its last step: the final state
            std::memcpy(h_r, j.r.data(), sizeof(double) * 3 * (size_t)j.n);
            std::memcpy(h_v, j.v.data(), sizeof(double) * 3 * (size_t)j.n);
            if (j.n_gas) std::memcpy(h_e, j.e.data(), sizeof(double) * (size_t)j.n_gas);
        }
        if (j.state == JOB_FAILED) return j.error ? j.error : SPH_ERR_CUDA;
    }
    const size_t n = j.n, ng = j.n_gas;
    if (j.state == JOB_RUNNING) {
        SPH_CUDA_TRY(cudaMemcpyAsync(h_r, j.st.r, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
        SPH_CUDA_TRY(cudaMemcpyAsync(h_v, j.st.v, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (ng) SPH_CUDA_TRY(cudaMemcpyAsync(h_e, j.st.e, ng * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (ng) {
        // the smoothing length of the last evaluation: the h of the FP32
        // working copy (x, y, z, h) its sort and density read
        std::vector<float> ph(4 * ng);
        SPH_CUDA_TRY(cudaMemcpyAsync(ph.data(), j.st.pos_h, 16 * ng, cudaMemcpyDeviceToHost, st));
        SPH_CUDA_TRY(cudaStreamSynchronize(st));
        for (size_t q = 0; q < ng; ++q) h_h[q] = ph[4 * q + 3];
    }
    SPH_CUDA_TRY(cudaStreamSynchronize(st));
    *h_steps_done = j.steps_done;
    return SPH_OK;
}

extern "C" int sim_release(sph_server *s, uint64_t job_id) {
    if (!s) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return SPH_ERR_NOT_FOUND;
    if (it->second.state == JOB_RUNNING) return SPH_ERR_INVALID_ARG;
    if (it->second.state == JOB_QUEUED) {
        auto q = std::find(s->queue.begin(), s->queue.end(), job_id);
        if (q != s->queue.end()) s->queue.erase(q);
    }
    free_device(s, it->second);
    s->jobs.erase(it);
    return SPH_OK;
}

extern "C" int sph_server_info(sph_server *s, SphServerInfo *out) {
    if (!s || !out) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    out->queued = (int32_t)s->queue.size();
    out->resident = (int32_t)s->resident.size();
    out->arena_bytes = s->arena.size;
    out->arena_free_bytes = s->arena.free_bytes();
    return SPH_OK;
}
