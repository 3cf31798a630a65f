// Serving: continuous batching of independent simulations on one GPU.
//
// Requests (lattice size, probabilities, seed, MCS count, observation times) are queued by any
// host thread.  One scheduler thread admits them in arrival order whenever a slot (a stream,
// an event and a pinned result buffer) is free and the device-memory budget still holds their
// state; admitted requests get stream-ordered memory from a pool, so admission never
// synchronises the device.  Every active request keeps at most one piece of work in flight on
// its own stream, so pieces of different requests overlap on the GPU, and a request that
// arrives while others run starts as soon as a slot and memory free up.  Short requests run on
// a high-priority stream, so their blocks go first when the GPU is shared.  Steps run as a
// captured CUDA graph of kChunk MCS, replayed with a device-resident MCS counter (the update
// kernels read t from it), so the host issues one graph launch per kChunk MCS instead of one
// or two kernel launches per MCS.  Each request's dynamics are exactly those of a single
// simulation with the same parameters (same kernels, same Philox counters), so its results do
// not depend on what else is running.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "sca.h"
#include "sca_internal.h"

namespace sca {

constexpr uint32_t kChunk = 64;        // MCS per replayed graph (even: fused buffers return)
constexpr uint32_t kChunksPerPiece = 4;
// Requests of at most this many site updates (L^2 x MCS; about 8 ms of GPU work) run on their
// slot's high-priority stream: when SM slots free up, the GPU's block scheduler starts their
// blocks before those of larger requests, so short requests are not held behind long ones
// (shortest-first on the device; admission stays in arrival order).
constexpr uint64_t kShortWork = 1ull << 33;

static uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServeReq {
    uint64_t ticket = 0;
    sca_params P{};
    uint64_t n_mcs = 0;
    std::vector<uint64_t> times;        // observation times, increasing, last == n_mcs
    int status = SCA_EBUSY;             // SCA_EBUSY until finished
    int phase = 0;                      // 0 pending, 1 active, 2 finished
    bool cancel = false;
    uint64_t t_submit = 0, t_admit = 0, t_done = 0;
    size_t need = 0;
    int slot = -1;
    std::vector<sca_obs> obs;
    uint32_t *final_words = nullptr;    // caller-owned host buffer for the final state (or null)
    // scheduler-owned while active
    cudaStream_t st = nullptr;          // the slot's stream this request runs on
    void *mem = nullptr;
    sca_sim *sim = nullptr;
    uint64_t *t_dev = nullptr;
    uint32_t next_obs = 0;
    bool inflight = false, copying = false, t_dev_synced = false;
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};   // per state-buffer parity
    int chunk_cur[2] = {-1, -1};
};

struct Slot {
    cudaStream_t stream = nullptr;      // default priority
    cudaStream_t stream_hi = nullptr;   // highest priority (short requests)
    cudaEvent_t ev = nullptr;
    sca_obs *pinned = nullptr;          // kResCap records
    bool busy = false;
};

}  // namespace sca

using namespace sca;

struct sca_server {
    size_t budget = 0, used = 0;
    uint32_t max_active = 0, max_L = 0;
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<Slot> slots;
    std::deque<ServeReq *> pending;
    std::map<uint64_t, ServeReq *> reqs;
    std::vector<ServeReq *> active;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t t0 = 0;
    sca_server_stats st{};
};

namespace sca {

static double secs(const sca_server *s, uint64_t t) { return t ? (double)(t - s->t0) * 1e-9 : 0.0; }

static void fill_info(const sca_server *s, const ServeReq *r, sca_request_info *info)
{
    if (!info) return;
    info->ticket = r->ticket;
    info->n_mcs = r->n_mcs;
    info->n_obs = (uint32_t)r->times.size();
    info->status = r->status;
    info->L = r->P.L;
    info->submit_s = secs(s, r->t_submit);
    info->admit_s = secs(s, r->t_admit);
    info->done_s = secs(s, r->t_done);
}

// Capture kChunk MCS of this request's update kernels, relative to its device counter, for the
// state-buffer parity the simulation has now.
static cudaError_t capture_chunk(ServeReq *r, cudaStream_t st)
{
    sca_sim *s = r->sim;
    const int par = s->cur;
    if (r->chunk[par]) return cudaSuccess;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    int tbk = 0;
    const int kern = effective_kernel(s, &tbk);
    const bool fused = kern == 2;
    int cur = s->cur;
    cudaError_t le = cudaSuccess;
    const bool tb = kern == 3 || kern == 4;
    if (tb) {                                  // temporal blocking: kChunk / tbk launches
        for (uint32_t i = 0; i < kChunk && le == cudaSuccess; i += (uint32_t)tbk) {
            le = kern == 3 ? launch_tblock(s->buf[cur], s->buf[cur ^ 1], s->L, i, (uint32_t)tbk, s->R,
                                           st, r->t_dev)
                           : launch_wave(s->buf[cur], s->buf[cur ^ 1], s->L, i, (uint32_t)tbk, s->R,
                                         st, r->t_dev, s->wave_bands);
            cur ^= 1;
        }
    }
    for (uint32_t i = 0; !tb && i < kChunk && le == cudaSuccess; ++i) {
        if (fused) {
            le = launch_fused_mcs(s->buf[cur], s->buf[cur ^ 1], s->L, i, s->R, s->err, st, r->t_dev,
                                  s->fused_V, s->fused_ring);
            cur ^= 1;
        } else {
            le = launch_half_step(s->buf[cur], s->L, i, 0, s->R, st, r->t_dev);
            if (le == cudaSuccess) le = launch_half_step(s->buf[cur], s->L, i, 1, s->R, st, r->t_dev);
        }
    }
    if (le == cudaSuccess) le = launch_add_t(r->t_dev, kChunk, st);
    e = cudaStreamEndCapture(st, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&r->chunk[par], g, 0);
    cudaGraphDestroy(g);
    return e;
}

static void release_gpu(sca_server *srv, ServeReq *r)
{
    Slot &sl = srv->slots[r->slot];
    if (r->sim) {
        sca_free(r->sim);            // synchronises the request's stream; memory is the pool's
        r->sim = nullptr;
    }
    for (int p = 0; p < 2; ++p)
        if (r->chunk[p]) {
            cudaGraphExecDestroy(r->chunk[p]);
            r->chunk[p] = nullptr;
        }
    if (r->mem) {
        cudaFreeAsync(r->mem, r->st);
        r->mem = nullptr;
    }
}

// Called by the scheduler with the lock NOT held.
static void finish(sca_server *srv, ServeReq *r, int status)
{
    Slot &sl = srv->slots[r->slot];
    if (status == SCA_OK) {
        const size_t n = r->times.size();
        r->obs.assign(sl.pinned, sl.pinned + n);
        for (auto &o : r->obs) {
            const double num = std::ldexp((double)o.num_hi, 64) + (double)o.num_lo;
            o.w2 = num / ((double)o.N * (double)o.N);
            if (o.status && status == SCA_OK) status = o.status;
        }
    }
    release_gpu(srv, r);
    std::lock_guard<std::mutex> lk(srv->mu);
    r->status = status;
    r->phase = 2;
    r->t_done = now_ns();
    sl.busy = false;
    srv->used -= r->need;
    if (status == SCA_OK) {
        srv->st.completed++;
        srv->st.updates_done += (uint64_t)r->P.L * r->P.L * r->n_mcs;
    } else if (status == SCA_ECANCELED) {
        srv->st.cancelled++;
    } else {
        srv->st.failed++;
    }
    srv->cv_done.notify_all();
}

static int start(sca_server *srv, ServeReq *r)
{
    Slot &sl = srv->slots[r->slot];
    r->st = (uint64_t)r->P.L * r->P.L * r->n_mcs <= kShortWork ? sl.stream_hi : sl.stream;
    cudaError_t e = cudaMallocFromPoolAsync(&r->mem, r->need + 256, srv->pool, r->st);
    if (e != cudaSuccess) return fail(SCA_ENOMEM, "pool allocation");
    const size_t ws = sca_workspace_bytes(r->P.L);
    r->t_dev = reinterpret_cast<uint64_t *>(static_cast<char *>(r->mem) + ((ws + 255) & ~(size_t)255));
    int rc = sca_init(&r->P, r->st, r->mem, ws, &r->sim);
    if (rc) return rc;
    // Requests share the GPU, so a request takes the kernel with the most throughput per SM,
    // not the one that finishes a lattice alone soonest: per-site uniforms run the two-pass
    // kernel at every size.  Temporal blocking plans one large-shared-memory CTA per SM even
    // for a small lattice, so its launches cannot share the SMs with other requests' work, and
    // its recomputed halos repeat Philox calls.
    if (r->sim->R.mode == 2) {
        rc = sca_set_kernel(r->sim, 1);
        if (rc) return rc;
    }
    return SCA_OK;
}

// Enqueue the next piece of a request's work; returns false when nothing more is needed.
static int enqueue_piece(sca_server *srv, ServeReq *r)
{
    Slot &sl = srv->slots[r->slot];
    sca_sim *s = r->sim;
    const uint32_t n = (uint32_t)r->times.size();
    while (r->next_obs < n && r->times[r->next_obs] == s->t) {
        cudaError_t e = launch_observe(s->buf[s->cur], s->L, s->h0, s->part, s->res + r->next_obs,
                                       s->t, r->st);
        if (e != cudaSuccess) return cuda_fail(e, "observe launch");
        r->next_obs++;
    }
    if (r->next_obs == n) {
        cudaError_t e = cudaMemcpyAsync(sl.pinned, s->res, n * sizeof(sca_obs), cudaMemcpyDeviceToHost, r->st);
        if (e != cudaSuccess) return cuda_fail(e, "result copy");
        if (r->final_words) {
            e = cudaMemcpyAsync(r->final_words, s->buf[s->cur], s->lo.state_bytes, cudaMemcpyDeviceToHost,
                                r->st);
            if (e != cudaSuccess) return cuda_fail(e, "final state copy");
        }
        r->copying = true;
    } else {
        const uint64_t gap = r->times[r->next_obs] - s->t;
        if (gap >= kChunk) {
            cudaError_t e = capture_chunk(r, r->st);
            if (e != cudaSuccess) return cuda_fail(e, "step graph");
            if (!r->t_dev_synced) {
                e = launch_set_t(r->t_dev, s->t, r->st);
                if (e != cudaSuccess) return cuda_fail(e, "counter");
                r->t_dev_synced = true;
            }
            uint64_t k = gap / kChunk;
            if (k > kChunksPerPiece) k = kChunksPerPiece;
            for (uint64_t c = 0; c < k; ++c) {
                e = cudaGraphLaunch(r->chunk[s->cur], r->st);
                if (e != cudaSuccess) return cuda_fail(e, "graph launch");
                {
                    int tk = 0;
                    const int kk = effective_kernel(s, &tk);
                    count_launches((kk >= 3 ? kChunk / (uint32_t)tk : kChunk * (kk == 2 ? 1 : 2)) + 1);
                }
            }
            s->t += k * kChunk;
            {
                // each graph replay swaps the state buffers once per launch that writes the
                // other buffer: kChunk times (fused) or kChunk / tbk times (temporal blocking)
                int tk = 0;
                const int kk = effective_kernel(s, &tk);
                const uint32_t swaps = kk == 2 ? kChunk : kk >= 3 ? kChunk / (uint32_t)tk : 0u;
                if (swaps & 1u) s->cur ^= (int)(k & 1u);
            }
        } else {
            int rc = step_impl(s, gap);
            if (rc) return rc;
            r->t_dev_synced = false;
        }
    }
    cudaError_t e = cudaEventRecord(sl.ev, r->st);
    if (e != cudaSuccess) return cuda_fail(e, "event");
    r->inflight = true;
    return SCA_OK;
}

static void scheduler(sca_server *srv)
{
    cudaSetDevice(srv->device);
    std::vector<ServeReq *> admitted;
    for (;;) {
        admitted.clear();
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->stop) break;
            while (!srv->pending.empty()) {
                ServeReq *r = srv->pending.front();
                if (r->cancel) {
                    srv->pending.pop_front();
                    r->status = SCA_ECANCELED;
                    r->phase = 2;
                    r->t_done = now_ns();
                    srv->st.cancelled++;
                    srv->cv_done.notify_all();
                    continue;
                }
                if (srv->used + r->need > srv->budget) break;     // wait for memory
                int free_slot = -1;
                for (uint32_t i = 0; i < srv->slots.size(); ++i)
                    if (!srv->slots[i].busy) { free_slot = (int)i; break; }
                if (free_slot < 0) break;                            // wait for a slot
                srv->pending.pop_front();
                srv->slots[free_slot].busy = true;
                r->slot = free_slot;
                r->phase = 1;
                r->t_admit = now_ns();
                srv->used += r->need;
                srv->st.admitted++;
                admitted.push_back(r);
            }
        }
        for (ServeReq *r : admitted) {
            int rc = start(srv, r);
            if (rc) finish(srv, r, rc);
            else srv->active.push_back(r);
        }
        bool progress = !admitted.empty();
        for (size_t i = 0; i < srv->active.size();) {
            ServeReq *r = srv->active[i];
            Slot &sl = srv->slots[r->slot];
            bool done = false;
            int status = SCA_OK;
            if (r->inflight) {
                cudaError_t q = cudaEventQuery(sl.ev);
                if (q == cudaErrorNotReady) { ++i; continue; }
                r->inflight = false;
                progress = true;
                if (q != cudaSuccess) { done = true; status = cuda_fail(q, "request work"); }
                else if (r->copying) done = true;
            }
            if (!done && r->cancel) { done = true; status = SCA_ECANCELED; }
            if (!done) {
                int rc = enqueue_piece(srv, r);
                if (rc) { done = true; status = rc; }
                progress = true;
            }
            if (done) {
                finish(srv, r, status);
                srv->active[i] = srv->active.back();
                srv->active.pop_back();
            } else {
                ++i;
            }
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
    // shutdown: cancel everything still running
    for (ServeReq *r : srv->active) finish(srv, r, SCA_ECANCELED);
    srv->active.clear();
}

}  // namespace sca

extern "C" {

int sca_server_create(size_t budget_bytes, uint32_t max_active, uint32_t max_L, sca_server **out)
{
    if (!out || max_active == 0 || sca_workspace_bytes(max_L) == 0)
        return fail(SCA_EINVAL, "bad server parameters");
    *out = nullptr;
    sca_server *srv = new sca_server();
    srv->budget = budget_bytes;
    srv->max_active = max_active;
    srv->max_L = max_L;
    srv->t0 = now_ns();
    srv->st.budget_bytes = budget_bytes;
    cudaError_t e = cudaGetDevice(&srv->device);
    if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&srv->pool, srv->device);
    if (e == cudaSuccess) {
        uint64_t thr = budget_bytes;     // keep freed state memory in the pool up to the budget
        e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    int prio_least = 0, prio_greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    srv->slots.resize(max_active);
    for (uint32_t i = 0; i < max_active && e == cudaSuccess; ++i) {
        Slot &sl = srv->slots[i];
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, prio_greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.pinned, kResCap * sizeof(sca_obs));
    }
    if (e != cudaSuccess) {
        sca_server_destroy(srv);
        return cuda_fail(e, "sca_server_create");
    }
    srv->worker = std::thread(scheduler, srv);
    *out = srv;
    return SCA_OK;
}

static int submit_impl(sca_server *srv, const sca_params *params, uint64_t n_mcs, const uint64_t *times,
                       uint32_t n_times, uint32_t *final_words, size_t n_words, uint64_t *ticket)
{
    if (!srv || !params || !ticket || n_mcs == 0) return fail(SCA_EINVAL, "NULL argument or zero MCS");
    if (final_words && n_words < 4 * (size_t)params->L * (params->L / 64))
        return fail(SCA_EINVAL, "final-state buffer shorter than 4 * L * L/64 words");
    if (params->L > srv->max_L) return fail(SCA_EINVAL, "L exceeds the server's maximum");
    if (params->Ly != 0 && params->Ly != params->L)
        return fail(SCA_EINVAL, "served lattices are square (Ly = 0 or L)");
    if (params->dynamics != SCA_DYN_SCA) return fail(SCA_EINVAL, "served lattices run the SCA dynamics");
    const size_t need = sca_workspace_bytes(params->L);
    if (need == 0) return fail(SCA_EINVAL, "L must be a multiple of 64 in [64, 131072]");
    if (need + 256 > srv->budget) return fail(SCA_EBUDGET, "request state exceeds the device budget");
    Rule R;
    int rc = make_rule(*params, R);
    if (rc) return rc;
    ServeReq *r = new ServeReq();
    r->P = *params;
    r->n_mcs = n_mcs;
    r->final_words = final_words;
    if (times && n_times) {
        if (n_times > (uint32_t)kResCap) { delete r; return fail(SCA_EINVAL, "at most 64 observation times"); }
        uint64_t prev = 0;
        for (uint32_t i = 0; i < n_times; ++i) {
            if (times[i] <= prev || times[i] > n_mcs) {
                delete r;
                return fail(SCA_EINVAL, "times must increase within 1..n_mcs");
            }
            prev = times[i];
        }
        r->times.assign(times, times + n_times);
        if (r->times.back() != n_mcs) {
            if (r->times.size() == (size_t)kResCap) { delete r; return fail(SCA_EINVAL, "too many times"); }
            r->times.push_back(n_mcs);
        }
    } else {
        for (uint64_t t = 1; t < n_mcs; t *= 2) r->times.push_back(t);
        r->times.push_back(n_mcs);
        if (r->times.size() > (size_t)kResCap) { delete r; return fail(SCA_EINVAL, "too many times"); }
    }
    r->need = need + 256;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        r->ticket = srv->next_ticket++;
        r->t_submit = now_ns();
        srv->reqs[r->ticket] = r;
        srv->pending.push_back(r);
        srv->st.submitted++;
        *ticket = r->ticket;
    }
    srv->cv_work.notify_one();
    return SCA_OK;
}

int sca_server_submit(sca_server *srv, const sca_params *params, uint64_t n_mcs,
                      const uint64_t *times, uint32_t n_times, uint64_t *ticket)
{
    return submit_impl(srv, params, n_mcs, times, n_times, nullptr, 0, ticket);
}

int sca_server_submit_state(sca_server *srv, const sca_params *params, uint64_t n_mcs,
                            const uint64_t *times, uint32_t n_times, uint32_t *final_words,
                            size_t n_words, uint64_t *ticket)
{
    if (!final_words) return fail(SCA_EINVAL, "NULL final-state buffer");
    return submit_impl(srv, params, n_mcs, times, n_times, final_words, n_words, ticket);
}

static int collect(sca_server *srv, ServeReq *r, sca_obs *out, uint32_t n_out, sca_request_info *info)
{
    fill_info(srv, r, info);
    if (r->phase != 2) return SCA_EBUSY;
    if (out && r->status == SCA_OK) {
        const uint32_t n = (uint32_t)r->obs.size() < n_out ? (uint32_t)r->obs.size() : n_out;
        std::memcpy(out, r->obs.data(), n * sizeof(sca_obs));
    }
    return r->status;
}

int sca_server_poll(sca_server *srv, uint64_t ticket, sca_obs *out, uint32_t n_out,
                    sca_request_info *info)
{
    if (!srv) return fail(SCA_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(SCA_ENOTFOUND, "unknown ticket");
    return collect(srv, it->second, out, n_out, info);
}

int sca_server_wait(sca_server *srv, uint64_t ticket, int timeout_ms, sca_obs *out, uint32_t n_out,
                    sca_request_info *info)
{
    if (!srv) return fail(SCA_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(SCA_ENOTFOUND, "unknown ticket");
    ServeReq *r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (r->phase != 2) {
        if (timeout_ms < 0) srv->cv_done.wait(lk);
        else if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->phase != 2) {
            fill_info(srv, r, info);
            return fail(SCA_ETIMEOUT, "request not finished before the timeout");
        }
    }
    return collect(srv, r, out, n_out, info);
}

int sca_server_cancel(sca_server *srv, uint64_t ticket)
{
    if (!srv) return fail(SCA_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return fail(SCA_ENOTFOUND, "unknown ticket");
        if (it->second->phase == 2) return SCA_OK;
        it->second->cancel = true;
    }
    srv->cv_work.notify_one();
    return SCA_OK;
}

int sca_server_release(sca_server *srv, uint64_t ticket)
{
    if (!srv) return fail(SCA_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(SCA_ENOTFOUND, "unknown ticket");
    if (it->second->phase != 2) return fail(SCA_EBUSY, "request still pending or running");
    delete it->second;
    srv->reqs.erase(it);
    return SCA_OK;
}

int sca_server_get_stats(sca_server *srv, sca_server_stats *out)
{
    if (!srv || !out) return fail(SCA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    out->active = 0;
    for (const Slot &sl : srv->slots) out->active += sl.busy ? 1u : 0u;
    out->pending = (uint32_t)srv->pending.size();
    out->bytes_in_use = srv->used;
    out->budget_bytes = srv->budget;
    return SCA_OK;
}

void sca_server_destroy(sca_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    for (auto &kv : srv->reqs) delete kv.second;
    for (Slot &sl : srv->slots) {
        for (cudaStream_t st : {sl.stream, sl.stream_hi}) {
            if (!st) continue;
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    delete srv;
}

}  // extern "C"
