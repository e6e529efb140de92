// Serving runtime for streams of independent scans on one GPU.
//
// One device arena (a single cudaMalloc at creation) is carved by a first-fit
// allocator with coalescing into resident slots, each holding one scan's
// sinogram, volume, reconstruction workspace and statistics. Two host threads
// run the pipeline:
//   scheduler  -- admits queued scans in arrival order (reusing an idle slot of
//                 the same geometry and parameters, else allocating one, else
//                 evicting idle slots least recently used first, else waiting
//                 for a completion), picks the compute lane with the least
//                 work queued, then enqueues: host-to-device copy on the
//                 copy-in stream, the reconstruction on the lane's compute
//                 stream (after an event on the copy), device-to-host copies
//                 on the lane's copy-out stream (after an event on the
//                 compute);
//   completion -- waits for each scan's final event (in issue order with one
//                 lane; by polling with several), stamps the times, frees the
//                 slot for reuse and wakes the waiters.
// With k lanes, k reconstructions run at once. The TV step is a cooperative
// kernel whose blocks wait on one another; the scheduler thread launches it
// on 1/k of the GPU's resident capacity, so the k solves in flight always
// fit together, and the other kernels never wait on anything, so a solve
// whose blocks are not yet resident gets them as those kernels drain. The
// solve's sums are independent of its grid size, so a served scan equals a
// direct reconstruction bit for bit. With graphs enabled, a slot's first
// reconstruction is captured (on a private stream) and instantiated; later
// scans in the slot replay the graph with a single launch.
//
// Step reuse (config.reuse_steps): the step size tau = 1/L of each multigrid
// level comes from power iterations on kappa P^T P, which depend on the
// geometry and the schedule only, never on a scan's data. The first scan of a
// (geometry, parameters) pair runs them and its statistics record tau and L;
// later scans of the pair run with those taus given. The kernels are
// deterministic, so the given taus are the very doubles the power iterations
// would produce again, and a scan that reuses them still equals the direct
// reconstruction bit for bit (its statistics report the same tau and L).
#include "cbct_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cstddef>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace cbct {
void set_thread_quiet(bool quiet);
}

constexpr int kMaxLanes = 16;

using namespace cbct;

namespace {

constexpr size_t kAlign = 256;
constexpr int kPinnedHeads = 64;   // statistics heads copied out at once for step reuse
// leading fields of cbct_recon_stats that step reuse reads back: tau, lipschitz,
// n_iters, flags, status
constexpr size_t kStatsHead = offsetof(cbct_recon_stats, n_steps);
size_t round_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing on free.
class Arena {
  public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            in_use_ += bytes;
            peak_ = std::max(peak_, in_use_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes);
        in_use_ -= bytes;
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
    size_t size() const { return size_; }
    size_t in_use() const { return in_use_; }
    size_t peak() const { return peak_; }

  private:
    size_t size_, in_use_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length
};

struct Slot {
    const cbct_geometry *geom = nullptr;
    uint64_t geom_serial = 0;   // geometries are matched by serial, never by address
    cbct_recon_params params{};       // as submitted (slots are matched on these)
    cbct_recon_params run{};          // as launched: with reused taus filled in
    bool run_reuses_steps = false;    // the captured graph (if any) was made from such params
    size_t off = 0, bytes = 0;
    float *sino = nullptr, *vol = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cbct_recon_stats *stats = nullptr;
    size_t nvox = 0, nray = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    bool busy = false;
    bool live = false;
    uint64_t last_used = 0;
};

struct Job {
    uint64_t ticket = 0;
    const cbct_geometry *geom = nullptr;
    cbct_recon_params params{};
    const float *h_sino = nullptr;
    float *h_vol = nullptr;
    cbct_recon_stats *h_stats = nullptr;
    cbct_scan_result res{};
    int slot = -1;
    int lane = 0;
    double cost = 0.0;   // work estimate: rays x in-plane voxels along a ray
    cbct_recon_params run{};   // params as launched (reused taus filled in)
    int step_entry = -1;       // entry of the step cache this scan reads or fills
    bool steps_reused = false; // runs with the entry's taus instead of power iterations
    int pin = -1;              // pinned statistics head this scan fills the entry from
    cudaEvent_t ev_in = nullptr, ev_start = nullptr, ev_stop = nullptr, ev_out = nullptr;
    bool done = false;
};

bool same_params(const cbct_recon_params &a, const cbct_recon_params &b)
{
    return std::memcmp(&a, &b, sizeof(a)) == 0;
}

// Does the reconstruction run power iterations on some level (tau not given)?
bool needs_power(const cbct_recon_params &p)
{
    for (int l = 0; l < p.n_levels && l < CBCT_MAX_LEVELS; l++)
        if (!(p.tau[l] > 0)) return true;
    return false;
}

// Step sizes learned for one (geometry, parameters) pair.
struct StepEntry {
    uint64_t geom_serial = 0;
    cbct_recon_params params{};
    bool ready = false;     // tau and lipschitz hold the pair's values
    bool pending = false;   // a scan in flight will fill them
    double tau[CBCT_MAX_LEVELS] = {};
    double lipschitz[CBCT_MAX_LEVELS] = {};
};

size_t slot_bytes(const cbct_geometry *G, const cbct_recon_params *p, size_t *ws_bytes)
{
    const VolGeom *v = geometry_level(G, 0);
    const DetGeom *d = geometry_detector(G);
    size_t ws = 0;
    if (cbct_workspace_size(G, p, &ws) != CBCT_OK) return 0;
    *ws_bytes = ws;
    return round_up(sizeof(float) * (size_t)d->n_views * d->nv * d->nu) +
           round_up(sizeof(float) * (size_t)v->nx * v->ny * v->nz) + round_up(ws) +
           round_up(sizeof(cbct_recon_stats));
}

} // namespace

struct cbct_server {
    int device = 0;
    cbct_server_config cfg{};
    char *base = nullptr;
    std::unique_ptr<Arena> arena;
    cudaStream_t s_in = nullptr, s_cap = nullptr;
    int lanes = 1;
    cudaStream_t s_comp[kMaxLanes] = {}, s_out[kMaxLanes] = {};
    double lane_work[kMaxLanes] = {};   // cost of the scans in flight per lane
    std::chrono::steady_clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<std::shared_ptr<Job>> queue;       // submitted, not admitted
    std::deque<std::shared_ptr<Job>> inflight;    // issued, not completed
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
    std::vector<Slot> slots;
    std::vector<StepEntry> steps;      // step cache (reuse_steps)
    char *pinned = nullptr;            // kPinnedHeads statistics heads, page-locked
    std::vector<int> pin_free;
    uint64_t next_ticket = 1, use_clock = 0;
    bool stop = false;
    int64_t submitted = 0, completed = 0, evictions = 0, step_reuses = 0;
    int graphs_captured = 0, graph_failures = 0;
    std::thread sched, compl_;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void free_slot(cbct_server *S, int i)
{
    Slot &sl = S->slots[i];
    if (sl.graph) cudaGraphExecDestroy(sl.graph);
    S->arena->release(sl.off, sl.bytes);
    sl = Slot{};
}

// Find or make a slot for the job; -1 when none is possible right now.
int acquire_slot(cbct_server *S, const Job &j)
{
    int idle_same = -1;
    for (int i = 0; i < (int)S->slots.size(); i++) {
        const Slot &sl = S->slots[i];
        if (sl.live && !sl.busy && sl.geom_serial == geometry_serial(j.geom) && same_params(sl.params, j.params)) {
            idle_same = i;
            break;
        }
    }
    if (idle_same >= 0) return idle_same;
    size_t ws_bytes = 0;
    const size_t need = slot_bytes(j.geom, &j.params, &ws_bytes);
    int live = 0;
    for (const Slot &sl : S->slots) live += sl.live;
    size_t off = 0;
    while (true) {
        const bool cap_ok = S->cfg.max_resident <= 0 || live < S->cfg.max_resident;
        if (cap_ok && S->arena->alloc(need, &off)) break;
        // evict the least recently used idle slot
        int victim = -1;
        for (int i = 0; i < (int)S->slots.size(); i++) {
            const Slot &sl = S->slots[i];
            if (sl.live && !sl.busy && (victim < 0 || sl.last_used < S->slots[victim].last_used)) victim = i;
        }
        if (victim < 0) return -1;
        free_slot(S, victim);
        live--;
        S->evictions++;
    }
    int idx = -1;
    for (int i = 0; i < (int)S->slots.size(); i++)
        if (!S->slots[i].live) {
            idx = i;
            break;
        }
    if (idx < 0) {
        S->slots.emplace_back();
        idx = (int)S->slots.size() - 1;
    }
    Slot &sl = S->slots[idx];
    const VolGeom *v = geometry_level(j.geom, 0);
    const DetGeom *d = geometry_detector(j.geom);
    sl.live = true;
    sl.geom = j.geom;
    sl.geom_serial = geometry_serial(j.geom);
    sl.params = j.params;
    sl.run = j.params;
    sl.run_reuses_steps = false;
    sl.off = off;
    sl.bytes = need;
    sl.nray = (size_t)d->n_views * d->nv * d->nu;
    sl.nvox = (size_t)v->nx * v->ny * v->nz;
    char *p = S->base + off;
    sl.sino = reinterpret_cast<float *>(p);
    p += round_up(sizeof(float) * sl.nray);
    sl.vol = reinterpret_cast<float *>(p);
    p += round_up(sizeof(float) * sl.nvox);
    sl.ws = p;
    sl.ws_bytes = ws_bytes;
    p += round_up(ws_bytes);
    sl.stats = reinterpret_cast<cbct_recon_stats *>(p);
    return idx;
}

// The reconstruction of one slot, as enqueued work on stream s.
cbct_status enqueue_recon(Slot &sl, cudaStream_t s)
{
    if (cudaMemsetAsync(sl.vol, 0, sizeof(float) * sl.nvox, s) != cudaSuccess)
        return report_error(CBCT_ERR_CUDA, "cudaMemsetAsync of the slot volume failed");
    return cbct_reconstruct(sl.geom, sl.sino, sl.vol, &sl.run, sl.ws, sl.ws_bytes, sl.stats, s);
}

// Capture the slot's reconstruction once; false leaves the slot on direct launches.
bool capture_slot(cbct_server *S, Slot &sl)
{
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(S->s_cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const cbct_status st = enqueue_recon(sl, S->s_cap);
    const cudaError_t e = cudaStreamEndCapture(S->s_cap, &g);
    if (st != CBCT_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    sl.graph = ex;
    return true;
}

// Step reuse: give the job the cached taus of its (geometry, parameters)
// pair, or make it the scan that fills them (one filler at a time per pair).
void plan_steps(cbct_server *S, Job &j)
{
    j.run = j.params;
    if (!S->cfg.reuse_steps || !needs_power(j.params)) return;
    const uint64_t serial = geometry_serial(j.geom);
    int e = -1;
    for (int i = 0; i < (int)S->steps.size(); i++)
        if (S->steps[i].geom_serial == serial && same_params(S->steps[i].params, j.params)) {
            e = i;
            break;
        }
    if (e >= 0 && S->steps[e].ready) {
        for (int l = 0; l < j.params.n_levels && l < CBCT_MAX_LEVELS; l++)
            if (!(j.params.tau[l] > 0)) j.run.tau[l] = S->steps[e].tau[l];
        j.step_entry = e;
        j.steps_reused = true;
        return;
    }
    if ((e >= 0 && S->steps[e].pending) || S->pin_free.empty()) return;
    if (e < 0) {
        StepEntry se;
        se.geom_serial = serial;
        se.params = j.params;
        S->steps.push_back(se);
        e = (int)S->steps.size() - 1;
    }
    S->steps[e].pending = true;
    j.step_entry = e;
    j.pin = S->pin_free.back();
    S->pin_free.pop_back();
}

// After the job's copy-out: a filler stores the taus its power iterations
// found (if the reconstruction succeeded); a reuser reports the cached L in
// its statistics, as the power iterations would have.
void finish_steps(cbct_server *S, Job &j, bool ok)
{
    if (j.step_entry < 0) return;
    StepEntry &se = S->steps[j.step_entry];
    if (j.pin >= 0) {
        cbct_recon_stats head;
        std::memcpy(&head, S->pinned + (size_t)j.pin * kStatsHead, kStatsHead);
        if (ok && head.status == CBCT_OK) {
            for (int l = 0; l < CBCT_MAX_LEVELS; l++) {
                se.tau[l] = head.tau[l];
                se.lipschitz[l] = head.lipschitz[l];
            }
            se.ready = true;
        }
        se.pending = false;
        S->pin_free.push_back(j.pin);
        j.pin = -1;
    }
    if (j.steps_reused && ok && j.h_stats)
        for (int l = 0; l < j.params.n_levels && l < CBCT_MAX_LEVELS; l++)
            if (!(j.params.tau[l] > 0)) j.h_stats->lipschitz[l] = se.lipschitz[l];
}

void fail_job(cbct_server *S, const std::shared_ptr<Job> &j, cbct_status st)
{
    j->res.status = st;
    j->res.t_done = S->now();
    j->done = true;
    S->completed++;
}

void scheduler_loop(cbct_server *S)
{
    cudaSetDevice(S->device);
    set_thread_quiet(true);
    // the TV solves this thread launches (directly or into graphs) take 1/lanes of the GPU
    set_rof_grid_share(S->lanes);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_sched.wait(lk, [&] { return S->stop || !S->queue.empty(); });
        if (S->queue.empty()) {
            if (S->stop) break;
            continue;
        }
        std::shared_ptr<Job> j = S->queue.front();
        if (j->step_entry < 0) plan_steps(S, *j);
        const int si = acquire_slot(S, *j);
        if (si < 0) {  // every slot busy: wait for a completion
            S->cv_sched.wait(lk);
            continue;
        }
        S->queue.pop_front();
        Slot &sl = S->slots[si];
        sl.busy = true;
        sl.last_used = ++S->use_clock;
        j->slot = si;
        j->res.slot = si;
        j->res.t_admit = S->now();
        // the lane with the least work in flight
        int lane = 0;
        for (int l = 1; l < S->lanes; l++)
            if (S->lane_work[l] < S->lane_work[lane]) lane = l;
        j->lane = lane;
        {
            const VolGeom *v = geometry_level(j->geom, 0);
            const DetGeom *d = geometry_detector(j->geom);
            j->cost = (double)d->n_views * d->nv * d->nu * (double)std::max(v->nx, v->ny);
        }
        S->lane_work[lane] += j->cost;
        cudaStream_t s_comp = S->s_comp[lane], s_out = S->s_out[lane];
        if (!same_params(sl.run, j->run) || sl.run_reuses_steps != j->steps_reused) {
            // the slot's graph was made from other launch parameters
            if (sl.graph) cudaGraphExecDestroy(sl.graph);
            sl.graph = nullptr;
            sl.graph_failed = false;
            sl.run = j->run;
            sl.run_reuses_steps = j->steps_reused;
        }
        // issue (the lock is held: slots and the arena are not touched elsewhere
        // while this runs, and the enqueue calls do not block)
        cbct_status st = CBCT_OK;
        bool ok = cudaMemcpyAsync(sl.sino, j->h_sino, sizeof(float) * sl.nray, cudaMemcpyHostToDevice,
                                  S->s_in) == cudaSuccess &&
                  cudaEventRecord(j->ev_in, S->s_in) == cudaSuccess &&
                  cudaStreamWaitEvent(s_comp, j->ev_in, 0) == cudaSuccess;
        if (ok && S->cfg.use_graphs && !sl.graph && !sl.graph_failed) {
            if (capture_slot(S, sl)) {
                S->graphs_captured++;
            } else {
                sl.graph_failed = true;
                S->graph_failures++;
            }
        }
        ok = ok && cudaEventRecord(j->ev_start, s_comp) == cudaSuccess;
        if (ok) {
            if (sl.graph) {
                ok = cudaGraphLaunch(sl.graph, s_comp) == cudaSuccess;
                j->res.graph_replay = 1;
            } else {
                st = enqueue_recon(sl, s_comp);
                ok = st == CBCT_OK;
            }
        }
        ok = ok && cudaEventRecord(j->ev_stop, s_comp) == cudaSuccess &&
             cudaStreamWaitEvent(s_out, j->ev_stop, 0) == cudaSuccess &&
             cudaMemcpyAsync(j->h_vol, sl.vol, sizeof(float) * sl.nvox, cudaMemcpyDeviceToHost, s_out) ==
                 cudaSuccess &&
             (!j->h_stats || cudaMemcpyAsync(j->h_stats, sl.stats, sizeof(cbct_recon_stats),
                                             cudaMemcpyDeviceToHost, s_out) == cudaSuccess) &&
             (j->pin < 0 || cudaMemcpyAsync(S->pinned + (size_t)j->pin * kStatsHead, sl.stats, kStatsHead,
                                            cudaMemcpyDeviceToHost, s_out) == cudaSuccess) &&
             cudaEventRecord(j->ev_out, s_out) == cudaSuccess;
        if (!ok) {
            // work may be partially enqueued: let it drain before the slot is reused
            cudaGetLastError();
            cudaStreamSynchronize(S->s_in);
            cudaStreamSynchronize(s_comp);
            cudaStreamSynchronize(s_out);
            S->lane_work[lane] -= j->cost;
            sl.busy = false;
            finish_steps(S, *j, false);
            fail_job(S, j, st != CBCT_OK ? st : CBCT_ERR_CUDA);
            S->cv_done.notify_all();
            continue;
        }
        if (j->steps_reused) S->step_reuses++;
        S->inflight.push_back(j);
        S->cv_done.notify_all();
    }
}

void complete_job(cbct_server *S, const std::shared_ptr<Job> &j, cudaError_t e)
{
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, j->ev_start, j->ev_stop);
    Slot &sl = S->slots[j->slot];
    j->res.gpu_ms = ms;
    j->res.status = e == cudaSuccess ? CBCT_OK : CBCT_ERR_CUDA;
    if (e == cudaSuccess && j->h_stats) j->res.recon_flags = j->h_stats->flags;
    j->res.steps_reused = j->steps_reused ? 1 : 0;
    finish_steps(S, *j, e == cudaSuccess);
    j->res.t_done = S->now();
    j->done = true;
    S->lane_work[j->lane] -= j->cost;
    sl.busy = false;
    sl.last_used = ++S->use_clock;
    S->completed++;
}

void completion_loop(cbct_server *S)
{
    cudaSetDevice(S->device);
    set_thread_quiet(true);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_done.wait(lk, [&] { return !S->inflight.empty() || (S->stop && S->queue.empty()); });
        if (S->inflight.empty()) {
            if (S->stop && S->queue.empty()) break;
            continue;
        }
        if (S->lanes == 1) {
            // one lane completes in issue order: wait for the oldest scan
            std::shared_ptr<Job> j = S->inflight.front();
            lk.unlock();
            const cudaError_t e = cudaEventSynchronize(j->ev_out);
            lk.lock();
            S->inflight.pop_front();
            complete_job(S, j, e);
        } else {
            // several lanes finish out of order: collect every finished scan, else
            // poll again shortly
            bool any = false;
            for (auto it = S->inflight.begin(); it != S->inflight.end();) {
                const cudaError_t e = cudaEventQuery((*it)->ev_out);
                if (e == cudaErrorNotReady) {
                    ++it;
                    continue;
                }
                complete_job(S, *it, e);
                it = S->inflight.erase(it);
                any = true;
            }
            if (!any) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(100));
                lk.lock();
                continue;
            }
        }
        S->cv_done.notify_all();
        S->cv_sched.notify_all();
    }
}

} // namespace

extern "C" cbct_status cbct_server_create(const cbct_server_config *cfg, cbct_server **out)
{
    if (!out) return report_error(CBCT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    cbct_server_config c{};
    if (cfg) c = *cfg;
    if (c.max_resident < 0) return report_error(CBCT_ERR_INVALID_ARG, "max_resident must be >= 0");
    if (c.concurrency < 0 || c.concurrency > kMaxLanes)
        return report_error(CBCT_ERR_INVALID_ARG, "concurrency must be between 0 and 16");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return report_error(CBCT_ERR_CUDA, "no CUDA device");
    if (c.arena_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return report_error(CBCT_ERR_CUDA, "cudaMemGetInfo failed");
        c.arena_bytes = std::min(fr / 2, (size_t)64 << 30);
    }
    c.arena_bytes = round_up(c.arena_bytes);
    auto S = std::make_unique<cbct_server>();
    S->device = dev;
    S->cfg = c;
    S->t0 = std::chrono::steady_clock::now();
    if (cudaMalloc((void **)&S->base, c.arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        return report_error(CBCT_ERR_OUT_OF_MEMORY, "cudaMalloc of the serving arena failed");
    }
    S->arena = std::make_unique<Arena>(c.arena_bytes);
    if (c.reuse_steps) {
        if (cudaHostAlloc((void **)&S->pinned, kStatsHead * kPinnedHeads, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(S->base);
            return report_error(CBCT_ERR_OUT_OF_MEMORY, "cudaHostAlloc of the step-reuse buffer failed");
        }
        for (int i = kPinnedHeads - 1; i >= 0; i--) S->pin_free.push_back(i);
    }
    S->lanes = c.concurrency > 1 ? c.concurrency : 1;
    std::vector<cudaStream_t *> streams = {&S->s_in, &S->s_cap};
    for (int l = 0; l < S->lanes; l++) {
        streams.push_back(&S->s_comp[l]);
        streams.push_back(&S->s_out[l]);
    }
    for (cudaStream_t *s : streams)
        if (cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t *t : streams)
                if (*t) cudaStreamDestroy(*t);
            if (S->pinned) cudaFreeHost(S->pinned);
            cudaFree(S->base);
            return report_error(CBCT_ERR_CUDA, "cudaStreamCreate failed");
        }
    cbct_server *raw = S.get();
    S->sched = std::thread(scheduler_loop, raw);
    S->compl_ = std::thread(completion_loop, raw);
    *out = S.release();
    return CBCT_OK;
}

extern "C" void cbct_server_destroy(cbct_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_sched.notify_all();
    S->cv_done.notify_all();
    if (S->sched.joinable()) S->sched.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
    }
    S->cv_done.notify_all();
    if (S->compl_.joinable()) S->compl_.join();
    cudaSetDevice(S->device);
    for (auto &kv : S->jobs) {
        Job &j = *kv.second;
        cudaEvent_t evs[4] = {j.ev_in, j.ev_start, j.ev_stop, j.ev_out};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
    }
    for (Slot &sl : S->slots)
        if (sl.graph) cudaGraphExecDestroy(sl.graph);
    cudaStream_t streams[2] = {S->s_in, S->s_cap};
    for (cudaStream_t s : streams)
        if (s) cudaStreamDestroy(s);
    for (int l = 0; l < S->lanes; l++) {
        if (S->s_comp[l]) cudaStreamDestroy(S->s_comp[l]);
        if (S->s_out[l]) cudaStreamDestroy(S->s_out[l]);
    }
    if (S->pinned) cudaFreeHost(S->pinned);
    cudaFree(S->base);
    delete S;
}

extern "C" cbct_status cbct_server_submit(cbct_server *S, const cbct_geometry *G, const cbct_recon_params *p,
                                          const float *h_sino, float *h_vol, cbct_recon_stats *h_stats,
                                          uint64_t *ticket)
{
    if (!S || !G || !p || !h_sino || !h_vol || !ticket) return report_error(CBCT_ERR_INVALID_ARG, "NULL argument");
    if (p->replay) return report_error(CBCT_ERR_INVALID_ARG, "a served scan takes no replay schedule");
    if (geometry_device(G) != S->device) return report_error(CBCT_ERR_INVALID_ARG, "geometry belongs to another device");
    const void *host_ptrs[3] = {h_sino, h_vol, h_stats};
    for (const void *hp : host_ptrs) {
        if (!hp) continue;
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, hp) != cudaSuccess || a.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return report_error(CBCT_ERR_INVALID_ARG, "host buffers must be page-locked (cudaHostAlloc/cudaHostRegister)");
        }
    }
    size_t ws_bytes = 0;
    const size_t need = slot_bytes(G, p, &ws_bytes);
    if (need == 0) return report_error(CBCT_ERR_INVALID_ARG, "invalid reconstruction parameters");
    if (need > S->arena->size())
        return report_error(CBCT_ERR_OUT_OF_MEMORY, "the scan's slot is larger than the serving arena");
    auto j = std::make_shared<Job>();
    j->geom = G;
    j->params = *p;
    j->h_sino = h_sino;
    j->h_vol = h_vol;
    j->h_stats = h_stats;
    cudaSetDevice(S->device);
    cudaEvent_t *evs[4] = {&j->ev_in, &j->ev_start, &j->ev_stop, &j->ev_out};
    for (int i = 0; i < 4; i++) {
        const unsigned flags = (i == 1 || i == 2) ? cudaEventDefault : (cudaEventDisableTiming | cudaEventBlockingSync);
        if (cudaEventCreateWithFlags(evs[i], flags) != cudaSuccess) {
            for (int k = 0; k < i; k++) cudaEventDestroy(*evs[k]);
            return report_error(CBCT_ERR_CUDA, "cudaEventCreate failed");
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        j->ticket = S->next_ticket++;
        j->res.ticket = j->ticket;
        j->res.t_submit = S->now();
        j->res.slot = -1;
        S->jobs[j->ticket] = j;
        S->queue.push_back(j);
        S->submitted++;
        *ticket = j->ticket;
    }
    S->cv_sched.notify_all();
    return CBCT_OK;
}

extern "C" cbct_status cbct_server_wait(cbct_server *S, uint64_t ticket, cbct_scan_result *res)
{
    if (!S) return report_error(CBCT_ERR_INVALID_ARG, "server is NULL");
    std::shared_ptr<Job> j;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->jobs.find(ticket);
        if (it == S->jobs.end()) return report_error(CBCT_ERR_INVALID_ARG, "unknown or already collected ticket");
        j = it->second;
        S->cv_done.wait(lk, [&] { return j->done; });
        S->jobs.erase(it);
    }
    cudaEvent_t evs[4] = {j->ev_in, j->ev_start, j->ev_stop, j->ev_out};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (res) *res = j->res;
    return j->res.status == CBCT_OK ? CBCT_OK
                                    : report_error((cbct_status)j->res.status, "the scan's reconstruction failed");
}

extern "C" cbct_status cbct_server_query(cbct_server *S, cbct_server_info *info)
{
    if (!S || !info) return report_error(CBCT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    info->arena_bytes = S->arena->size();
    info->bytes_in_use = S->arena->in_use();
    info->peak_bytes_in_use = S->arena->peak();
    info->slots = 0;
    info->busy_slots = 0;
    for (const Slot &sl : S->slots) {
        info->slots += sl.live;
        info->busy_slots += sl.live && sl.busy;
    }
    info->graphs_captured = S->graphs_captured;
    info->graph_failures = S->graph_failures;
    info->submitted = S->submitted;
    info->completed = S->completed;
    info->evictions = S->evictions;
    info->step_reuses = S->step_reuses;
    return CBCT_OK;
}
