// Serving loop: clustering requests of very different sizes arrive over time
// (in-situ analysis of many sub-volumes); a scheduler thread admits them in
// batches under an HBM budget and runs each batch through the batched
// pipeline (one pass over a concatenated, segmented hierarchy) on one of a
// few slot streams, so batches that are admitted while others run overlap on
// the GPU (continuous batching).  Each request's labels are exactly those
// abx_dbscan gives for it alone: labels are a pure function of (points, eps,
// minPts), whatever else shares the batch.
//
// Host-side fault injection for tests (never a GPU fault): the environment
// variable ABX_SERVE_FAULT, read when a server is created, set to "hold"
// admits nothing (requests wait until destroy cancels them) and set to
// "alloc" makes every batch's device allocation fail.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "work.cuh"

namespace abx {
abx_status bvh_device_ctx(cudaMemPool_t *pool, unsigned **status, int *n_sms);
}

using namespace abx;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    bool on_device = false;   // points and labels are device memory
    const float *pts = nullptr;
    int64_t n = 0;
    float eps = 0.0f;
    int32_t minpts = 0;
    int32_t *labels = nullptr;
    cudaEvent_t ready = nullptr;  // device requests: the producer stream at submit
    double t_submit = 0, t_done = 0;
    abx_status status = ABX_OK;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    bool busy = false;                   // owned by the scheduler while busy
    std::atomic<bool> gpu_done{false};   // set by the stream's completion callback
    abx_server *owner = nullptr;
    std::vector<Request *> reqs;
    std::vector<int64_t> off;
    std::vector<float> eps;
    std::vector<int32_t> minpts;
    int64_t total = 0;
    size_t reserved = 0;
    float *h_pts = nullptr;   // pinned staging, grow-only
    int32_t *h_lab = nullptr;
    int64_t cap = 0;
    abx_status launch_rc = ABX_OK;
};

}  // namespace

struct abx_server {
    abx_serve_config cfg{};
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> live;
    uint64_t next_ticket = 1;
    std::vector<std::unique_ptr<Slot>> slots;
    size_t bytes_in_use = 0, peak_bytes = 0;
    bool stop = false;
    bool fault_hold = false, fault_alloc = false;
    bool stage_points = false;  // host points through pinned staging (ABX_SERVE_STAGING=1)
                                // instead of straight from the caller's memory
    // statistics
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, batches = 0, batched_requests = 0;
    std::vector<double> latencies;
    double t_first = -1, t_last = -1;
};

namespace {

// Host copies of large staging buffers are split over a few threads (one core
// copies pageable memory far below what the host-device link carries).
void par_memcpy(void *dst, const void *src, size_t bytes)
{
    const size_t chunk = (size_t)16 << 20;
    if (bytes <= 2 * chunk) {
        memcpy(dst, src, bytes);
        return;
    }
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>(std::min<size_t>(16, hw), (bytes + chunk - 1) / chunk);
    const size_t per = (bytes + nt - 1) / nt;
    std::vector<std::thread> ts;
    for (size_t t = 1; t < nt; t++) {
        const size_t a = t * per, b = std::min(bytes, a + per);
        if (a < b)
            ts.emplace_back([=] { memcpy((char *)dst + a, (const char *)src + a, b - a); });
    }
    memcpy(dst, src, std::min(bytes, per));
    for (auto &t : ts)
        t.join();
}

// Device bytes a batch of `n` points in `nseg` segments holds while it runs:
// points and labels plus the pipeline's workspace.
size_t batch_bytes(int64_t n, int nseg)
{
    return (size_t)n * (3 * sizeof(float) + sizeof(int32_t)) + work_bytes(n < 1 ? 1 : n, nseg) + (1 << 20);
}

// Runs on a CUDA-internal thread once the slot's stream has passed the batch.
// It takes the server lock only for an instant (so the scheduler cannot miss
// the wakeup between its check and its wait); this is safe because no thread
// ever holds that lock across a CUDA call.
void CUDART_CB on_batch_done(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    abx_server *sv = sl->owner;
    sl->gpu_done.store(true);
    { std::lock_guard<std::mutex> lk(sv->mu); }
    sv->cv_work.notify_all();
}

void finish_request(abx_server *sv, Request *r, abx_status st, double t)
{
    r->status = st;
    r->done = true;
    r->t_done = t;
    if (st == ABX_OK) {
        sv->completed++;
        sv->latencies.push_back(t - r->t_submit);
        sv->t_last = std::max(sv->t_last, t);
    } else if (st == ABX_ECANCELLED) {
        sv->cancelled++;
    } else {
        sv->failed++;
    }
}

// Called with the lock held once the slot's stream has passed the batch.
void finish_slot(abx_server *sv, Slot &sl)
{
    const double t = now_s();
    const abx_status st = sl.launch_rc;
    for (size_t k = 0; k < sl.reqs.size(); k++) {
        Request *r = sl.reqs[k];
        if (st == ABX_OK && !r->on_device)
            par_memcpy(r->labels, sl.h_lab + sl.off[k], (size_t)r->n * sizeof(int32_t));
        finish_request(sv, r, st, t);
    }
    sv->bytes_in_use -= sl.reserved;
    sl.reserved = 0;
    sl.reqs.clear();
    sl.busy = false;
    sl.gpu_done.store(false);
    sv->cv_done.notify_all();
}

// Enqueue one admitted batch on its slot.  Called WITHOUT the server lock:
// staging copies and CUDA calls (some of which synchronise with the device)
// must never run while the lock is held, or a completion callback waiting for
// the lock would deadlock them.  The slot and its requests belong to the
// scheduler thread until the batch finishes.
void launch_slot(abx_server *sv, Slot &sl)
{
    sl.launch_rc = ABX_OK;
    const int nseg = (int)sl.reqs.size();
    sl.off.assign(1, 0);
    sl.eps.clear();
    sl.minpts.clear();
    for (Request *r : sl.reqs) {
        sl.off.push_back(sl.off.back() + r->n);
        sl.eps.push_back(r->eps);
        sl.minpts.push_back(r->minpts);
    }
    sl.total = sl.off.back();
    int64_t host_pts = 0;
    for (Request *r : sl.reqs)
        host_pts += r->on_device ? 0 : r->n;
    // labels of host requests come back through pinned memory (a copy into
    // pageable memory would wait for the batch); points are copied from the
    // caller's memory by the driver, or staged here with ABX_SERVE_STAGING=1
    const bool stage = host_pts > 0;
    if (stage && sl.total > sl.cap) {
        if (sl.h_pts)
            cudaFreeHost(sl.h_pts);
        if (sl.h_lab)
            cudaFreeHost(sl.h_lab);
        sl.h_pts = nullptr;
        sl.h_lab = nullptr;
        sl.cap = 0;
        // once, at the batch size limit (up to 2^25 points; past that, as
        // large as the batch): pinning memory takes long enough to show in
        // the latency of the batch that would wait for it
        const int64_t cap = std::max<int64_t>(sl.total, std::min<int64_t>(sv->cfg.max_batch_points, 1ll << 25));
        if ((sv->stage_points && cudaMallocHost((void **)&sl.h_pts, (size_t)cap * 3 * sizeof(float)) != cudaSuccess) ||
            cudaMallocHost((void **)&sl.h_lab, (size_t)cap * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            sl.launch_rc = ABX_ENOMEM;
        } else {
            sl.cap = cap;
        }
    }
    void *d_pts = nullptr, *d_lab = nullptr;
    if (sl.launch_rc == ABX_OK) {
        for (int k = 0; stage && sv->stage_points && k < nseg; k++)
            if (!sl.reqs[k]->on_device)
                par_memcpy(sl.h_pts + 3 * sl.off[k], sl.reqs[k]->pts, (size_t)sl.reqs[k]->n * 3 * sizeof(float));
        if (sv->fault_alloc ||
            cudaMallocFromPoolAsync(&d_pts, (size_t)sl.total * 3 * sizeof(float), sv->pool, sl.stream) != cudaSuccess ||
            cudaMallocFromPoolAsync(&d_lab, (size_t)sl.total * sizeof(int32_t), sv->pool, sl.stream) != cudaSuccess) {
            cudaGetLastError();
            sl.launch_rc = ABX_ENOMEM;
        }
    }
    if (sl.launch_rc == ABX_OK) {
        float *dp = static_cast<float *>(d_pts);
        int32_t *dl = static_cast<int32_t *>(d_lab);
        for (int k = 0; k < nseg; k++) {  // gather the batch into one array
            Request *r = sl.reqs[k];
            if (r->ready) {  // after everything the producer had enqueued at submit
                cudaStreamWaitEvent(sl.stream, r->ready, 0);
                cudaEventDestroy(r->ready);  // released once the event has completed
                r->ready = nullptr;
            }
            const float *src = r->on_device || !sv->stage_points ? r->pts : sl.h_pts + 3 * sl.off[k];
            cudaMemcpyAsync(dp + 3 * sl.off[k], src, (size_t)r->n * 3 * sizeof(float),
                            r->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, sl.stream);
        }
        abx_status rc = abx_dbscan_batch(dp, sl.off.data(), nseg, sl.eps.data(), sl.minpts.data(), dl,
                                         reinterpret_cast<abx_stream>(sl.stream));
        if (rc != ABX_OK)
            sl.launch_rc = rc;
        else
            for (int k = 0; k < nseg; k++) {  // and scatter the labels back
                const Request *r = sl.reqs[k];
                cudaMemcpyAsync(r->on_device ? r->labels : sl.h_lab + sl.off[k], dl + sl.off[k],
                                (size_t)r->n * sizeof(int32_t),
                                r->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, sl.stream);
            }
    }
    if (d_pts)
        cudaFreeAsync(d_pts, sl.stream);
    if (d_lab)
        cudaFreeAsync(d_lab, sl.stream);
    for (Request *r : sl.reqs)  // a batch that failed before its copies
        if (r->ready) {
            cudaEventDestroy(r->ready);
            r->ready = nullptr;
        }
    if (cudaLaunchHostFunc(sl.stream, on_batch_done, &sl) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(sl.stream);
        if (sl.launch_rc == ABX_OK)
            sl.launch_rc = ABX_ECUDA;
        sl.gpu_done.store(true);
    }
}

// Take requests from the head of the queue while they fit the slot, the batch
// limits and the HBM budget left.  Called with the lock held.
bool admit(abx_server *sv, Slot &sl)
{
    int64_t pts = 0;
    size_t bytes = 0;
    while (!sv->pending.empty() && (int)sl.reqs.size() < sv->cfg.max_batch_requests) {
        Request *r = sv->pending.front();
        const int64_t np = pts + r->n;
        const size_t nb = batch_bytes(np, (int)sl.reqs.size() + 1);
        if (!sl.reqs.empty() && np > sv->cfg.max_batch_points)
            break;
        if (sv->bytes_in_use + nb > sv->cfg.hbm_budget_bytes)
            break;
        sl.reqs.push_back(r);
        sv->pending.pop_front();
        pts = np;
        bytes = nb;
    }
    if (sl.reqs.empty())
        return false;
    sl.reserved = bytes;
    sv->bytes_in_use += bytes;
    sv->peak_bytes = std::max(sv->peak_bytes, sv->bytes_in_use);
    sl.busy = true;
    sl.gpu_done.store(false);
    sv->batches++;
    sv->batched_requests += (uint64_t)sl.reqs.size();
    return true;
}

void scheduler(abx_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        bool any_busy = false;
        for (auto &sp : sv->slots) {
            if (sp->busy && sp->gpu_done.load())
                finish_slot(sv, *sp);
            any_busy |= sp->busy;
        }
        if (!sv->stop && !sv->fault_hold) {
            for (auto &sp : sv->slots) {
                if (sp->busy || sv->pending.empty())
                    continue;
                if (!admit(sv, *sp))
                    break;
                lk.unlock();
                launch_slot(sv, *sp);
                lk.lock();
                any_busy = true;
            }
        }
        if (sv->stop && !any_busy)
            break;
        bool ready = false;
        for (auto &sp : sv->slots)
            ready |= sp->busy && sp->gpu_done.load();
        if (!ready)
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(20));
    }
}

}  // namespace

extern "C" {

abx_status abx_serve_create(const abx_serve_config *cfg, abx_server **out)
{
    if (!out)
        return ABX_EINVAL;
    abx_serve_config c{};
    if (cfg)
        c = *cfg;
    if (c.hbm_budget_bytes == 0)
        c.hbm_budget_bytes = 40ull << 30;
    if (c.max_slots == 0)
        c.max_slots = 2;
    if (c.max_batch_requests == 0)
        c.max_batch_requests = 512;
    if (c.max_batch_points == 0)
        c.max_batch_points = 1ll << 25;
    if (c.max_queue == 0)
        c.max_queue = 1 << 20;
    if (c.max_slots < 1 || c.max_slots > 16 || c.max_batch_requests < 1 || c.max_batch_points < 1 ||
        c.max_batch_points > INT32_MAX || c.max_queue < 1 || c.device < 0)
        return ABX_EINVAL;
    if (cudaSetDevice(c.device) != cudaSuccess)
        return ABX_ECUDA;
    abx_server *sv = new abx_server();
    sv->cfg = c;
    sv->device = c.device;
    unsigned *status;
    int n_sms;
    abx_status rc = bvh_device_ctx(&sv->pool, &status, &n_sms);
    if (rc != ABX_OK) {
        delete sv;
        return rc;
    }
    const char *f = getenv("ABX_SERVE_FAULT");
    sv->fault_hold = f && !strcmp(f, "hold");
    sv->fault_alloc = f && !strcmp(f, "alloc");
    const char *st = getenv("ABX_SERVE_STAGING");  // "1": stage host points through pinned buffers
    sv->stage_points = st && !strcmp(st, "1");
    for (int k = 0; k < c.max_slots; k++) {
        sv->slots.emplace_back(new Slot());
        Slot &sl = *sv->slots.back();
        sl.owner = sv;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto &t : sv->slots)
                if (t->stream)
                    cudaStreamDestroy(t->stream);
            delete sv;
            return ABX_ECUDA;
        }
    }
    sv->th = std::thread(scheduler, sv);
    *out = sv;
    return ABX_OK;
}

abx_status abx_serve_submit(abx_server *sv, const float *points, int64_t n, float eps, int32_t minpts,
                            int32_t *labels, abx_stream producer, uint64_t *ticket)
{
    if (!sv || !ticket || n < 0 || n > INT32_MAX || minpts < 1 || !(eps >= 0.0f) || eps == __builtin_inff() ||
        (n > 0 && (!points || !labels)))
        return ABX_EINVAL;
    if (n > sv->cfg.max_batch_points || batch_bytes(n, 1) > sv->cfg.hbm_budget_bytes)
        return ABX_ENOMEM_BUDGET;
    // device-resident requests (the in-situ case) skip the host staging
    bool on_device = false;
    if (n > 0) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, points) == cudaSuccess)
            on_device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        else
            cudaGetLastError();
        cudaPointerAttributes b;
        bool lab_dev = false;
        if (cudaPointerGetAttributes(&b, labels) == cudaSuccess)
            lab_dev = b.type == cudaMemoryTypeDevice || b.type == cudaMemoryTypeManaged;
        else
            cudaGetLastError();
        if (lab_dev != on_device)
            return ABX_EINVAL;  // points and labels must live on the same side
    }
    cudaEvent_t ready = nullptr;
    if (on_device) {
        // the server reads the points on its own streams: order that after
        // the work the caller's producer stream holds now
        if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ready, reinterpret_cast<cudaStream_t>(producer)) != cudaSuccess) {
            cudaGetLastError();
            if (ready)
                cudaEventDestroy(ready);
            return ABX_ECUDA;
        }
    }
    Request *r = new Request();
    r->ready = ready;
    r->on_device = on_device;
    r->pts = points;
    r->n = n;
    r->eps = eps;
    r->minpts = minpts;
    r->labels = labels;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop || (int64_t)sv->pending.size() >= sv->cfg.max_queue) {
        if (r->ready)
            cudaEventDestroy(r->ready);
        const abx_status rc = sv->stop ? ABX_ECANCELLED : ABX_EBUSY;
        delete r;
        return rc;
    }
    r->ticket = sv->next_ticket++;
    r->t_submit = now_s();
    if (sv->t_first < 0)
        sv->t_first = r->t_submit;
    sv->submitted++;
    sv->live[r->ticket] = r;
    *ticket = r->ticket;
    if (n == 0) {
        finish_request(sv, r, ABX_OK, r->t_submit);
        sv->cv_done.notify_all();
        return ABX_OK;
    }
    sv->pending.push_back(r);
    sv->cv_work.notify_all();
    return ABX_OK;
}

abx_status abx_serve_wait(abx_server *sv, uint64_t ticket, int32_t timeout_ms)
{
    if (!sv)
        return ABX_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->live.find(ticket);
    if (it == sv->live.end())
        return ABX_EINVAL;
    Request *r = it->second;
    auto pred = [r] { return r->done; };
    if (timeout_ms < 0)
        sv->cv_done.wait(lk, pred);
    else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return ABX_ETIMEOUT;
    const abx_status st = r->status;
    sv->live.erase(it);
    delete r;
    return st;
}

static double percentile(std::vector<double> v, double q)
{
    if (v.empty())
        return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

abx_status abx_serve_stats(abx_server *sv, abx_serve_report *out)
{
    if (!sv || !out)
        return ABX_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->cancelled = sv->cancelled;
    out->batches = sv->batches;
    out->queued = sv->pending.size();
    out->bytes_in_use = sv->bytes_in_use;
    out->peak_bytes = sv->peak_bytes;
    out->p50_ms = 1e3 * percentile(sv->latencies, 0.50);
    out->p99_ms = 1e3 * percentile(sv->latencies, 0.99);
    double sum = 0, mx = 0;
    for (double x : sv->latencies) {
        sum += x;
        mx = std::max(mx, x);
    }
    out->mean_ms = sv->latencies.empty() ? 0.0 : 1e3 * sum / (double)sv->latencies.size();
    out->max_ms = 1e3 * mx;
    const double span = sv->t_last - sv->t_first;
    out->requests_per_s = span > 0 ? (double)sv->completed / span : 0.0;
    out->mean_batch_requests = sv->batches ? (double)sv->batched_requests / (double)sv->batches : 0.0;
    return ABX_OK;
}

abx_status abx_serve_destroy(abx_server *sv)
{
    if (!sv)
        return ABX_EINVAL;
    std::vector<cudaEvent_t> events;  // released after the lock (no CUDA call under it)
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        const double t = now_s();
        for (Request *r : sv->pending) {
            if (r->ready)
                events.push_back(r->ready);
            r->ready = nullptr;
            finish_request(sv, r, ABX_ECANCELLED, t);
        }
        sv->pending.clear();
    }
    for (cudaEvent_t e : events)
        cudaEventDestroy(e);
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
    if (sv->th.joinable())
        sv->th.join();  // batches already on the GPU run to completion
    for (auto &sp : sv->slots) {
        cudaStreamSynchronize(sp->stream);
        cudaStreamDestroy(sp->stream);
        if (sp->h_pts)
            cudaFreeHost(sp->h_pts);
        if (sp->h_lab)
            cudaFreeHost(sp->h_lab);
    }
    for (auto &kv : sv->live)
        delete kv.second;
    delete sv;
    return ABX_OK;
}

}  // extern "C"
