// server.cu -- native serving engine: requests of mixed page sizes and
// windows are admitted under a device-memory budget and binarized by
// continuous batching, with the host<->device copies overlapped on their own
// streams.  Host code only; the kernels are the fused / batched ones.
//
// One scheduler thread moves every request through
//   waiting -> admitted (input copy in flight) -> ready -> running (one
//   batched launch per step, steps alternate between compute streams) ->
//   delivering (mask copy in flight) -> done (polled by the caller).
// Admission is in arrival order and waits (never drops) while the arena has
// no free range for the request's buffers.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxStreams = 4;

struct Req {
    bnz_request r{};
    size_t in_bytes = 0, out_bytes = 0; // device buffers (pitched)
    size_t sp = 0, dp = 0;              // device pitches
    void *blk = nullptr;                // pool block holding both
    const uint8_t *d_src = nullptr;
    uint8_t *d_dst = nullptr;
    cudaEvent_t ev = nullptr;           // input copy, then mask copy
    Clock::time_point t0;
    double latency = 0.0;
    int status = BNZ_OK;
};

struct Step {
    cudaEvent_t ev = nullptr;
    std::vector<Req *> reqs;
    bnz_batch *batch = nullptr;
    int stream = 0;       // compute stream index (its statistics slot)
    int status = BNZ_OK;  // a launch failure after some of the step's kernels were queued
    bool inject = false;  // test hook: report this step as timed out
};

} // namespace

struct bnz_server {
    bnz_server_config cfg{};
    int device = 0;
    void *arena = nullptr;
    bnz_pool *pool = nullptr;
    cudaStream_t cin = nullptr, cout = nullptr, comp[kMaxStreams] = {};
    void *desc[kMaxStreams] = {};
    size_t desc_bytes = 0;
    cudaEvent_t inflight[kMaxStreams] = {};
    // per compute stream: the kernels' 4 statistics counters on the device and
    // their copy in pinned host memory, read when the step is retired
    unsigned long long *d_stats = nullptr, *h_stats = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> waiting, done;
    long long outstanding = 0; // submitted, not yet polled
    std::string error;         // last failure inside the scheduler
    std::atomic<bool> stop{false};
    std::thread th;

    // scheduler thread only
    std::deque<Req *> admitted, ready, back;
    std::deque<Step> steps;
    std::vector<cudaEvent_t> events;
    int rr = 0;

    // statistics (scheduler writes, callers read under mu)
    long long completed = 0, nsteps = 0, alloc_waits = 0;
};

namespace {

void set_error(bnz_server *s, const std::string &msg)
{
    std::lock_guard<std::mutex> g(s->mu);
    s->error = msg;
}

cudaEvent_t get_event(bnz_server *s)
{
    if (!s->events.empty()) {
        cudaEvent_t e = s->events.back();
        s->events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

void put_event(bnz_server *s, cudaEvent_t e)
{
    if (e)
        s->events.push_back(e);
}

bool event_done(cudaEvent_t e)
{
    const cudaError_t q = cudaEventQuery(e);
    if (q == cudaErrorNotReady)
        return false;
    return true; // success, or an error that the next call reports
}

// Finish a request: release its device memory and hand it to the caller.
void finish(bnz_server *s, Req *q, int status)
{
    q->status = status;
    q->latency = std::chrono::duration<double>(Clock::now() - q->t0).count();
    if (q->blk)
        bnz_pool_free(s->pool, q->blk);
    q->blk = nullptr;
    put_event(s, q->ev);
    q->ev = nullptr;
    std::lock_guard<std::mutex> g(s->mu);
    s->done.push_back(q);
    ++s->completed;
    s->cv_done.notify_all();
}

bool admit(bnz_server *s)
{
    bool moved = false;
    for (;;) {
        Req *q;
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->waiting.empty())
                break;
            q = s->waiting.front();
        }
        void *blk = nullptr;
        if (bnz_pool_alloc(s->pool, q->in_bytes + q->out_bytes, &blk) != BNZ_OK) {
            ++s->alloc_waits;
            break; // wait for memory: later requests must not overtake
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->waiting.pop_front();
        }
        q->blk = blk;
        uint8_t *base = static_cast<uint8_t *>(blk);
        q->d_dst = base + q->in_bytes;
        q->ev = get_event(s);
        if (q->r.src_on_device) {
            q->d_src = q->r.src; // resident input: nothing to copy
            q->sp = q->r.src_pitch;
            cudaEventRecord(q->ev, s->cin);
        } else {
            q->d_src = base;
            const size_t row = (size_t)q->r.width * q->r.channels;
            const cudaError_t e =
                (q->sp == row && q->r.src_pitch == row) // one linear copy when both sides are dense
                    ? cudaMemcpyAsync(base, q->r.src, row * q->r.height, cudaMemcpyHostToDevice, s->cin)
                    : cudaMemcpy2DAsync(base, q->sp, q->r.src, q->r.src_pitch, row, q->r.height,
                                        cudaMemcpyHostToDevice, s->cin);
            if (e != cudaSuccess) {
                set_error(s, std::string("input copy: ") + cudaGetErrorString(e));
                finish(s, q, BNZ_ECUDA);
                moved = true;
                continue;
            }
            cudaEventRecord(q->ev, s->cin);
        }
        s->admitted.push_back(q);
        moved = true;
    }
    return moved;
}

bool collect_inputs(bnz_server *s)
{
    bool moved = false;
    while (!s->admitted.empty() && event_done(s->admitted.front()->ev)) { // copies finish in issue order
        s->ready.push_back(s->admitted.front());
        s->admitted.pop_front();
        moved = true;
    }
    return moved;
}

// Steps of fewer pages run plain launches: the batch kernel's work queue
// hands out short pieces, and for one or two pages that costs more than it
// saves (one 10-Mpixel RGB page: 77 against 45 us; two: 123 against 102 us;
// four: 208 against 241 us).
constexpr int kMinBatchPages = 3;

bool launch(bnz_server *s)
{
    if (s->ready.empty())
        return false;
    const int k = s->rr;
    if (s->inflight[k])
        return false; // one step per compute stream, until collect_steps has retired it (the stream is idle then)
    // one kernel instance (channels, rule, W mod 8) per step: the oldest ready page
    // picks it, later pages of the same instance join (up to max_batch); a launch
    // that mixes instances runs several code paths at once on the SMs and thrashes
    // their instruction caches (measured 2x slower)
    auto key = [](const Req *q) { return q->r.channels * 16 + q->r.rule * 8 + (q->r.W & 7); };
    const int want = key(s->ready.front());
    Step st;
    for (auto it = s->ready.begin(); it != s->ready.end() && (int)st.reqs.size() < s->cfg.max_batch;) {
        if (key(*it) == want) {
            st.reqs.push_back(*it);
            it = s->ready.erase(it);
        } else {
            ++it;
        }
    }
    const int n = (int)st.reqs.size();
    cudaStream_t stream = s->comp[k];
    st.stream = k;
    unsigned long long *dst = s->d_stats + 4 * k;
    int rc = BNZ_OK;
    int queued = 0; // kernels of this step already on the stream
    if (cudaMemsetAsync(dst, 0, 4 * sizeof(unsigned long long), stream) != cudaSuccess)
        rc = bnz::cuda_fail(cudaGetLastError(), "statistics reset");
    if (rc != BNZ_OK) {
    } else if (s->cfg.batched && n >= kMinBatchPages) {
        std::vector<bnz_page> pages(n);
        for (int i = 0; i < n; ++i) {
            const bnz_request &r = st.reqs[i]->r;
            bnz_page &pg = pages[i];
            memset(&pg, 0, sizeof pg);
            pg.d_src = st.reqs[i]->d_src;
            pg.src_pitch = st.reqs[i]->sp;
            pg.height = r.height;
            pg.width = r.width;
            pg.channels = r.channels;
            pg.W = r.W;
            pg.rule = r.rule;
            pg.packed = r.packed;
            pg.k = r.k;
            pg.R = r.R;
            pg.d_dst = st.reqs[i]->d_dst;
            pg.dst_pitch = st.reqs[i]->dp;
        }
        rc = bnz_batch_create_async(pages.data(), n, s->desc[k], s->desc_bytes, stream, dst, &st.batch);
        if (rc == BNZ_OK) {
            queued = 1; // the descriptor copy
            rc = bnz_batch_run(st.batch, stream);
        }
    } else {
        for (int i = 0; i < n && rc == BNZ_OK; ++i) {
            const Req *q = st.reqs[i];
            rc = bnz_binarize_dev(q->d_src, q->sp, q->r.height, q->r.width, q->r.channels, q->r.W, q->r.rule,
                                  q->r.k, q->r.R, q->d_dst, q->dp, q->r.packed, nullptr, stream, dst);
            if (rc == BNZ_OK)
                ++queued;
        }
    }
    if (rc != BNZ_OK) {
        set_error(s, bnz_last_error());
        if (!queued) { // nothing of the step reached the stream: its buffers are free now
            if (st.batch)
                bnz_batch_destroy(st.batch);
            for (Req *q : st.reqs)
                finish(s, q, rc);
            return true;
        }
        // kernels of earlier requests are queued: fail the step only once the stream has passed them,
        // so no pool block is handed out while a kernel may still write it
        st.status = rc;
    }
    if (rc == BNZ_OK)
        cudaMemcpyAsync(s->h_stats + 4 * k, dst, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream);
    st.inject = s->cfg.reserved > 0 && (s->nsteps + 1) % s->cfg.reserved == 0;
    st.ev = get_event(s);
    cudaEventRecord(st.ev, stream);
    s->inflight[k] = st.ev;
    s->rr = (k + 1) % s->cfg.compute_streams;
    s->steps.push_back(std::move(st));
    ++s->nsteps;
    return true;
}

bool collect_steps(bnz_server *s)
{
    bool moved = false;
    for (auto it = s->steps.begin(); it != s->steps.end();) {
        if (!event_done(it->ev)) {
            ++it;
            continue;
        }
        const cudaError_t e = cudaEventQuery(it->ev);
        // a CTA whose bounded wait gave up wrote no output: the step's masks are incomplete
        const unsigned long long tmo = (e == cudaSuccess && it->status == BNZ_OK)
                                           ? s->h_stats[4 * it->stream + BNZ_STATS_TIMEOUTS] + (it->inject ? 1 : 0)
                                           : 0;
        if (tmo)
            set_error(s, "a device wait timed out in a launch step; its requests fail with BNZ_ETIMEOUT");
        for (Req *q : it->reqs) {
            if (e != cudaSuccess) {
                set_error(s, std::string("kernel: ") + cudaGetErrorString(e));
                finish(s, q, BNZ_ECUDA);
                continue;
            }
            if (it->status != BNZ_OK || tmo) {
                finish(s, q, it->status != BNZ_OK ? it->status : BNZ_ETIMEOUT);
                continue;
            }
            const size_t row = q->r.packed ? ((size_t)q->r.width + 7) / 8 : (size_t)q->r.width;
            const cudaError_t c =
                (q->dp == row && q->r.dst_pitch == row)
                    ? cudaMemcpyAsync(q->r.dst, q->d_dst, row * q->r.height, cudaMemcpyDeviceToHost, s->cout)
                    : cudaMemcpy2DAsync(q->r.dst, q->r.dst_pitch, q->d_dst, q->dp, row, q->r.height,
                                        cudaMemcpyDeviceToHost, s->cout);
            if (c != cudaSuccess) {
                set_error(s, std::string("mask copy: ") + cudaGetErrorString(c));
                finish(s, q, BNZ_ECUDA);
                continue;
            }
            cudaEventRecord(q->ev, s->cout);
            s->back.push_back(q);
        }
        if (it->batch)
            bnz_batch_destroy(it->batch); // its stream has passed the step
        for (int k = 0; k < kMaxStreams; ++k)
            if (s->inflight[k] == it->ev)
                s->inflight[k] = nullptr;
        put_event(s, it->ev);
        it = s->steps.erase(it);
        moved = true;
    }
    return moved;
}

bool deliver(bnz_server *s)
{
    bool moved = false;
    while (!s->back.empty() && event_done(s->back.front()->ev)) { // copies finish in issue order
        Req *q = s->back.front();
        s->back.pop_front();
        finish(s, q, cudaEventQuery(q->ev) == cudaSuccess ? BNZ_OK : BNZ_ECUDA);
        moved = true;
    }
    return moved;
}

void run(bnz_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool moved = admit(s);
        moved |= collect_inputs(s);
        moved |= launch(s);
        moved |= collect_steps(s);
        moved |= deliver(s);
        const bool idle = s->admitted.empty() && s->ready.empty() && s->steps.empty() && s->back.empty();
        if (moved)
            continue;
        std::unique_lock<std::mutex> g(s->mu);
        if (idle && s->waiting.empty()) {
            if (s->stop)
                break;
            s->cv_work.wait_for(g, std::chrono::milliseconds(5)); // nothing in flight: sleep until a submit
        } else {
            g.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(10)); // work on the device: poll again soon
        }
    }
}

void destroy(bnz_server *s)
{
    if (s->th.joinable()) {
        s->stop = true;
        s->cv_work.notify_all();
        s->th.join();
    }
    for (Req *q : s->done)
        delete q;
    for (cudaEvent_t e : s->events)
        cudaEventDestroy(e);
    for (int k = 0; k < kMaxStreams; ++k) {
        if (s->comp[k])
            cudaStreamDestroy(s->comp[k]);
        if (s->desc[k])
            cudaFree(s->desc[k]);
    }
    if (s->cin)
        cudaStreamDestroy(s->cin);
    if (s->cout)
        cudaStreamDestroy(s->cout);
    if (s->pool)
        bnz_pool_destroy(s->pool);
    if (s->d_stats)
        cudaFree(s->d_stats);
    if (s->h_stats)
        cudaFreeHost(s->h_stats);
    if (s->arena)
        cudaFree(s->arena);
    delete s;
}

size_t round16(size_t v) { return (v + 15) & ~size_t(15); }

} // namespace

extern "C" {

int bnz_server_create(const bnz_server_config *cfg, bnz_server **out)
{
    using bnz::fail;
    if (!cfg || !out)
        return fail(BNZ_EINVAL, "bnz_server_create: null argument");
    *out = nullptr;
    if (cfg->budget_bytes < (1u << 20) || cfg->max_batch < 1 || cfg->max_batch > 4096 || cfg->compute_streams < 1 ||
        cfg->compute_streams > kMaxStreams)
        return fail(BNZ_EINVAL, "bnz_server_create: budget >= 1 MiB, max_batch in [1, 4096], compute_streams in [1, %d]",
                    kMaxStreams);
    int dev = 0, count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
        cudaGetLastError();
        return fail(BNZ_ENODEV, "no CUDA device available; this library has no CPU path");
    }
    cudaGetDevice(&dev);
    bnz_server *s = new (std::nothrow) bnz_server();
    if (!s)
        return fail(BNZ_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->device = dev;
    cudaError_t e = cudaMalloc(&s->arena, cfg->budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy(s);
        return fail(BNZ_ENOMEM, "device budget of %zu bytes could not be reserved", cfg->budget_bytes);
    }
    int rc = bnz_pool_create(s->arena, cfg->budget_bytes, &s->pool);
    if (rc != BNZ_OK) {
        destroy(s);
        return rc;
    }
    s->desc_bytes = bnz_batch_desc_bytes(cfg->max_batch);
    e = cudaMalloc(&s->d_stats, kMaxStreams * 4 * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMallocHost(&s->h_stats, kMaxStreams * 4 * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&s->cin, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&s->cout, cudaStreamNonBlocking);
    for (int k = 0; k < cfg->compute_streams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->comp[k], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaMalloc(&s->desc[k], s->desc_bytes);
    }
    if (e != cudaSuccess) {
        destroy(s);
        return bnz::cuda_fail(e, "bnz_server_create");
    }
    s->th = std::thread(run, s);
    *out = s;
    return BNZ_OK;
}

int bnz_server_submit(bnz_server *s, const bnz_request *req)
{
    using bnz::fail;
    if (!s || !req)
        return fail(BNZ_EINVAL, "bnz_server_submit: null argument");
    const bnz_request &r = *req;
    int rc = bnz::check_common(r.src, r.src_pitch, r.height, r.width, r.channels, r.W, r.rule, r.k, r.R, r.dst,
                               r.dst_pitch, r.packed);
    if (rc != BNZ_OK)
        return rc;
    if (r.src_on_device && ((reinterpret_cast<uintptr_t>(r.src) & 15u) || (r.src_pitch & 15u)))
        return fail(BNZ_EINVAL, "a device source must be 16-byte aligned with a pitch that is a multiple of 16");
    Req *q = new (std::nothrow) Req();
    if (!q)
        return fail(BNZ_ENOMEM, "host allocation failed");
    q->r = r;
    q->sp = round16((size_t)r.width * r.channels);
    q->dp = round16(r.packed ? ((size_t)r.width + 7) / 8 : (size_t)r.width);
    q->in_bytes = r.src_on_device ? 0 : (q->sp * r.height + 255) / 256 * 256;
    q->out_bytes = q->dp * r.height;
    if (q->in_bytes + q->out_bytes > s->cfg.budget_bytes) {
        delete q;
        return fail(BNZ_ENOMEM, "a request needs more device memory than the whole budget");
    }
    q->t0 = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->waiting.push_back(q);
        ++s->outstanding;
    }
    s->cv_work.notify_one();
    return BNZ_OK;
}

int bnz_server_poll(bnz_server *s, unsigned long long *tags, int *status, double *latency_s, int max, int timeout_ms)
{
    if (!s || !tags || max < 1)
        return bnz::fail(BNZ_EINVAL, "bnz_server_poll: null argument or max < 1");
    std::unique_lock<std::mutex> g(s->mu);
    if (s->done.empty() && timeout_ms > 0)
        s->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), [s] { return !s->done.empty(); });
    int n = 0;
    while (n < max && !s->done.empty()) {
        Req *q = s->done.front();
        s->done.pop_front();
        tags[n] = q->r.tag;
        if (status)
            status[n] = q->status;
        if (latency_s)
            latency_s[n] = q->latency;
        --s->outstanding;
        delete q;
        ++n;
    }
    return n;
}

int bnz_server_stats(bnz_server *s, long long *outstanding, long long *completed, long long *steps,
                     long long *alloc_waits, size_t *high_water)
{
    if (!s)
        return bnz::fail(BNZ_EINVAL, "bnz_server_stats: null server");
    std::lock_guard<std::mutex> g(s->mu);
    if (outstanding)
        *outstanding = s->outstanding;
    if (completed)
        *completed = s->completed;
    if (steps)
        *steps = s->nsteps;
    if (alloc_waits)
        *alloc_waits = s->alloc_waits;
    if (high_water)
        bnz_pool_stats(s->pool, nullptr, high_water, nullptr, nullptr);
    return BNZ_OK;
}

int bnz_server_error(bnz_server *s, char *buf, size_t n)
{
    if (!s || !buf || n == 0)
        return bnz::fail(BNZ_EINVAL, "bnz_server_error: null argument");
    std::lock_guard<std::mutex> g(s->mu);
    const size_t m = std::min(n - 1, s->error.size());
    memcpy(buf, s->error.data(), m);
    buf[m] = '\0';
    return BNZ_OK;
}

int bnz_server_destroy(bnz_server *s)
{
    if (!s)
        return BNZ_OK;
    destroy(s);
    return BNZ_OK;
}

} // extern "C"
