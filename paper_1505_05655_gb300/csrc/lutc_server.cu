// Serving: an in-process request loop (lutc_server_*).
//
// The paper's framework is a GPU server that receives tasks from clients,
// processes them and returns the results (Sections I-II).  This is that
// server's core, in process: no sockets, requests are function calls.
//
//   submit ──> pending queue ──> batcher thread ──> in-flight batches ──> completer thread ──> wait
//               (bounded;        admission by the      (up to `streams`,     (event polling,
//                cancel takes    device budget,         each a lutc_batch     frees memory,
//                a request out)  window of max_batch    on its own stream)    wakes waiters)
//                                or max_wait_us
//
// Continuous batching: a request that finds no batch on the device launches at
// once; while batches run on some streams, the batcher gathers new requests
// into the next batch, which leaves on a free stream when it is full, when its
// window closes or when the device goes idle, and memory allows.  Device memory comes from one slab of
// budget_bytes allocated at creation and handed out first-fit (Arena); it
// holds the cached sensor coefficients, host requests' staging buffers and
// each batch's workspace.  A request waits in the queue until its memory
// fits.
//
// The executor can be replaced by a host-only fake (fake_device) so that the
// queueing, admission, window, timeout, shutdown and failure logic can be
// exercised without a GPU; fail_every fails batches on the host (injected
// fault, no GPU involvement).
#include <stdint.h>
#include <string.h>
#ifdef __linux__
#include <sys/prctl.h>
#endif

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lutc_internal.cuh"

using namespace lutc;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over offsets [0, size), 256-byte granules, coalescing frees.
class Arena {
public:
    void init(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
        used_ = 0;
    }
    bool alloc(size_t n, size_t* off)
    {
        n = align_up(n ? n : 1, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = align_up(n ? n : 1, 256);
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

struct Sensor {
    int width = 0, bands = 0, bits = 0;
    std::vector<int32_t> A, G, O;  // host copies, [bands][width]
    bool cached = false;
    size_t off = 0;                // device copy: A | G | O, each [bands][width]
};

struct Request {
    uint64_t ticket = 0;
    int sensor = 0, H = 0, flags = 0;
    const uint16_t* in = nullptr;
    int64_t pitch = 0;
    uint8_t* out = nullptr;
    int64_t out_pitch = 0;
    double t_submit = 0, t_start = 0, t_launched = 0, t_done = 0;
    int status = LUTC_OK, batch_size = 0, cache_miss = 0;
    bool done = false;
    size_t in_off = 0, in_bytes = 0, out_off = 0, out_bytes = 0;  // staging (host requests)
    int64_t dpitch = 0, dopitch = 0;
    bool sm_copy = false;  // host buffers the kernels can address: rows copied by the SMs
};

struct Flight {
    std::vector<Request*> reqs;
    std::vector<const Sensor*> sensors;  // per request, snapshotted under the lock
    int slot = -1;
    size_t ws_off = 0, ws_bytes = 0;
    lutc_batch batch = nullptr;
    double t_ready = 0;  // fake executor
    double t_launched = 0;
    int status = LUTC_OK;
};

int64_t round16(int64_t v) { return (v + 15) / 16 * 16; }

}  // namespace

struct lutc_server_st {
    lutc_server_config cfg;
    int device = 0;
    void* base = nullptr;  // device slab (null with the fake executor)
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_batcher, cv_done, cv_wait;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> tickets;
    std::unordered_map<int, Sensor> sensors;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<char> slot_busy;
    cudaStream_t upload = nullptr;
    std::deque<Flight*> flights;
    std::thread batcher, completer;
    bool stop = false, stop_completer = false;
    uint64_t next_ticket = 1, completed = 0, batches = 0;
    int32_t largest = 0;

    uint8_t* dev(size_t off) { return base ? reinterpret_cast<uint8_t*>(base) + off : nullptr; }
    size_t request_staging(const Sensor& s, int H, int64_t* dpitch, int64_t* dopitch) const
    {
        *dpitch = round16(2 * (int64_t)s.width);
        *dopitch = round16(s.width);
        return (size_t)(s.bands * (int64_t)H) * (size_t)(*dpitch + *dopitch);
    }
    static size_t table_estimate(const Sensor& s)
    {
        // upper bound of a request's share of a batch workspace: histograms, stretch tables,
        // descriptors, or the workspace of a one-by-one correction
        return (size_t)s.bands * ((size_t)9 << s.bits) + (size_t)s.bands * 64 + 1536;
    }
    static size_t coef_bytes(const Sensor& s) { return (size_t)3 * s.bands * s.width * 4; }
    bool reserve(Request* r, Sensor& s, bool miss);
    void unreserve(Request* r, std::vector<int>& uploads);
    size_t exact_workspace(const std::vector<Request*>& take);
    void run_batcher();
    void run_completer();
    int launch(Flight* f);
    void finish(Flight* f);
};

// Called with the lock held: staging buffers of a host request and the sensor's coefficient
// cache on a miss; all or nothing.
bool lutc_server_st::reserve(Request* r, Sensor& s, bool miss)
{
    size_t oc = 0, oi = 0, oo = 0;
    if (miss && !arena.alloc(coef_bytes(s), &oc)) return false;
    if (r->flags & LUTC_REQ_HOST) {
        request_staging(s, r->H, &r->dpitch, &r->dopitch);
        r->in_bytes = (size_t)s.bands * r->H * r->dpitch;
        r->out_bytes = (size_t)s.bands * r->H * r->dopitch;
        if (!arena.alloc(r->in_bytes, &oi)) {
            if (miss) arena.release(oc, coef_bytes(s));
            return false;
        }
        if (!arena.alloc(r->out_bytes, &oo)) {
            arena.release(oi, r->in_bytes);
            if (miss) arena.release(oc, coef_bytes(s));
            return false;
        }
        r->in_off = oi;
        r->out_off = oo;
    }
    if (miss) s.off = oc;
    return true;
}

void lutc_server_st::unreserve(Request* r, std::vector<int>& uploads)
{
    if (r->flags & LUTC_REQ_HOST) {
        arena.release(r->in_off, r->in_bytes);
        arena.release(r->out_off, r->out_bytes);
    }
    if (r->cache_miss) {
        Sensor& s = sensors[r->sensor];
        arena.release(s.off, coef_bytes(s));
        uploads.erase(std::find(uploads.begin(), uploads.end(), r->sensor));
        r->cache_miss = 0;
    }
}

// Exact workspace of a batch of these requests (a host-only computation: addresses that decide
// the kernel path are the real ones for device requests and 256-aligned for staged ones).
size_t lutc_server_st::exact_workspace(const std::vector<Request*>& take)
{
    const size_t n = take.size();
    std::vector<std::vector<lutc_coeffs>> coefs(n);
    std::vector<lutc_job> jobs(n);
    const bool fake = cfg.fake_device != 0;
    static const int32_t dummy[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < n; ++i) {
        const Request* r = take[i];
        const Sensor& s = sensors[r->sensor];
        coefs[i].assign(s.bands, lutc_coeffs{dummy, dummy, dummy, s.width});
        const bool host = (r->flags & LUTC_REQ_HOST) != 0 || fake;
        int64_t dp = 0, dop = 0;
        request_staging(s, r->H, &dp, &dop);
        lutc_job& j = jobs[i];
        j.in.data = host ? reinterpret_cast<const uint16_t*>(256) : r->in;
        j.in.pitch_bytes = host ? dp : r->pitch;
        j.in.width = s.width;
        j.in.height = r->H;
        j.in.bands = s.bands;
        j.in.bits = s.bits;
        j.per_band = coefs[i].data();
        j.out = host ? reinterpret_cast<void*>(256) : r->out;
        j.out_pitch_bytes = host ? dop : r->out_pitch;
        j.flags = LUTC_STRETCH;
    }
    return lutc_batch_workspace(jobs.data(), (int)n);
}

int lutc_server_st::launch(Flight* f)
{
    const bool fake = cfg.fake_device != 0;
    const int n = (int)f->reqs.size();
    cudaStream_t st = fake ? nullptr : streams[f->slot];
    std::vector<std::vector<lutc_coeffs>> coefs(n);
    std::vector<lutc_job> jobs(n);
    for (int i = 0; i < n; ++i) {
        Request* r = f->reqs[i];
        const Sensor& s = *f->sensors[i];
        const int64_t plane = (int64_t)s.bands * s.width;
        coefs[i].resize(s.bands);
        for (int b = 0; b < s.bands; ++b) {
            const int32_t* base_c = reinterpret_cast<const int32_t*>(dev(s.off));
            coefs[i][b].A = base_c ? base_c + (int64_t)b * s.width : nullptr;
            coefs[i][b].G = base_c ? base_c + plane + (int64_t)b * s.width : nullptr;
            coefs[i][b].O = base_c ? base_c + 2 * plane + (int64_t)b * s.width : nullptr;
            coefs[i][b].ncols = s.width;
        }
        lutc_job& j = jobs[i];
        const bool host = (r->flags & LUTC_REQ_HOST) != 0;
        j.in.data = host ? reinterpret_cast<const uint16_t*>(dev(r->in_off)) : r->in;
        j.in.pitch_bytes = host ? r->dpitch : r->pitch;
        j.in.width = s.width;
        j.in.height = r->H;
        j.in.bands = s.bands;
        j.in.bits = s.bits;
        j.per_band = coefs[i].data();
        j.out = host ? dev(r->out_off) : r->out;
        j.out_pitch_bytes = host ? r->dopitch : r->out_pitch;
        j.flags = LUTC_STRETCH;
    }
    if (fake) {
        f->t_ready = now_s() + cfg.fake_latency_us * 1e-6;
        return LUTC_OK;
    }
    int rc;
    // A lone request takes the single-image fused path: no plan to build and copy to the device, its
    // tensor map in the kernel parameters, three kernels chained on the device.  Larger batches are
    // planned first: the plan's tables go to the device from host memory, a copy that waits for the
    // stream's earlier work, so it must not queue behind this batch's own copies in.
    if (n > 1) {
        const size_t need = lutc_batch_workspace(jobs.data(), n);
        if (need > f->ws_bytes) return LUTC_ENOMEM;
        const lutc_batch_config bc = {0, 0, 0};
        if ((rc = lutc_batch_create(jobs.data(), n, &bc, dev(f->ws_off), f->ws_bytes, (lutc_stream)st, &f->batch)))
            return rc;
    } else if (lutc_correct_image_workspace(&jobs[0].in) > f->ws_bytes) {
        return LUTC_ENOMEM;
    }
    for (int i = 0; i < n; ++i) {
        Request* r = f->reqs[i];
        if (!(r->flags & LUTC_REQ_HOST)) continue;
        const Sensor& s = *f->sensors[i];
        rc = r->sm_copy ? copy_rows(dev(r->in_off), r->dpitch, r->in, r->pitch, 2 * (int64_t)s.width,
                                    (int64_t)s.bands * r->H, st)
                        : cuda_status(cudaMemcpy2DAsync(dev(r->in_off), r->dpitch, r->in, r->pitch,
                                                        2 * (size_t)s.width, (size_t)s.bands * r->H,
                                                        cudaMemcpyHostToDevice, st));
        if (rc) return rc;
    }
    rc = n > 1 ? lutc_batch_run(f->batch, (lutc_stream)st)
               : lutc_correct_image(&jobs[0].in, jobs[0].per_band, jobs[0].flags, jobs[0].out, jobs[0].out_pitch_bytes,
                                    dev(f->ws_off), f->ws_bytes, (lutc_stream)st);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        Request* r = f->reqs[i];
        if (!(r->flags & LUTC_REQ_HOST)) continue;
        const Sensor& s = *f->sensors[i];
        rc = r->sm_copy ? copy_rows(r->out, r->out_pitch, dev(r->out_off), r->dopitch, (int64_t)s.width,
                                    (int64_t)s.bands * r->H, st)
                        : cuda_status(cudaMemcpy2DAsync(r->out, r->out_pitch, dev(r->out_off), r->dopitch,
                                                        (size_t)s.width, (size_t)s.bands * r->H,
                                                        cudaMemcpyDeviceToHost, st));
        if (rc) return rc;
    }
    return cuda_status(cudaEventRecord(events[f->slot], st));
}

void lutc_server_st::run_batcher()
{
    if (!cfg.fake_device) cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_batcher.wait(lk, [&] { return stop || !pending.empty(); });
        if (stop) return;
        // the batch window: full, the oldest request has waited max_wait_us, or nothing is on the
        // device (the completer wakes this thread when a batch finishes)
        const double deadline = pending.front()->t_submit + cfg.max_wait_us * 1e-6;
        while (!stop && (int)pending.size() < cfg.max_batch && (cfg.hold_when_idle || !flights.empty())) {
            const double left = deadline - now_s();
            if (left <= 0) break;
            cv_batcher.wait_for(lk, std::chrono::duration<double>(left));
        }
        if (stop) return;
        int slot = -1;
        cv_batcher.wait(lk, [&] {
            if (stop) return true;
            for (int s = 0; s < (int)slot_busy.size(); ++s)
                if (!slot_busy[s]) { slot = s; return true; }
            return false;
        });
        if (stop) return;
        if (pending.empty()) continue;  // every queued request was withdrawn meanwhile
        // admission: take requests in arrival order while their memory fits
        Flight* f = new Flight();
        std::vector<int> uploads;  // sensors first used by this batch
        while (!pending.empty() && (int)f->reqs.size() < cfg.max_batch) {
            Request* r = pending.front();
            Sensor& sn = sensors[r->sensor];
            const bool miss = !sn.cached && std::find(uploads.begin(), uploads.end(), r->sensor) == uploads.end();
            if (!reserve(r, sn, miss)) break;
            if (miss) {
                uploads.push_back(r->sensor);
                r->cache_miss = 1;
            }
            pending.pop_front();
            f->reqs.push_back(r);
        }
        // the batch's workspace; drop requests from the back until it fits
        size_t ws_need = 0;
        while (!f->reqs.empty()) {
            ws_need = exact_workspace(f->reqs);
            if (ws_need > 0 && arena.alloc(ws_need, &f->ws_off)) break;
            Request* r = f->reqs.back();
            f->reqs.pop_back();
            unreserve(r, uploads);
            pending.push_front(r);
        }
        if (f->reqs.empty()) {
            delete f;
            if (flights.empty()) {
                // nothing in flight will free memory: the head request can never fit
                Request* r = pending.front();
                pending.pop_front();
                r->status = LUTC_ENOMEM;
                r->done = true;
                r->t_done = now_s();
                cv_wait.notify_all();
            } else {
                cv_batcher.wait(lk);
            }
            continue;
        }
        for (Request* r : f->reqs) f->sensors.push_back(&sensors[r->sensor]);
        f->ws_bytes = ws_need;
        f->slot = slot;
        slot_busy[slot] = 1;
        const uint64_t number = ++batches;
        const int nreq = (int)f->reqs.size();
        largest = std::max(largest, nreq);
        const double t0 = now_s();
        for (Request* r : f->reqs) {
            r->t_start = t0;
            r->batch_size = nreq;
        }
        // outside the lock: first uploads of coefficients, then the batch
        std::vector<Sensor*> up;
        for (int sid : uploads) up.push_back(&sensors.find(sid)->second);
        lk.unlock();
        int rc = LUTC_OK;
        for (Sensor* sp : up) {
            Sensor& s = *sp;
            if (cfg.fake_device) continue;
            const size_t plane = (size_t)s.bands * s.width * 4;
            uint8_t* d = dev(s.off);
            if (!rc) rc = cuda_status(cudaMemcpyAsync(d, s.A.data(), plane, cudaMemcpyHostToDevice, upload));
            if (!rc) rc = cuda_status(cudaMemcpyAsync(d + plane, s.G.data(), plane, cudaMemcpyHostToDevice, upload));
            if (!rc) rc = cuda_status(cudaMemcpyAsync(d + 2 * plane, s.O.data(), plane, cudaMemcpyHostToDevice, upload));
        }
        if (!uploads.empty() && !cfg.fake_device && !rc) rc = cuda_status(cudaStreamSynchronize(upload));
        const int upload_rc = rc;
        if (!rc) rc = launch(f);
        if (cfg.fail_every > 0 && number % (uint64_t)cfg.fail_every == 0) rc = LUTC_ECUDA;  // injected on the host
        f->status = rc;
        if (rc && !cfg.fake_device) cudaGetLastError();
        const double t1 = now_s();
        lk.lock();
        for (Request* r : f->reqs) r->t_launched = t1;
        f->t_launched = t1;
        // an uploaded sensor stays cached even if its batch failed later; after a failed upload
        // (no kernel of this batch was launched) its memory is returned and the next request retries
        for (Sensor* sp : up) {
            sp->cached = upload_rc == LUTC_OK;
            if (upload_rc != LUTC_OK) arena.release(sp->off, coef_bytes(*sp));
        }
        flights.push_back(f);
        cv_done.notify_all();
    }
}

void lutc_server_st::finish(Flight* f)
{
    // called with the lock held
    const double t = now_s();
    for (Request* r : f->reqs) {
        if (r->flags & LUTC_REQ_HOST) {
            arena.release(r->in_off, r->in_bytes);
            arena.release(r->out_off, r->out_bytes);
        }
        r->status = f->status;
        r->t_done = t;
        r->done = true;
        ++completed;
    }
    arena.release(f->ws_off, f->ws_bytes);
    if (f->batch) lutc_batch_destroy(f->batch);
    slot_busy[f->slot] = 0;
    delete f;
}

void lutc_server_st::run_completer()
{
    if (!cfg.fake_device) cudaSetDevice(device);
#ifdef __linux__
    // this thread polls in short sleeps while batches run: with the default 50 us timer slack a 10 us
    // sleep lasts ~60 us, and that delay would land on every request's latency
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
    // within kSpinWindow of the newest launch the thread polls every ~2 us without sleeping (a lone
    // request's kernels take tens of microseconds: a 10 us sleep would add ~5 us to it on average);
    // later, and while nothing runs, it sleeps
    constexpr double kSpinWindow = 300e-6, kSpinPause = 2e-6;
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_done.wait(lk, [&] { return stop_completer || !flights.empty(); });
        if (flights.empty() && stop_completer) return;
        bool any = false;
        for (auto it = flights.begin(); it != flights.end();) {
            Flight* f = *it;
            bool ready;
            if (cfg.fake_device || f->status != LUTC_OK) {
                ready = !cfg.fake_device || now_s() >= f->t_ready;
                if (f->status != LUTC_OK && !cfg.fake_device) {
                    // a failed launch may still have work queued on its stream
                    ready = cudaEventQuery(events[f->slot]) != cudaErrorNotReady;
                    cudaGetLastError();
                    if (ready) cudaStreamSynchronize(streams[f->slot]);
                }
            } else {
                const cudaError_t e = cudaEventQuery(events[f->slot]);
                ready = e != cudaErrorNotReady;
                if (ready && e != cudaSuccess) {
                    f->status = LUTC_ECUDA;
                    cudaGetLastError();
                }
            }
            if (ready) {
                finish(f);
                it = flights.erase(it);
                any = true;
            } else {
                ++it;
            }
        }
        if (any) {
            cv_wait.notify_all();
            cv_batcher.notify_all();
        } else {
            double newest = 0;
            for (const Flight* f : flights) newest = std::max(newest, f->t_launched);
            const double t = now_s();
            lk.unlock();
            if (!cfg.fake_device && t - newest < kSpinWindow) {
                while (now_s() - t < kSpinPause) {
                }
            } else {
                std::this_thread::sleep_for(std::chrono::microseconds(10));
            }
            lk.lock();
        }
    }
}

extern "C" int lutc_server_create(const lutc_server_config* config, lutc_server* out)
{
    if (!out) return LUTC_EINVAL;
    lutc_server_config c = config ? *config : lutc_server_config{};
    if (c.budget_bytes == 0) c.budget_bytes = (size_t)40 << 30;
    if (c.max_batch <= 0) c.max_batch = 32;
    if (c.max_wait_us <= 0) c.max_wait_us = 2000;
    if (c.streams <= 0) c.streams = 3;
    if (c.max_queue <= 0) c.max_queue = 4096;
    if (c.max_batch > 4096 || c.streams > 64 || c.fake_latency_us < 0 || c.fail_every < 0 ||
        (c.hold_when_idle != 0 && c.hold_when_idle != 1))
        return LUTC_EINVAL;
    lutc_server s = new (std::nothrow) lutc_server_st();
    if (!s) return LUTC_ENOMEM;
    s->cfg = c;
    if (!c.fake_device) {
        if (cudaGetDevice(&s->device) != cudaSuccess || tma_preload() != LUTC_OK || tables_preload() != LUTC_OK ||
            cudaMalloc(&s->base, c.budget_bytes) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return LUTC_ENOMEM;
        }
        s->streams.resize(c.streams);
        s->events.resize(c.streams);
        bool ok = cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; i < c.streams && ok; ++i)
            ok = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (cudaStream_t st : s->streams) if (st) cudaStreamDestroy(st);
            for (cudaEvent_t e : s->events) if (e) cudaEventDestroy(e);
            if (s->upload) cudaStreamDestroy(s->upload);
            cudaFree(s->base);
            delete s;
            return LUTC_ECUDA;
        }
    }
    s->slot_busy.assign(c.streams, 0);
    s->arena.init(c.budget_bytes);
    s->batcher = std::thread([s] { s->run_batcher(); });
    s->completer = std::thread([s] { s->run_completer(); });
    *out = s;
    return LUTC_OK;
}

extern "C" int lutc_server_register_sensor(lutc_server s, int sensor_id, int width, int bands, int bits,
                                           const int32_t* A, const int32_t* G, const int32_t* O)
{
    if (!s || sensor_id < 0 || sensor_id > 65535 || width < 1 || bands < 1 || bands > LUTC_MAX_BANDS ||
        bits < LUTC_MIN_BITS || bits > LUTC_MAX_BITS || !A || !G || !O)
        return LUTC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->sensors.count(sensor_id)) return LUTC_EINVAL;
    Sensor& x = s->sensors[sensor_id];
    x.width = width;
    x.bands = bands;
    x.bits = bits;
    const size_t n = (size_t)bands * width;
    x.A.assign(A, A + n);
    x.G.assign(G, G + n);
    x.O.assign(O, O + n);
    return LUTC_OK;
}

extern "C" int lutc_server_submit(lutc_server s, int sensor_id, const uint16_t* raster, int height,
                                  int64_t pitch_bytes, uint8_t* out, int64_t out_pitch_bytes, int flags,
                                  uint64_t* ticket)
{
    if (!s || !ticket || height < 1 || (flags & ~LUTC_REQ_HOST)) return LUTC_EINVAL;
    // host buffers the kernels can address (page-locked memory) are copied by the SMs: a request's
    // short strided rows are slow for the copy engines
    const bool sm_copy = (flags & LUTC_REQ_HOST) && !s->cfg.fake_device && raster && out &&
                         device_can_access(raster) && device_can_access(out);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return LUTC_ESHUTDOWN;
    auto it = s->sensors.find(sensor_id);
    if (it == s->sensors.end()) return LUTC_EINVAL;
    const Sensor& x = it->second;
    if (!s->cfg.fake_device && (!raster || !out)) return LUTC_EINVAL;
    if (pitch_bytes < 2 * (int64_t)x.width || out_pitch_bytes < x.width) return LUTC_EINVAL;
    if ((int)s->pending.size() >= s->cfg.max_queue) return LUTC_EBUSY;
    int64_t dp, dop;
    const size_t alone = ((flags & LUTC_REQ_HOST) ? s->request_staging(x, height, &dp, &dop) : 0) +
                         (size_t)3 * x.bands * x.width * 4 + lutc_server_st::table_estimate(x) + 8192;
    if (alone > s->arena.size()) return LUTC_EBUSY;
    Request* r = new (std::nothrow) Request();
    if (!r) return LUTC_ENOMEM;
    r->ticket = s->next_ticket++;
    r->sensor = sensor_id;
    r->H = height;
    r->flags = flags;
    r->in = raster;
    r->pitch = pitch_bytes;
    r->out = out;
    r->out_pitch = out_pitch_bytes;
    r->sm_copy = sm_copy;
    r->t_submit = now_s();
    s->tickets[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
    s->cv_batcher.notify_all();
    return LUTC_OK;
}

extern "C" int lutc_server_wait(lutc_server s, uint64_t ticket, int64_t timeout_us, lutc_request_info* info)
{
    if (!s) return LUTC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return LUTC_EINVAL;
    Request* r = it->second;
    if (timeout_us < 0) {
        s->cv_wait.wait(lk, [&] { return r->done; });
    } else if (!s->cv_wait.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
        return LUTC_ETIMEOUT;
    }
    if (info) {
        info->status = r->status;
        info->batch_size = r->batch_size;
        info->submit_s = r->t_submit;
        info->start_s = r->t_start;
        info->launched_s = r->t_launched;
        info->done_s = r->t_done;
        info->cache_miss = r->cache_miss;
        info->pad = 0;
    }
    s->tickets.erase(it);
    delete r;
    return LUTC_OK;
}

extern "C" int lutc_server_cancel(lutc_server s, uint64_t ticket)
{
    if (!s) return LUTC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return LUTC_EINVAL;
    Request* r = it->second;
    // queued requests hold no reservation: admission reserves and dequeues under this lock
    auto q = std::find(s->pending.begin(), s->pending.end(), r);
    if (q == s->pending.end()) return LUTC_EBUSY;
    s->pending.erase(q);
    r->status = LUTC_ECANCELED;
    r->t_done = now_s();
    r->done = true;
    s->cv_wait.notify_all();
    s->cv_batcher.notify_all();
    return LUTC_OK;
}

extern "C" int lutc_server_stats(lutc_server s, uint64_t* completed, uint64_t* batches, size_t* budget_in_use,
                                 int32_t* largest_batch)
{
    if (!s) return LUTC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (batches) *batches = s->batches;
    if (budget_in_use) *budget_in_use = s->arena.used();
    if (largest_batch) *largest_batch = s->largest;
    return LUTC_OK;
}

extern "C" int lutc_server_destroy(lutc_server s)
{
    if (!s) return LUTC_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        const double t = now_s();
        for (Request* r : s->pending) {
            r->status = LUTC_ESHUTDOWN;
            r->done = true;
            r->t_done = t;
        }
        s->pending.clear();
        s->cv_batcher.notify_all();
        s->cv_wait.notify_all();
    }
    s->batcher.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop_completer = true;
        s->cv_done.notify_all();
    }
    s->completer.join();
    for (auto& kv : s->tickets) delete kv.second;
    if (!s->cfg.fake_device) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        for (cudaEvent_t e : s->events) cudaEventDestroy(e);
        if (s->upload) cudaStreamDestroy(s->upload);
        cudaFree(s->base);
    }
    delete s;
    return LUTC_OK;
}
