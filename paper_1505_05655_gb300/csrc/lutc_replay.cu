// Open-loop replay of a request schedule against the serving loop (lutc_server_replay).
//
// The paper's server answers requests from clients that do not wait for one
// another (Sections I-II).  Measuring such a server's latency at a given load
// needs a load generator that keeps its own schedule: each request is handed
// over at the time drawn for it, whatever the collecting side is doing, and
// the latency is counted from that scheduled time, so that a late hand-over
// shows up as the generator's lateness (submit_s - scheduled) and never
// hides inside the server's figure.  Here one native thread submits on
// schedule (it sleeps until ~2 ms before a request is due, then spins) and
// the calling thread collects the tickets in order; no interpreter lock or
// garbage collector of the caller sits between the two.  Host code only.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <thread>

#include "lutc_internal.cuh"

namespace {

double steady_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr double kSpinWindow = 2e-3;       // spin, rather than sleep, this close to a due time (a sleep on a
                                           // busy host can end a millisecond or more late)
constexpr double kBusyRetry = 20e-6;       // a queue-full refusal (closed bursts) is retried this often
constexpr double kGiveUp = 120.0;          // longest a submit may keep being refused, or a ticket may run
constexpr int64_t kWaitSliceUs = 1000000;  // one lutc_server_wait call (re-issued until kGiveUp)
constexpr double kMaxSchedule = 3600.0;    // latest arrival time accepted

}  // namespace

extern "C" int lutc_server_replay(lutc_server server, const lutc_replay_request* req, int n, lutc_request_info* info,
                                  double* scheduled_s)
{
    if (!server || n < 0 || (n > 0 && (!req || !info))) return LUTC_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!(req[i].at_s >= 0.0 && req[i].at_s <= kMaxSchedule) || (i > 0 && req[i].at_s < req[i - 1].at_s))
            return LUTC_EINVAL;
    if (n == 0) return LUTC_OK;

    std::unique_ptr<uint64_t[]> tickets(new (std::nothrow) uint64_t[n]);
    if (!tickets) return LUTC_ENOMEM;
    std::atomic<int> submitted{0};  // requests 0 .. submitted-1 hold a ticket
    std::atomic<int> failed{0};     // the submit error that stopped the schedule, or 0
    const double t0 = steady_s() + 1e-3;

    std::thread submitter([&] {
        for (int i = 0; i < n; ++i) {
            const double due = t0 + req[i].at_s;
            for (;;) {
                if (failed.load(std::memory_order_acquire)) return;  // the collector gave up
                const double left = due - steady_s();
                if (left <= 0.0) break;
                if (left > kSpinWindow)
                    std::this_thread::sleep_for(std::chrono::duration<double>(std::min(left - kSpinWindow, 0.01)));
            }
            const lutc_replay_request& r = req[i];
            const double refused_since = steady_s();
            int rc;
            while ((rc = lutc_server_submit(server, r.sensor_id, r.raster, r.height, r.pitch_bytes, r.out,
                                            r.out_pitch_bytes, r.flags, &tickets[i])) == LUTC_EBUSY &&
                   steady_s() - refused_since < kGiveUp)
                std::this_thread::sleep_for(std::chrono::duration<double>(kBusyRetry));
            if (rc != LUTC_OK) {
                failed.store(rc == LUTC_EBUSY ? LUTC_ETIMEOUT : rc, std::memory_order_release);
                return;
            }
            submitted.store(i + 1, std::memory_order_release);
        }
    });

    int rc = LUTC_OK;
    for (int i = 0; i < n; ++i) {
        // the ticket of request i exists once the submitter got past it (or it stopped)
        while (submitted.load(std::memory_order_acquire) <= i && !failed.load(std::memory_order_acquire))
            std::this_thread::sleep_for(std::chrono::microseconds(10));
        if (submitted.load(std::memory_order_acquire) <= i) {
            rc = failed.load();
            for (int k = i; k < n; ++k) {
                info[k] = lutc_request_info{};
                info[k].status = rc;
            }
            break;
        }
        const double since = steady_s();
        int w;
        while ((w = lutc_server_wait(server, tickets[i], kWaitSliceUs, &info[i])) == LUTC_ETIMEOUT &&
               steady_s() - since < kGiveUp) {
        }
        if (w != LUTC_OK) {
            rc = w;
            for (int k = i; k < n; ++k) {
                info[k] = lutc_request_info{};
                info[k].status = w;
            }
            break;
        }
        if (scheduled_s) scheduled_s[i] = t0 + req[i].at_s;
    }
    if (rc != LUTC_OK) failed.store(rc);  // a stuck wait also stops the schedule
    submitter.join();
    return rc;
}
