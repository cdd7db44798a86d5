// The paper's client-server transport (Section II, Fig. 3) over the C ABI: a
// TCP server that receives a task header and its data, runs the task on the
// GPU through lutc_submit and sends the result back.
//
// A request is the 260-byte header of Fig. 3 -- task flag (29 bytes, the task
// name, NUL-padded), a '+' separator, the parameter list (200 bytes, as for
// lutc_submit) and the output name (30 bytes) -- followed by the payload's
// length (uint64, little endian) and the payload: the task's inputs packed
// back to back in the order lutc_submit takes them, every raster with packed
// rows.  The reply is the status (int32), the output name echoed (30 bytes),
// the result's length (uint64) and the result: the task's outputs packed back
// to back.  A connection carries any number of requests; each connection is
// served by its own thread and CUDA stream.
#include <arpa/inet.h>
#include <netinet/in.h>
#include <netinet/tcp.h>
#include <poll.h>
#include <stdint.h>
#include <string.h>
#include <sys/socket.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lutc_internal.cuh"

namespace lutc {
namespace {

constexpr size_t kFlagBytes = 29, kParamBytes = 200, kNameBytes = 30;
constexpr size_t kHeaderBytes = kFlagBytes + 1 + kParamBytes + kNameBytes;  // 260
constexpr uint64_t kMaxPayload = 64ull << 30;

bool read_all(int fd, void* buf, size_t n)
{
    uint8_t* p = reinterpret_cast<uint8_t*>(buf);
    while (n > 0) {
        const ssize_t r = recv(fd, p, n, 0);
        if (r <= 0) return false;
        p += r;
        n -= (size_t)r;
    }
    return true;
}

bool write_all(int fd, const void* buf, size_t n)
{
    const uint8_t* p = reinterpret_cast<const uint8_t*>(buf);
    while (n > 0) {
        const ssize_t r = send(fd, p, n, MSG_NOSIGNAL);
        if (r <= 0) return false;
        p += r;
        n -= (size_t)r;
    }
    return true;
}

bool discard(int fd, uint64_t n)
{
    uint8_t buf[65536];
    while (n > 0) {
        const size_t k = n < sizeof(buf) ? (size_t)n : sizeof(buf);
        if (!read_all(fd, buf, k)) return false;
        n -= k;
    }
    return true;
}

int task_of(const std::string& name)
{
    static const struct { const char* name; int task; } kTasks[] = {
        {"lutgen", LUTC_TASK_LUTGEN},           {"hist", LUTC_TASK_HIST},
        {"stretch", LUTC_TASK_STRETCH},         {"compose", LUTC_TASK_COMPOSE},
        {"apply", LUTC_TASK_APPLY},             {"correct_image", LUTC_TASK_CORRECT_IMAGE},
        {"device_info", LUTC_TASK_DEVICE_INFO}, {"demosaic", LUTC_TASK_DEMOSAIC},
        {"fit", LUTC_TASK_FIT},
    };
    for (const auto& t : kTasks)
        if (name == t.name) return t.task;
    return -1;
}

// Packed byte sizes of a task's inputs and outputs; false if the parameters do not describe one.
bool io_sizes(int task, const TaskParams& p, uint64_t payload, std::vector<uint64_t>& in, std::vector<uint64_t>& out)
{
    const bool wok = p.width >= 0 && p.width <= INT32_MAX, hok = p.height >= 0 && p.height <= INT32_MAX;
    const bool dims = wok && hok && p.bands >= 1 && p.bands <= LUTC_MAX_BANDS;
    const bool bits = p.bits >= LUTC_MIN_BITS && p.bits <= LUTC_MAX_BITS;
    const uint64_t W = (uint64_t)std::max<int64_t>(p.width, 0), H = (uint64_t)std::max<int64_t>(p.height, 0),
                   B = (uint64_t)p.bands, L = bits ? (uint64_t)1 << p.bits : 0;
    const uint64_t px = B * H * W;
    switch (task) {
    case LUTC_TASK_LUTGEN:
        if (!wok || !bits) return false;
        in = {4 * W, 4 * W, 4 * W};
        out = {2 * W * L};
        return true;
    case LUTC_TASK_HIST:
        if (!dims || !bits) return false;
        in = {2 * px, 4 * B * W, 4 * B * W, 4 * B * W};
        out = {8 * B * L};
        return true;
    case LUTC_TASK_STRETCH:
        if (!bits || p.bands < 1 || p.bands > LUTC_MAX_BANDS) return false;
        in = {8 * B * L};
        out = {B * L, 8 * B};
        return true;
    case LUTC_TASK_COMPOSE:
        if (!wok || !bits) return false;
        in = {2 * W * L, L};
        out = {W * L};
        return true;
    case LUTC_TASK_APPLY:
        if (!dims || !bits || p.table == 0) return false;
        in = {2 * px, (p.table == 1 ? 2 : 1) * B * W * L};
        out = {(p.table == 1 ? 2 : 1) * px};
        return true;
    case LUTC_TASK_CORRECT_IMAGE:
        if (!dims || !bits) return false;
        in = {2 * px, 4 * B * W, 4 * B * W, 4 * B * W};
        out = {(p.stretch ? 1 : 2) * px};
        return true;
    case LUTC_TASK_DEMOSAIC:
        if (!dims || !bits || p.bands != 1) return false;
        // the coefficients are optional: the payload's length says whether they came
        in = {2 * H * W};
        if (payload == 2 * H * W + 12 * W) in = {2 * H * W, 4 * W, 4 * W, 4 * W};
        out = {6 * H * W};
        return true;
    case LUTC_TASK_FIT:
        if (!wok || !hok || p.order < 1 || p.order > LUTC_FIT_MAX_ORDER) return false;
        in = {2 * H * W, p.targets ? 8 * H * W : 8 * H};
        out = {8 * W * (uint64_t)(p.order + 1), 4 * W};
        return true;
    case LUTC_TASK_DEVICE_INFO:
        in = {};
        out = {};
        return true;
    default:
        return false;
    }
}

struct DeviceBuffers {
    std::vector<void*> ptrs;
    ~DeviceBuffers()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    void* add(uint64_t bytes)
    {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 256) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return p;
    }
};

// Runs one request; fills `result` (outputs packed back to back).
int run_task(int task, const char* params, const TaskParams& p, const std::vector<uint8_t>& payload,
             const std::vector<uint64_t>& in_sizes, const std::vector<uint64_t>& out_sizes, cudaStream_t st,
             std::vector<uint8_t>& result)
{
    if (task == LUTC_TASK_DEVICE_INFO) {
        size_t need = 0;
        lutc_device_info(nullptr, 0, &need);
        result.assign(need, 0);
        const int rc = lutc_device_info(reinterpret_cast<char*>(result.data()), need, nullptr);
        if (rc == LUTC_OK) result.resize(need - 1);  // without the terminating NUL
        return rc;
    }
    DeviceBuffers bufs;
    std::vector<const void*> ins;
    std::vector<void*> outs;
    uint64_t off = 0;
    for (uint64_t n : in_sizes) {
        void* d = bufs.add(n);
        if (!d) return LUTC_ECUDA;
        if (n && cudaMemcpyAsync(d, payload.data() + off, n, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return LUTC_ECUDA;
        ins.push_back(d);
        off += n;
    }
    uint64_t total = 0;
    for (uint64_t n : out_sizes) {
        void* d = bufs.add(n);
        if (!d) return LUTC_ECUDA;
        outs.push_back(d);
        total += n;
    }
    void* ws = nullptr;
    size_t ws_bytes = 0;
    if (task == LUTC_TASK_CORRECT_IMAGE && p.stretch) {
        const lutc_raster r = raster_of(p, ins[0]);
        ws_bytes = lutc_correct_image_workspace(&r);
        if (!(ws = bufs.add(ws_bytes))) return LUTC_ECUDA;
    }
    int rc = lutc_submit(task, params, ins.data(), (int)ins.size(), outs.data(), (int)outs.size(), ws, ws_bytes,
                         (lutc_stream)st);
    if (rc) return rc;
    result.assign(total, 0);
    off = 0;
    for (size_t k = 0; k < outs.size(); ++k) {
        if (out_sizes[k] &&
            cudaMemcpyAsync(result.data() + off, outs[k], out_sizes[k], cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return LUTC_ECUDA;
        off += out_sizes[k];
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return LUTC_ECUDA;
    }
    return LUTC_OK;
}

}  // namespace
}  // namespace lutc

using namespace lutc;

struct lutc_net_server {
    int listen_fd = -1;
    int port = 0;
    int device = 0;
    std::atomic<bool> stop{false};
    std::thread acceptor;
    std::mutex mu;
    std::vector<std::thread> workers;
    std::vector<int> conns;
    std::atomic<uint64_t> requests{0}, failures{0};

    void serve(int fd)
    {
        cudaStream_t st = nullptr;
        const bool gpu = cudaSetDevice(device) == cudaSuccess &&
                         cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (!gpu) cudaGetLastError();
        for (;;) {
            uint8_t header[kHeaderBytes];
            uint64_t len = 0;
            if (!read_all(fd, header, sizeof(header)) || !read_all(fd, &len, sizeof(len))) break;
            const std::string flag(reinterpret_cast<char*>(header), strnlen(reinterpret_cast<char*>(header), kFlagBytes));
            char params[kParamBytes + 1] = {0};
            memcpy(params, header + kFlagBytes + 1, kParamBytes);
            char name[kNameBytes];
            memcpy(name, header + kFlagBytes + 1 + kParamBytes, kNameBytes);
            int rc = LUTC_OK;
            std::vector<uint8_t> result;
            const int task = task_of(flag);
            TaskParams p;
            std::vector<uint64_t> in_sizes, out_sizes;
            uint64_t expect = 0;
            if (header[kFlagBytes] != '+' || task < 0 || parse_task_params(params, p) != LUTC_OK ||
                !io_sizes(task, p, len, in_sizes, out_sizes))
                rc = LUTC_EINVAL;
            for (uint64_t n : in_sizes) expect += n;
            if (rc == LUTC_OK && len != expect) rc = LUTC_EINVAL;
            if (len > kMaxPayload) {
                failures++;
                break;  // cannot resynchronise on an absurd length: drop the connection
            }
            if (rc != LUTC_OK) {
                if (!discard(fd, len)) break;
            } else {
                std::vector<uint8_t> payload(len);
                if (len && !read_all(fd, payload.data(), len)) break;
                rc = (gpu || task == LUTC_TASK_DEVICE_INFO)
                         ? run_task(task, params, p, payload, in_sizes, out_sizes, st, result)
                         : LUTC_ECUDA;
            }
            requests++;
            if (rc != LUTC_OK) {
                failures++;
                result.clear();
            }
            const int32_t status = rc;
            const uint64_t n = result.size();
            if (!write_all(fd, &status, sizeof(status)) || !write_all(fd, name, kNameBytes) ||
                !write_all(fd, &n, sizeof(n)) || (n && !write_all(fd, result.data(), n)))
                break;
        }
        if (st) cudaStreamDestroy(st);
        close_conn(fd);
    }

    void close_conn(int fd)
    {
        std::lock_guard<std::mutex> lock(mu);
        for (size_t i = 0; i < conns.size(); ++i)
            if (conns[i] == fd) {
                conns.erase(conns.begin() + (long)i);
                close(fd);
                return;
            }
    }

    void accept_loop()
    {
        while (!stop) {
            pollfd pf = {listen_fd, POLLIN, 0};
            if (poll(&pf, 1, 100) <= 0) continue;
            const int fd = accept(listen_fd, nullptr, nullptr);
            if (fd < 0) continue;
            const int one = 1;
            setsockopt(fd, IPPROTO_TCP, TCP_NODELAY, &one, sizeof(one));
            std::lock_guard<std::mutex> lock(mu);
            if (stop) {
                close(fd);
                break;
            }
            conns.push_back(fd);
            workers.emplace_back([this, fd] { serve(fd); });
        }
    }
};

extern "C" int lutc_net_server_create(const char* address, int port, int device, lutc_net_server** out)
{
    if (!out || port < 0 || port > 65535 || device < 0) return LUTC_EINVAL;
    *out = nullptr;
    sockaddr_in sa;
    memset(&sa, 0, sizeof(sa));
    sa.sin_family = AF_INET;
    sa.sin_port = htons((uint16_t)port);
    if (inet_pton(AF_INET, address ? address : "127.0.0.1", &sa.sin_addr) != 1) return LUTC_EINVAL;
    const int fd = socket(AF_INET, SOCK_STREAM, 0);
    if (fd < 0) return LUTC_EBUSY;
    const int one = 1;
    setsockopt(fd, SOL_SOCKET, SO_REUSEADDR, &one, sizeof(one));
    if (bind(fd, reinterpret_cast<sockaddr*>(&sa), sizeof(sa)) != 0 || listen(fd, 64) != 0) {
        close(fd);
        return LUTC_EBUSY;
    }
    socklen_t sl = sizeof(sa);
    getsockname(fd, reinterpret_cast<sockaddr*>(&sa), &sl);
    lutc_net_server* s = new (std::nothrow) lutc_net_server;
    if (!s) {
        close(fd);
        return LUTC_ENOMEM;
    }
    s->listen_fd = fd;
    s->port = ntohs(sa.sin_port);
    s->device = device;
    s->acceptor = std::thread([s] { s->accept_loop(); });
    *out = s;
    return LUTC_OK;
}

extern "C" int lutc_net_server_port(const lutc_net_server* s) { return s ? s->port : LUTC_EINVAL; }

extern "C" int lutc_net_server_stats(const lutc_net_server* s, uint64_t* requests, uint64_t* failures)
{
    if (!s) return LUTC_EINVAL;
    if (requests) *requests = s->requests;
    if (failures) *failures = s->failures;
    return LUTC_OK;
}

extern "C" int lutc_net_server_destroy(lutc_net_server* s)
{
    if (!s) return LUTC_EINVAL;
    s->stop = true;
    if (s->acceptor.joinable()) s->acceptor.join();
    close(s->listen_fd);
    std::vector<std::thread> workers;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (int fd : s->conns) shutdown(fd, SHUT_RDWR);  // wakes workers blocked in recv
        workers.swap(s->workers);
    }
    for (auto& t : workers)
        if (t.joinable()) t.join();
    delete s;
    return LUTC_OK;
}
