// The fused correction of a raster in host memory: copies in, both passes and
// copies out pipelined in one call (the paper's client ships its data to the
// GPU server and gets the corrected image back, Section II; its future work
// names the host-device transfer as the cost to cut).
//
// On GB300 the host is reached over NVLink-C2C; copy engines run both
// directions at once and overlap with the kernels.  The raster is cut into
// chunks of rows per band:
//
//   copy-in stream   H2D chunk (b, c) ............................
//   caller's stream      pass 1 (b, c)  [after the last chunk of b: scan b]  pass 2 (b, c) ...
//   copy-out stream                                                              D2H chunk (b, c)
//
// Band b+1's copies in and pass 1 overlap band b's pass 2 and copies out, so
// a call costs about the larger of its two copy directions plus one band's
// drain.  The device keeps a full copy of the raster (pass 2 re-reads it)
// and stages the output, both in the caller's workspace.  A sequence of
// frames (lutc_correct_frames_host) alternates two workspace halves, so a
// frame's copies in also overlap the previous frame's drain.
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "lutc_internal.cuh"

namespace lutc {
namespace {

constexpr int kMaxDevices = 64;
constexpr int kEvents = 1024;                 // reused round-robin: each is waited on right after its record
constexpr size_t kChunkBytes = 48u << 20;     // target input bytes per chunk

struct HostPipe {
    std::mutex mu;
    bool ready = false;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev[kEvents];
    int next = 0;
    // a workspace half's last read of its raster copy / last copy out of its staged output: recorded at
    // the end of frame f, waited on at the start of frame f + 2 (dedicated: many pool events pass between)
    cudaEvent_t raw_free[2], out_free[2];
};
HostPipe g_pipes[kMaxDevices];

// call with g_pipes[dev].mu held
int pipe_init(int dev, HostPipe** out)
{
    HostPipe& p = g_pipes[dev];
    if (!p.ready) {
        if (cudaStreamCreateWithFlags(&p.h2d, cudaStreamNonBlocking) != cudaSuccess) return LUTC_ECUDA;
        if (cudaStreamCreateWithFlags(&p.d2h, cudaStreamNonBlocking) != cudaSuccess) return LUTC_ECUDA;
        for (int i = 0; i < kEvents; ++i)
            if (cudaEventCreateWithFlags(&p.ev[i], cudaEventDisableTiming) != cudaSuccess) return LUTC_ECUDA;
        for (int h = 0; h < 2; ++h)
            if (cudaEventCreateWithFlags(&p.raw_free[h], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&p.out_free[h], cudaEventDisableTiming) != cudaSuccess)
                return LUTC_ECUDA;
        p.ready = true;
    }
    *out = &p;
    return LUTC_OK;
}

struct HostLayout {
    size_t tables, raw, out, total;
    int64_t raw_pitch, out_pitch;
};

HostLayout host_layout(const lutc_raster* in, bool stretch)
{
    HostLayout l;
    const int64_t rows = (int64_t)in->bands * in->height;
    l.raw_pitch = (int64_t)align_up(2 * (size_t)in->width, 16);
    l.out_pitch = (int64_t)align_up((stretch ? 1 : 2) * (size_t)in->width, 16);
    lutc_raster dev = *in;
    dev.pitch_bytes = l.raw_pitch;
    l.tables = stretch ? align_up(tables_bytes(&dev), 256) : 0;
    l.raw = l.tables;
    l.out = align_up(l.raw + (size_t)rows * l.raw_pitch, 256);
    l.total = align_up(l.out + (size_t)rows * l.out_pitch, 256);
    return l;
}

// Runs frames[0..n) (same shape, pitch and coefficients; inputs hin[f], outputs hout[f] in host
// memory).  Frame f uses workspace half f % 2: its copies in wait only for frame f-2's last reads
// of that half's raster copy, so they overlap frame f-1's pass 2 and copies out.
int run_frames(const lutc_raster* in, const uint8_t* const* hin, int n, const lutc_coeffs* per_band, int flags,
               uint8_t* const* hout, int64_t out_pitch_bytes, uint8_t* ws, cudaStream_t st)
{
    const bool stretch = (flags & LUTC_STRETCH) != 0;
    const int64_t elem = stretch ? 1 : 2;
    const HostLayout l = host_layout(in, stretch);
    const int W = in->width, H = in->height, bands = in->bands;
    const int64_t L = (int64_t)1 << in->bits;

    // rows per chunk: about kChunkBytes of input
    const int64_t rows = std::max<int64_t>(1, (int64_t)(kChunkBytes / (size_t)std::max<int64_t>(l.raw_pitch, 1)));
    const int64_t chunks = (H + rows - 1) / rows;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LUTC_ECUDA;
    HostPipe* p = nullptr;
    std::lock_guard<std::mutex> lock(g_pipes[dev].mu);  // one enqueue at a time per device: events are reused
    int rc = pipe_init(dev, &p);
    if (rc) return rc;
    // every wait is enqueued right after the record it waits for, so reusing the pool round-robin is safe
    auto ev = [&]() { cudaEvent_t e = p->ev[p->next]; p->next = (p->next + 1) % kEvents; return e; };
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };

    // Rows packed on both sides: one linear copy per chunk.  Strided rows: the SMs copy them when the
    // host buffer is device-addressable (the copy engines move short strided rows slowly), else a 2-D copy.
    // (packed: no gap between rows on either side, so a linear copy touches exactly the rows' bytes)
    const bool in_packed = in->pitch_bytes == 2 * (int64_t)W && l.raw_pitch == 2 * (int64_t)W;
    const bool out_packed = out_pitch_bytes == elem * W && l.out_pitch == elem * W;
    const bool in_sm = !in_packed && device_can_access(hin[0]), out_sm = !out_packed && device_can_access(hout[0]);
    auto copy_in = [&](void* dst, const uint8_t* src, int64_t nr) {
        if (in_packed) return ok(cudaMemcpyAsync(dst, src, (size_t)nr * l.raw_pitch, cudaMemcpyDefault, p->h2d));
        if (in_sm) return copy_rows(dst, l.raw_pitch, src, in->pitch_bytes, 2 * (int64_t)W, nr, p->h2d) == LUTC_OK;
        return ok(cudaMemcpy2DAsync(dst, l.raw_pitch, src, in->pitch_bytes, 2 * (size_t)W, (size_t)nr,
                                    cudaMemcpyDefault, p->h2d));
    };
    auto copy_out = [&](uint8_t* dst, const uint8_t* src, int64_t nr) {
        if (out_packed) return ok(cudaMemcpyAsync(dst, src, (size_t)nr * l.out_pitch, cudaMemcpyDefault, p->d2h));
        if (out_sm) return copy_rows(dst, out_pitch_bytes, src, l.out_pitch, elem * (int64_t)W, nr, p->d2h) == LUTC_OK;
        return ok(cudaMemcpy2DAsync(dst, out_pitch_bytes, src, l.out_pitch, elem * (size_t)W, (size_t)nr,
                                    cudaMemcpyDefault, p->d2h));
    };

    // the copy streams start after the caller's earlier work (inputs may be produced there, the
    // workspace may still be in use)
    cudaEvent_t start = ev();
    bool good = ok(cudaEventRecord(start, st)) && ok(cudaStreamWaitEvent(p->h2d, start, 0)) &&
                ok(cudaStreamWaitEvent(p->d2h, start, 0));
    bool used[2] = {false, false};  // a workspace half has a frame of this call behind it
    for (int f = 0; good && f < n; ++f) {
        const int h = f & 1;
        uint8_t* half = ws + (size_t)h * l.total;
        uint8_t* raw = half + l.raw;
        uint8_t* dout = half + l.out;
        lutc_raster dev_all = *in;
        dev_all.data = reinterpret_cast<const uint16_t*>(raw);
        dev_all.pitch_bytes = l.raw_pitch;
        size_t ho = 0, so = 0, lo = 0;
        if (stretch) tables_offsets(&dev_all, &ho, &so, &lo);
        unsigned long long* hist = reinterpret_cast<unsigned long long*>(half + ho);
        uint8_t* S = half + so;
        int32_t* lohi = reinterpret_cast<int32_t*>(half + lo);
        if (used[h]) good = ok(cudaStreamWaitEvent(p->h2d, p->raw_free[h], 0));
        if (good && stretch) good = ok(cudaMemsetAsync(hist, 0, (size_t)bands * L * 8, st));
        bool waited_out = false;
        for (int b = 0; good && b < bands; ++b) {
            lutc_raster band = dev_all;
            band.bands = 1;
            const lutc_coeffs* cb = per_band + b;
            auto chunk = [&](int64_t c, lutc_raster* r, int64_t* r0, int64_t* nr) {
                *r0 = c * rows;
                *nr = std::min<int64_t>(rows, H - *r0);
                *r = band;
                r->data = reinterpret_cast<const uint16_t*>(raw + ((int64_t)b * H + *r0) * l.raw_pitch);
                r->height = (int32_t)*nr;
            };
            for (int64_t c = 0; good && c < chunks; ++c) {
                lutc_raster r;
                int64_t r0, nr;
                chunk(c, &r, &r0, &nr);
                cudaEvent_t in_done = ev();
                good = copy_in(const_cast<uint16_t*>(r.data), hin[f] + ((int64_t)b * H + r0) * in->pitch_bytes, nr) &&
                       ok(cudaEventRecord(in_done, p->h2d)) && ok(cudaStreamWaitEvent(st, in_done, 0));
                if (good && stretch) good = pass1_accumulate(&r, cb, hist + b * L, st) == LUTC_OK;
            }
            if (good && stretch)
                good = launch_stretch(hist + b * L, 1, in->bits, S + b * L, lohi + 2 * b, st) == LUTC_OK;
            if (good && !waited_out && used[h]) good = ok(cudaStreamWaitEvent(st, p->out_free[h], 0));
            waited_out = true;
            for (int64_t c = 0; good && c < chunks; ++c) {
                lutc_raster r;
                int64_t r0, nr;
                chunk(c, &r, &r0, &nr);
                uint8_t* o = dout + ((int64_t)b * H + r0) * l.out_pitch;
                cudaEvent_t out_ready = ev();
                good = pass2(&r, cb, stretch ? S + b * L : nullptr, o, l.out_pitch, stretch, st) == LUTC_OK &&
                       ok(cudaEventRecord(out_ready, st)) && ok(cudaStreamWaitEvent(p->d2h, out_ready, 0)) &&
                       copy_out(hout[f] + ((int64_t)b * H + r0) * out_pitch_bytes, o, nr);
            }
        }
        if (good) {
            good = ok(cudaEventRecord(p->raw_free[h], st)) && ok(cudaEventRecord(p->out_free[h], p->d2h));
            used[h] = true;
        }
    }
    // the caller's stream continues after the last copy out (also after a failure part way)
    cudaEvent_t done_in = ev(), done_out = ev();
    const bool joined = ok(cudaEventRecord(done_in, p->h2d)) && ok(cudaEventRecord(done_out, p->d2h)) &&
                        ok(cudaStreamWaitEvent(st, done_in, 0)) && ok(cudaStreamWaitEvent(st, done_out, 0));
    if (!good || !joined) {
        cudaGetLastError();
        return LUTC_ECUDA;
    }
    return LUTC_OK;
}

int check_host_call(const lutc_raster* in, const lutc_coeffs* per_band, int flags, int64_t out_pitch_bytes)
{
    int rc = check_raster(in);
    if (rc) return rc;
    if ((rc = check_coeff_set(in, per_band))) return rc;
    if (flags & ~LUTC_STRETCH) return LUTC_EINVAL;
    const int64_t elem = (flags & LUTC_STRETCH) ? 1 : 2;
    if ((int64_t)in->width * in->height > 0 && (out_pitch_bytes < elem * in->width || out_pitch_bytes % elem))
        return LUTC_EINVAL;
    return LUTC_OK;
}

}  // namespace
}  // namespace lutc

using namespace lutc;

extern "C" size_t lutc_correct_image_host_workspace(const lutc_raster* in, int flags)
{
    if (check_raster(in) || (flags & ~LUTC_STRETCH)) return 0;
    return host_layout(in, (flags & LUTC_STRETCH) != 0).total;
}

extern "C" int lutc_correct_image_host(const lutc_raster* in, const lutc_coeffs* per_band, int flags, void* out,
                                       int64_t out_pitch_bytes, void* workspace, size_t workspace_bytes,
                                       lutc_stream stream)
{
    int rc = check_host_call(in, per_band, flags, out_pitch_bytes);
    if (rc) return rc;
    if ((int64_t)in->width * in->height == 0) return LUTC_OK;
    if (!out) return LUTC_EINVAL;
    if (!workspace || workspace_bytes < host_layout(in, (flags & LUTC_STRETCH) != 0).total) return LUTC_ENOMEM;
    if ((uintptr_t)workspace % 256) return LUTC_EINVAL;
    const uint8_t* hin = reinterpret_cast<const uint8_t*>(in->data);
    uint8_t* hout = reinterpret_cast<uint8_t*>(out);
    return run_frames(in, &hin, 1, per_band, flags, &hout, out_pitch_bytes, reinterpret_cast<uint8_t*>(workspace),
                      (cudaStream_t)stream);
}

extern "C" size_t lutc_correct_frames_host_workspace(const lutc_raster* in, int flags, int frames)
{
    if (frames < 1) return 0;
    return lutc_correct_image_host_workspace(in, flags) * (frames > 1 ? 2 : 1);
}

extern "C" int lutc_correct_frames_host(const lutc_raster* in, const void* const* frames, int n,
                                        const lutc_coeffs* per_band, int flags, void* const* outs,
                                        int64_t out_pitch_bytes, void* workspace, size_t workspace_bytes,
                                        lutc_stream stream)
{
    int rc = check_host_call(in, per_band, flags, out_pitch_bytes);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!frames || !outs))) return LUTC_EINVAL;
    if (n == 0 || (int64_t)in->width * in->height == 0) return LUTC_OK;
    for (int f = 0; f < n; ++f)
        if (!frames[f] || !outs[f] || ((uintptr_t)frames[f] & 1)) return LUTC_EINVAL;
    if (!workspace || workspace_bytes < lutc_correct_frames_host_workspace(in, flags, n)) return LUTC_ENOMEM;
    if ((uintptr_t)workspace % 256) return LUTC_EINVAL;
    return run_frames(in, reinterpret_cast<const uint8_t* const*>(frames), n, per_band, flags,
                      reinterpret_cast<uint8_t* const*>(outs), out_pitch_bytes, reinterpret_cast<uint8_t*>(workspace),
                      (cudaStream_t)stream);
}
