// The paper's task interface (lutc_submit) and GPU-information utility (lutc_device_info).
//
// Section II of the paper has a client fill a header with a task flag, a
// comma-separated parameter string of at most 200 bytes and an output name,
// followed by the data; the server picks the task from the flag.  Here the
// flag is an enum, the parameter string keeps its format, and the data and
// outputs are pointer arrays.  Section IV lists the device properties its
// GPU-information utility reports as an XML tree; lutc_device_info writes the
// same list.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "lutc_internal.cuh"

namespace lutc {

// "key=value,key=value": every key known, every value a non-negative decimal (or u16/u8 for table)
int parse_task_params(const char* text, TaskParams& p)
{
    if (!text) return LUTC_EINVAL;
    const size_t len = strnlen(text, LUTC_PARAMS_MAX + 1);
    if (len > LUTC_PARAMS_MAX) return LUTC_EINVAL;
    std::string s(text, len);
    size_t at = 0;
    while (at < s.size()) {
        size_t end = s.find(',', at);
        if (end == std::string::npos) end = s.size();
        const std::string item = s.substr(at, end - at);
        at = end + 1;
        const size_t eq = item.find('=');
        if (eq == std::string::npos || eq == 0 || eq + 1 >= item.size()) return LUTC_EINVAL;
        const std::string key = item.substr(0, eq), val = item.substr(eq + 1);
        if (key == "targets") {
            if (val == "line") p.targets = 0;
            else if (val == "sample") p.targets = 1;
            else return LUTC_EINVAL;
            continue;
        }
        if (key == "pattern") {
            static const char* kNames[4] = {"rggb", "bggr", "grbg", "gbrg"};
            p.pattern = -1;
            for (int k = 0; k < 4; ++k)
                if (val == kNames[k]) p.pattern = k;
            if (p.pattern < 0) return LUTC_EINVAL;
            continue;
        }
        if (key == "table") {
            if (val == "u16") p.table = 1;
            else if (val == "u8") p.table = 2;
            else return LUTC_EINVAL;
            continue;
        }
        if (val.size() > 15) return LUTC_EINVAL;
        int64_t v = 0;
        for (char ch : val) {
            if (ch < '0' || ch > '9') return LUTC_EINVAL;
            v = v * 10 + (ch - '0');
        }
        if (key == "width") p.width = v;
        else if (key == "height") p.height = v;
        else if (key == "bands") p.bands = v;
        else if (key == "bits") p.bits = v;
        else if (key == "pitch") p.pitch = v;
        else if (key == "out_pitch") p.out_pitch = v;
        else if (key == "stretch") p.stretch = v;
        else if (key == "capacity") p.capacity = v;
        else if (key == "order") p.order = v;
        else return LUTC_EINVAL;
    }
    return LUTC_OK;
}

bool task_params_ok(const TaskParams& p, bool width, bool height, bool bits)
{
    if (width && (p.width < 0 || p.width > INT32_MAX)) return false;
    if (height && (p.height < 0 || p.height > INT32_MAX)) return false;
    if (bits && (p.bits < LUTC_MIN_BITS || p.bits > LUTC_MAX_BITS)) return false;
    return p.bands >= 1 && p.bands <= LUTC_MAX_BANDS && (p.stretch == 0 || p.stretch == 1);
}

lutc_raster raster_of(const TaskParams& p, const void* data)
{
    lutc_raster r;
    r.data = reinterpret_cast<const uint16_t*>(data);
    r.pitch_bytes = p.pitch >= 0 ? p.pitch : 2 * p.width;
    r.width = (int32_t)p.width;
    r.height = (int32_t)p.height;
    r.bands = (int32_t)p.bands;
    r.bits = (int32_t)p.bits;
    return r;
}

// per-band coefficient sets of [bands][width] arrays
std::vector<lutc_coeffs> coeffs_of(const TaskParams& p, const void* A, const void* G, const void* O)
{
    std::vector<lutc_coeffs> c(p.bands);
    for (int64_t b = 0; b < p.bands; ++b) {
        c[b].A = reinterpret_cast<const int32_t*>(A) + b * p.width;
        c[b].G = reinterpret_cast<const int32_t*>(G) + b * p.width;
        c[b].O = reinterpret_cast<const int32_t*>(O) + b * p.width;
        c[b].ncols = (int32_t)p.width;
    }
    return c;
}

namespace {

int attr(cudaDeviceAttr a, int dev, int* v)
{
    return cudaDeviceGetAttribute(v, a, dev) == cudaSuccess ? 0 : -1;
}

}  // namespace
}  // namespace lutc

using namespace lutc;

extern "C" int lutc_submit(int task, const char* params, const void* const* in, int n_in, void* const* out,
                           int n_out, void* workspace, size_t workspace_bytes, lutc_stream stream)
{
    TaskParams p;
    int rc = parse_task_params(params, p);
    if (rc) return rc;
    if (n_in < 0 || n_out < 0 || (n_in > 0 && !in) || (n_out > 0 && !out)) return LUTC_EINVAL;
    switch (task) {
    case LUTC_TASK_LUTGEN: {
        if (!task_params_ok(p, true, false, true) || n_in < 3 || n_out < 1) return LUTC_EINVAL;
        lutc_coeffs c = {reinterpret_cast<const int32_t*>(in[0]), reinterpret_cast<const int32_t*>(in[1]),
                         reinterpret_cast<const int32_t*>(in[2]), (int32_t)p.width};
        return lutc_lutgen(&c, (int)p.bits, reinterpret_cast<uint16_t*>(out[0]), stream);
    }
    case LUTC_TASK_HIST: {
        if (!task_params_ok(p, true, true, true) || n_in < 4 || n_out < 1) return LUTC_EINVAL;
        const lutc_raster r = raster_of(p, in[0]);
        const std::vector<lutc_coeffs> c = coeffs_of(p, in[1], in[2], in[3]);
        return lutc_hist(&r, c.data(), reinterpret_cast<uint64_t*>(out[0]), stream);
    }
    case LUTC_TASK_STRETCH: {
        if (!task_params_ok(p, false, false, true) || n_in < 1 || n_out < 2) return LUTC_EINVAL;
        return lutc_stretch(reinterpret_cast<const uint64_t*>(in[0]), (int)p.bands, (int)p.bits,
                            reinterpret_cast<uint8_t*>(out[0]), reinterpret_cast<int32_t*>(out[1]), stream);
    }
    case LUTC_TASK_COMPOSE: {
        if (!task_params_ok(p, true, false, true) || n_in < 2 || n_out < 1) return LUTC_EINVAL;
        return lutc_compose(reinterpret_cast<const uint16_t*>(in[0]), reinterpret_cast<const uint8_t*>(in[1]),
                            (int)p.width, (int)p.bits, reinterpret_cast<uint8_t*>(out[0]), stream);
    }
    case LUTC_TASK_APPLY: {
        if (!task_params_ok(p, true, true, true) || p.table == 0 || n_in < 2 || n_out < 1) return LUTC_EINVAL;
        const lutc_raster r = raster_of(p, in[0]);
        if (p.table == 1)
            return lutc_apply_u16(&r, reinterpret_cast<const uint16_t*>(in[1]), reinterpret_cast<uint16_t*>(out[0]),
                                  p.out_pitch >= 0 ? p.out_pitch : 2 * p.width, stream);
        return lutc_apply_u8(&r, reinterpret_cast<const uint8_t*>(in[1]), reinterpret_cast<uint8_t*>(out[0]),
                             p.out_pitch >= 0 ? p.out_pitch : p.width, stream);
    }
    case LUTC_TASK_CORRECT_IMAGE: {
        if (!task_params_ok(p, true, true, true) || n_in < 4 || n_out < 1) return LUTC_EINVAL;
        const lutc_raster r = raster_of(p, in[0]);
        const std::vector<lutc_coeffs> c = coeffs_of(p, in[1], in[2], in[3]);
        const int64_t elem = p.stretch ? 1 : 2;
        return lutc_correct_image(&r, c.data(), p.stretch ? LUTC_STRETCH : 0, out[0],
                                  p.out_pitch >= 0 ? p.out_pitch : elem * p.width, workspace, workspace_bytes,
                                  stream);
    }
    case LUTC_TASK_DEMOSAIC: {
        if (!task_params_ok(p, true, true, true) || p.bands != 1 || p.pattern < 0 || n_in < 1 || n_out < 1) return LUTC_EINVAL;
        const lutc_raster r = raster_of(p, in[0]);
        const bool correct = n_in >= 4;
        const lutc_coeffs c = correct ? lutc_coeffs{reinterpret_cast<const int32_t*>(in[1]),
                                                    reinterpret_cast<const int32_t*>(in[2]),
                                                    reinterpret_cast<const int32_t*>(in[3]), (int32_t)p.width}
                                      : lutc_coeffs{nullptr, nullptr, nullptr, 0};
        return lutc_demosaic(&r, correct ? &c : nullptr, p.pattern, reinterpret_cast<uint16_t*>(out[0]),
                             p.out_pitch >= 0 ? p.out_pitch : 2 * p.width, stream);
    }
    case LUTC_TASK_FIT: {
        // width = detectors, height = calibration lines
        if (p.width < 0 || p.width > INT32_MAX || p.height < 0 || p.height > INT32_MAX || n_in < 2 || n_out < 2)
            return LUTC_EINVAL;
        const int64_t xp = p.pitch >= 0 ? p.pitch : 2 * p.width;
        return lutc_fit(reinterpret_cast<const uint16_t*>(in[0]), xp, reinterpret_cast<const double*>(in[1]),
                        p.targets ? 8 * p.width : 0, (int)p.height, (int)p.width, (int)p.order,
                        reinterpret_cast<double*>(out[0]), reinterpret_cast<int32_t*>(out[1]),
                        n_out >= 3 ? reinterpret_cast<int32_t*>(out[2]) : nullptr, stream);
    }
    case LUTC_TASK_DEVICE_INFO: {
        if (p.capacity < 1 || n_out < 1) return LUTC_EINVAL;
        return lutc_device_info(reinterpret_cast<char*>(out[0]), (size_t)p.capacity, nullptr);
    }
    default:
        return LUTC_EINVAL;
    }
}

extern "C" int lutc_device_info(char* xml, size_t capacity, size_t* needed)
{
    if (!xml && capacity > 0) return LUTC_EINVAL;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        count = 0;
    }
    std::string doc = "<?xml version=\"1.0\"?>\n<gpus count=\"" + std::to_string(count) + "\">\n";
    for (int d = 0; d < count; ++d) {
        char name[256] = {0};
        size_t total_b = 0;
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, d) == cudaSuccess) {
            snprintf(name, sizeof(name), "%s", prop.name);
            total_b = prop.totalGlobalMem;
        }
        int major = 0, minor = 0, warp = 0, cmem = 0, smem = 0, clock = 0, sms = 0, regs = 0, threads = 0;
        int gx = 0, gy = 0, gz = 0, bx = 0, by = 0, bz = 0;
        attr(cudaDevAttrComputeCapabilityMajor, d, &major);
        attr(cudaDevAttrComputeCapabilityMinor, d, &minor);
        attr(cudaDevAttrWarpSize, d, &warp);
        attr(cudaDevAttrTotalConstantMemory, d, &cmem);
        attr(cudaDevAttrMaxSharedMemoryPerBlock, d, &smem);
        attr(cudaDevAttrClockRate, d, &clock);
        attr(cudaDevAttrMultiProcessorCount, d, &sms);
        attr(cudaDevAttrMaxRegistersPerBlock, d, &regs);
        attr(cudaDevAttrMaxThreadsPerBlock, d, &threads);
        attr(cudaDevAttrMaxGridDimX, d, &gx);
        attr(cudaDevAttrMaxGridDimY, d, &gy);
        attr(cudaDevAttrMaxGridDimZ, d, &gz);
        attr(cudaDevAttrMaxBlockDimX, d, &bx);
        attr(cudaDevAttrMaxBlockDimY, d, &by);
        attr(cudaDevAttrMaxBlockDimZ, d, &bz);
        cudaGetLastError();
        // names are NVIDIA's and contain no XML metacharacters; escape them anyway
        std::string nm;
        for (const char* c = name; *c; ++c) {
            if (*c == '&') nm += "&amp;";
            else if (*c == '<') nm += "&lt;";
            else if (*c == '>') nm += "&gt;";
            else if (*c == '"') nm += "&quot;";
            else nm += *c;
        }
        char buf[2048];
        snprintf(buf, sizeof(buf),
                 "  <gpu index=\"%d\">\n"
                 "    <name>%s</name>\n"
                 "    <compute_capability>%d.%d</compute_capability>\n"
                 "    <warp_size>%d</warp_size>\n"
                 "    <total_constant_memory unit=\"bytes\">%d</total_constant_memory>\n"
                 "    <total_global_memory unit=\"bytes\">%zu</total_global_memory>\n"
                 "    <shared_memory_per_block unit=\"bytes\">%d</shared_memory_per_block>\n"
                 "    <clock_rate unit=\"kHz\">%d</clock_rate>\n"
                 "    <multiprocessor_count>%d</multiprocessor_count>\n"
                 "    <registers_per_block>%d</registers_per_block>\n"
                 "    <max_threads_per_block>%d</max_threads_per_block>\n"
                 "    <max_grid_size x=\"%d\" y=\"%d\" z=\"%d\"/>\n"
                 "    <max_threads_dim x=\"%d\" y=\"%d\" z=\"%d\"/>\n"
                 "  </gpu>\n",
                 d, nm.c_str(), major, minor, warp, cmem, total_b, smem, clock, sms, regs, threads, gx, gy, gz, bx, by,
                 bz);
        doc += buf;
    }
    doc += "</gpus>\n";
    if (needed) *needed = doc.size() + 1;
    if (capacity < doc.size() + 1) {
        if (capacity > 0) xml[0] = '\0';
        return LUTC_ENOMEM;
    }
    memcpy(xml, doc.c_str(), doc.size() + 1);
    return LUTC_OK;
}

// ---------------------------------------------------------------------------
// fp64 FMA rate probe: the device properties above state the clock and the
// multiprocessor count, not how many fp64 fused multiply-adds a
// multiprocessor issues per clock; this kernel measures it.  Each thread
// runs 8 independent dependency chains of fma() on registers (no memory
// traffic until the one store of its result), so the fp64 pipe's issue rate
// is the only bound once enough warps are resident.
// ---------------------------------------------------------------------------
namespace lutc {
namespace probe {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_probe_fp64(long long iters, double b, double c, double* sink)
{
    double a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace probe
}  // namespace lutc

extern "C" int lutc_probe_fp64_fma(int blocks, long long iters, double* sink, long long* fmas, lutc_stream stream)
{
    if (blocks < 1 || blocks > (1 << 20) || iters < 1 || iters > (1ll << 24) || !sink) return LUTC_EINVAL;
    // b and c chosen so that every chain stays finite and normal: a -> a * b + c converges to c / (1 - b)
    using namespace lutc::probe;
    k_probe_fp64<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, 0.999999, 1e-6, sink);
    if (fmas) *fmas = (long long)blocks * kProbeThreads * kProbeChains * iters;
    return lutc::cuda_status(cudaGetLastError());
}
