// lutc_correct_image_static: the fused correction for callers that cannot
// allocate device memory.
//
// lutc_correct_image needs a small scratch workspace (per-band histogram,
// stretch table and lo/hi) that the caller allocates.  Some callers cannot do
// that: a program that has no device allocator of its own and must not
// bring one in (plain C clients of this ABI, sandboxed plug-ins), code that
// runs where an allocation would stall or synchronise the device (a
// latency-bound loop that already owns all its buffers), or a framework whose
// memory manager owns every device allocation and forbids calls to
// cudaMalloc behind its back.  This entry point takes its scratch from a
// fixed, file-scope device array instead, so it allocates nothing.
//
// The array is LUTC_STATIC_SCRATCH_BYTES long and lives on every GPU that
// loads the library until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a stand-in
// object), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "lutc_internal.cuh"

namespace {

__device__ __align__(256) unsigned char g_static_scratch[LUTC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices];  // device address of g_static_scratch per device, or nullptr

// Device address of the scratch array on the current device (looked up on first use).
int static_scratch(void** addr)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LUTC_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return LUTC_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return LUTC_ECUDA;
        }
        g_static_addr[dev] = p;
    }
    *addr = g_static_addr[dev];
    return LUTC_OK;
}

}  // namespace

extern "C" int lutc_correct_image_static(const lutc_raster* in, const lutc_coeffs* per_band, int flags, void* out,
                                         int64_t out_pitch_bytes, lutc_stream stream)
{
    // lutc_correct_image's own checks first, in its order, so that a malformed call gets the same
    // LUTC_EINVAL whatever the raster's size; only then the limit of the fixed array
    int rc = lutc::check_raster(in);
    if (rc) return rc;
    if ((rc = lutc::check_coeff_set(in, per_band))) return rc;
    if (flags & ~LUTC_STRETCH) return LUTC_EINVAL;
    if (!(flags & LUTC_STRETCH))  // detector only: one pass, no scratch at all
        return lutc_correct_image(in, per_band, flags, out, out_pitch_bytes, nullptr, 0, stream);
    if ((int64_t)in->width * in->height > 0 && (!out || out_pitch_bytes < in->width)) return LUTC_EINVAL;
    if (lutc_correct_image_workspace(in) > (size_t)LUTC_STATIC_SCRATCH_BYTES) return LUTC_ENOMEM;
    void* scratch = nullptr;
    if ((rc = static_scratch(&scratch))) return rc;
    return lutc_correct_image(in, per_band, flags, out, out_pitch_bytes, scratch, LUTC_STATIC_SCRATCH_BYTES, stream);
}
