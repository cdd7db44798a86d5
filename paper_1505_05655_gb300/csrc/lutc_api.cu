// Version, status text and argument checks of the lutc C ABI.
#include <stdint.h>

#include <mutex>

#include "lutc_internal.cuh"

namespace lutc {

int check_raster(const lutc_raster* r)
{
    if (!r) return LUTC_EINVAL;
    if (r->bits < LUTC_MIN_BITS || r->bits > LUTC_MAX_BITS) return LUTC_EINVAL;
    if (r->bands < 1 || r->bands > LUTC_MAX_BANDS) return LUTC_EINVAL;
    if (r->width < 0 || r->height < 0) return LUTC_EINVAL;
    if ((int64_t)r->width * r->height > 0) {
        if (!r->data) return LUTC_EINVAL;
        if (r->pitch_bytes < 2 * (int64_t)r->width || (r->pitch_bytes & 1)) return LUTC_EINVAL;
        if (((uintptr_t)r->data) & 1) return LUTC_EINVAL;
    }
    return LUTC_OK;
}

int check_coeff_set(const lutc_raster* r, const lutc_coeffs* per_band)
{
    if (!per_band) return LUTC_EINVAL;
    for (int b = 0; b < r->bands; ++b) {
        const lutc_coeffs& c = per_band[b];
        if (c.ncols != r->width) return LUTC_EINVAL;
        if (r->width > 0 && (!c.A || !c.G || !c.O)) return LUTC_EINVAL;
    }
    return LUTC_OK;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    return n;
}

namespace {
std::mutex g_tuning_mu;
lutc_tuning g_tuning[LUTC_MAX_BITS + 1];
}  // namespace

lutc_tuning tuning_for(int bits)
{
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    return g_tuning[bits];
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return LUTC_OK;
    return LUTC_ECUDA;
}

}  // namespace lutc

extern "C" int lutc_version(void) { return 10000; }

extern "C" int lutc_set_tuning(int bits, const lutc_tuning* t)
{
    if (bits < LUTC_MIN_BITS || bits > LUTC_MAX_BITS) return LUTC_EINVAL;
    lutc_tuning v = {0, 0, 0};
    if (t) {
        if (t->path < LUTC_PATH_AUTO || t->path > LUTC_PATH_STRIP) return LUTC_EINVAL;
        if (t->column_threads != 0 && t->column_threads != 64 && t->column_threads != 128 && t->column_threads != 256)
            return LUTC_EINVAL;
        if (t->blocks_per_sm < 0 || t->blocks_per_sm > 32) return LUTC_EINVAL;
        v = *t;
    }
    std::lock_guard<std::mutex> lock(lutc::g_tuning_mu);
    lutc::g_tuning[bits] = v;
    return LUTC_OK;
}

extern "C" int lutc_get_tuning(int bits, lutc_tuning* t)
{
    if (!t || bits < LUTC_MIN_BITS || bits > LUTC_MAX_BITS) return LUTC_EINVAL;
    *t = lutc::tuning_for(bits);
    return LUTC_OK;
}

extern "C" const char* lutc_strerror(int status)
{
    switch (status) {
    case LUTC_OK: return "ok";
    case LUTC_EINVAL: return "invalid argument";
    case LUTC_EUNSUPPORTED: return "unsupported";
    case LUTC_ENOMEM: return "out of memory or workspace too small";
    case LUTC_ECUDA: return "CUDA error";
    case LUTC_ETIMEOUT: return "timed out";
    case LUTC_EBUSY: return "admission refused";
    case LUTC_ESHUTDOWN: return "shutting down";
    case LUTC_ECANCELED: return "cancelled";
    default: return "unknown status";
    }
}
