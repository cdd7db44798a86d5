// Internal declarations of the lutc CUDA library (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lutc.h"

namespace lutc {

// ---------------------------------------------------------------------------
// Step (L) on the device.
//
// D = clamp(floor((A x^2 + G x + O + 2^15) / 2^16), 0, M) for x <= M.
// A column is "int32-exact" when |A| M^2 + |G| M + |O + 2^15| < 2^31: then the
// true sum fits int32 for every x in [0, M], and evaluating it with
// wrap-around 32-bit arithmetic yields it exactly (the ring Z / 2^32 maps the
// in-range result to itself).  The bound itself is exact in uint64 for
// M < 2^16 (|A| M^2 < 2^63).  Other columns use int64, exact for bits <= 16
// (|A x^2| < 2^63 - 2^47).
// ---------------------------------------------------------------------------
__host__ __device__ inline bool col_fits_i32(int32_t A, int32_t G, int32_t O, int32_t M)
{
    const uint64_t m = (uint64_t)M;
    const uint64_t a = (uint64_t)(A < 0 ? -(int64_t)A : (int64_t)A);
    const uint64_t g = (uint64_t)(G < 0 ? -(int64_t)G : (int64_t)G);
    const int64_t o64 = (int64_t)O + 32768;
    const uint64_t o = (uint64_t)(o64 < 0 ? -o64 : o64);
    return a * (m * m) + g * m + o < ((uint64_t)1 << 31);
}

// int32-exact column; Op = O + 2^15 (fits int32 for such a column)
__device__ __forceinline__ uint32_t det_i32(int32_t A, int32_t G, int32_t Op, uint32_t x, int32_t M)
{
    const uint32_t t = (uint32_t)A * (x * x) + (uint32_t)G * x + (uint32_t)Op;
    const int32_t s = ((int32_t)t) >> 16;  // arithmetic shift: floor division by 2^16
    return (uint32_t)min(max(s, 0), M);
}

__device__ __forceinline__ uint32_t det_i64(int32_t A, int32_t G, int32_t O, uint32_t x, int32_t M)
{
    const int64_t t = (int64_t)A * (int64_t)((uint64_t)x * x) + (int64_t)G * (int64_t)x + (int64_t)O + 32768;
    const int64_t s = t >> 16;
    return (uint32_t)(s < 0 ? 0 : (s > M ? M : s));
}

// ---------------------------------------------------------------------------
// Host-side helpers shared by the entry points.
// ---------------------------------------------------------------------------
struct BandCoef {
    const int32_t* A;
    const int32_t* G;
    const int32_t* O;
};

inline int64_t table_len(int bits) { return (int64_t)1 << bits; }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// returns LUTC_OK or LUTC_EINVAL
int check_raster(const lutc_raster* r);
int check_coeff_set(const lutc_raster* r, const lutc_coeffs* per_band);
int sm_count();
lutc_tuning tuning_for(int bits);  // the stored configuration (zeros = automatic)
int cuda_status(cudaError_t e);  // cudaSuccess -> LUTC_OK, else LUTC_ECUDA (and clears the sticky-free error)

}  // namespace lutc
