// Internal declarations of the lutc CUDA library (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

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
    // |A| M^2 + |G| M + |O + 2^15| < 2^31, exactly: M <= 2^16 - 1 makes M^2 a uint32, |A| and |G| are
    // at most 2^31, so each product is one 32 x 32 -> 64-bit multiply and the sum stays below 2^64
    const uint32_t mm = (uint32_t)M * (uint32_t)M;
    const uint32_t a = A < 0 ? 0u - (uint32_t)A : (uint32_t)A;
    const uint32_t g = G < 0 ? 0u - (uint32_t)G : (uint32_t)G;
    const int64_t o64 = (int64_t)O + 32768;
    const uint64_t o = (uint64_t)(o64 < 0 ? -o64 : o64);
    return (uint64_t)a * mm + (uint64_t)g * (uint32_t)M + o < ((uint64_t)1 << 31);
}

// int32-exact column; Op = O + 2^15 (fits int32 for such a column).  Horner form in wrap-around
// 32-bit arithmetic: (A x + G) x + Op equals A x^2 + G x + Op modulo 2^32, and the true value fits
// int32, so the 32-bit result is exact.  Then clamp(floor(t / 2^16), 0, M) (arithmetic shift).
__device__ __forceinline__ uint32_t det_i32(int32_t A, int32_t G, int32_t Op, uint32_t x, int32_t M)
{
    const uint32_t t = ((uint32_t)A * x + (uint32_t)G) * x + (uint32_t)Op;
    return (uint32_t)__vimin_s32_relu(((int32_t)t) >> 16, M);
}

__device__ __forceinline__ uint32_t det_i64(int32_t A, int32_t G, int32_t O, uint32_t x, int32_t M)
{
    const int64_t t = (int64_t)A * (int64_t)((uint64_t)x * x) + (int64_t)G * (int64_t)x + (int64_t)O + 32768;
    const int64_t s = t >> 16;
    return (uint32_t)(s < 0 ? 0 : (s > M ? M : s));
}

// Debug builds (-DLUTC_CHECKED): in_bounds(ok, status) records LUTC_EINVAL in *status when a check
// fails (the first error wins) and returns ok, so that the guarded access is skipped; release builds
// compile every check away.
#ifdef LUTC_CHECKED
__device__ __forceinline__ bool in_bounds(bool ok, int* status)
{
    if (!ok) atomicCAS(status, 0, (int)LUTC_EINVAL);
    return ok;
}
#else
__device__ __forceinline__ bool in_bounds(bool, int*) { return true; }
#endif

// ---------------------------------------------------------------------------
// Host-side helpers shared by the entry points.
// ---------------------------------------------------------------------------
struct BandCoef {
    const int32_t* A;
    const int32_t* G;
    const int32_t* O;
};

inline int64_t table_len(int bits) { return (int64_t)1 << bits; }

// One image of a TMA-path launch.  For a single-image call it travels in the
// kernel parameters; a batch keeps an array of them in device memory.
struct JobDesc {
    int32_t W, H, bits, bands;
    int32_t strips, vout;
    int64_t unit_begin;     // first (band, strip, row) unit of this job in the launch
    uint8_t* out;
    int64_t out_pitch;
    int64_t hist_off;       // uint64 elements: band 0's histogram in the launch's histogram region
    int64_t S_off;          // bytes: band 0's stretch table in the launch's S region
    const BandCoef* coef;   // device [bands] (batch launches only)
};

// Per-band tables of a batched scan.
struct TableDesc {
    int64_t hist_off;  // uint64 elements
    int64_t S_off;     // bytes
    int64_t lohi_off;  // int32 elements
    int32_t bits;
    int32_t pad;
};

// Device-side description of a batch launch (all arrays in device memory).
struct BatchLaunch {
    const JobDesc* jobs;
    const CUtensorMap* maps;  // one per job, 64-byte aligned
    int32_t njobs;
    int32_t max_bits;
    int64_t unit_offset;      // first unit of the launch (jobs[0].unit_begin)
    int64_t units;
    const int64_t* starts;    // device [grid + 1]: block k walks units [starts[k], starts[k + 1])
    unsigned long long* ranges = nullptr;  // pass 1 only: [grid] packed (next << 32 | end) runs the blocks
                              // claim from and steal from, set to starts[] before the launch (or nullptr:
                              // static runs)
    int32_t granule = 0;      // units per claim of a stealing launch (0: eight tiles)
    int32_t grid;
    unsigned long long* hist;
    const uint8_t* S;
    uint8_t* S_out;
};

// TMA path (lutc_tma.cu)
bool tma_encode(CUtensorMap* map, const lutc_raster* in, int column_threads);
int tma_box_rows(int column_threads);
int tma_preload();     // loads every TMA kernel variant, caches occupancies
int tables_preload();  // loads the scan kernels
int tma_batch_pass(const BatchLaunch& b, int mode, int column_threads, int blocks_per_sm, cudaStream_t st);
// Blocks of a batch launch (SMs x resident blocks, capped by blocks_per_sm when > 0); 0 on error.
// Stealing launches pack unit numbers in 32 bits: their units must stay below this.
constexpr int64_t kStealMaxUnits = ((int64_t)1 << 32) - ((int64_t)1 << 20);
int tma_batch_grid(int mode, int column_threads, int max_bits, int blocks_per_sm);
// programmatic: launched right behind pass 1 of the same stream, overlapping its tail (see launch_programmatic)
int launch_stretch(const unsigned long long* hist, int bands, int bits, uint8_t* S, int32_t* lohi, cudaStream_t st,
                   bool programmatic = false);

// Launches `k` with the programmatic stream serialization attribute: it may start as soon as every
// block of the previous kernel in the stream has signalled (ptx::launch_dependents) and must call
// ptx::wait_prerequisites before it reads anything that kernel (or one before it) writes.  Used only
// between kernels of the library's own sequences, whose data flow is known.
template <class K, class... Args>
cudaError_t launch_programmatic(K k, dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}
int stretch_batch(const TableDesc* tables, int ntables, const unsigned long long* hist, uint8_t* S, int32_t* lohi,
                  cudaStream_t st);
enum { kModeHist = 0, kModeHistGlobal = 1, kModeApplyStretch = 2, kModeApplyDetector = 3 };

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Fused-path building blocks (lutc_correct.cu): pass 1 accumulating into a cleared histogram,
// pass 2 with (S != nullptr, stretch) or without the stretch, and the workspace table layout.
int pass1_accumulate(const lutc_raster* in, const lutc_coeffs* per_band, unsigned long long* hist, cudaStream_t st);
int pass2(const lutc_raster* in, const lutc_coeffs* per_band, const uint8_t* S, void* out, int64_t out_pitch,
          bool stretch, cudaStream_t st);
size_t tables_bytes(const lutc_raster* in);

// Row copies by the SMs (lutc_copy.cu): `rows` rows of `width` bytes from src (pitch spitch) to dst
// (pitch dpitch), any mix of device memory and device-accessible (page-locked) host memory.
int copy_rows(void* dst, int64_t dpitch, const void* src, int64_t spitch, int64_t width, int64_t rows,
              cudaStream_t st);
bool device_can_access(const void* p);  // page-locked host, device or managed memory at the same address
void tables_offsets(const lutc_raster* in, size_t* hist, size_t* S, size_t* lohi);

// returns LUTC_OK or LUTC_EINVAL
int check_raster(const lutc_raster* r);
int check_coeff_set(const lutc_raster* r, const lutc_coeffs* per_band);
int sm_count();
lutc_tuning tuning_for(int bits);  // the stored configuration (zeros = automatic)
cudaEvent_t* trace_slot();         // LUTC_TRACE_PHASES + 1 events of the next traced call, or nullptr
void record_path(bool tma);        // what lutc_last_path reports to the calling host thread
int cuda_status(cudaError_t e);  // cudaSuccess -> LUTC_OK, else LUTC_ECUDA (and clears the sticky-free error)
int* device_status_ptr();        // the kernel status word (lutc_device_status) of the current device, or nullptr
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();  // cuTensorMapEncodeTiled, or nullptr

// The task interface's parameter list (lutc_submit.cu): "key=value,..." of at most
// LUTC_PARAMS_MAX bytes; -1 marks a key that was not given.
struct TaskParams {
    int64_t width = -1, height = -1, bands = 1, bits = -1, pitch = -1, out_pitch = -1, stretch = 1, capacity = -1;
    int64_t order = -1;
    int table = 0;    // 0 unset, 1 u16, 2 u8
    int pattern = -1; // LUTC_BAYER_*
    int targets = 0;  // fit: 0 one target per line, 1 one per sample
};
int parse_task_params(const char* text, TaskParams& p);
bool task_params_ok(const TaskParams& p, bool width, bool height, bool bits);
lutc_raster raster_of(const TaskParams& p, const void* data);
std::vector<lutc_coeffs> coeffs_of(const TaskParams& p, const void* A, const void* G, const void* O);

}  // namespace lutc
