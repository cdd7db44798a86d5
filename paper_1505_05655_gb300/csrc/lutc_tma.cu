// TMA-staged, persistent strip kernels of the fused correction (sm_103a).
//
// Section I of the paper names LUT generation and image correction as a task
// the GPU server runs on a client's raster.  This file is the fast path of
// that task for rasters whose base and row pitch are 16-byte aligned and
// whose width is at least 256 columns; other rasters take the plain strip
// kernels of lutc_correct.cu.  Both produce identical results.
//
// Block = 8 consumer warps + 1 producer warp, 3 blocks per SM, persistent (one wave).
//  * Work: the raster is cut into column strips of 8 * TC columns (TC column
//    threads, each owning 8 adjacent detectors); the (band, strip, row) units
//    of a launch are laid out linearly.  A single image gives every block an
//    equal contiguous share; a batch gives each block a contiguous run of
//    about equal modelled cost (starts[], planned on the host), over the
//    concatenated units of all its images.  The job descriptor stays in
//    memory (kernel parameters or the batch's job table): the walk keeps only
//    the fields it needs on every tile.
//  * Producer: one thread streams tiles of (1024 / TC) rows x (8 TC) columns
//    (16 KB) into a 3-stage shared-memory ring with 2-D tensor TMA loads
//    (cp.async.bulk.tensor), completion counted on a per-stage mbarrier;
//    144 KB are in flight per SM.  Columns past the image edge and rows past
//    the raster are zero-filled by TMA and ignored by the consumers.
//  * Consumers: each thread reads its 8 pixels of a row (one 16-byte shared
//    load), clamps them with a packed 16x2 min, evaluates step (L) in
//    wrap-around int32 (det_i32: Horner form, exact when the column bound
//    |A| M^2 + |G| M + |O + 2^15| < 2^31 holds; other columns in int64) and then
//      pass 1: increments the band's histogram in shared memory (one warp-wide
//              atomic per pixel); at each band change and at the end it is
//              added into the band's global uint64 histogram;
//      pass 2: looks up S[D] in the band's stretch table in shared memory and
//              stores 8 output bytes per row (detector-only: 16 bytes of D).
//  * Every wait is bounded (about two seconds of clock); on expiry the block
//    records LUTC_ETIMEOUT in the library's device status word, the producer
//    waits (bounded) for its copies in flight, and the block returns.
//  * Debug builds (-DLUTC_CHECKED) check every tile offset, row, column, bin
//    and table index (in_bounds) and record LUTC_EINVAL instead of an access
//    out of range.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <utility>

#include "lutc_internal.cuh"
#include "lutc_ptx.cuh"

namespace lutc {

namespace {

constexpr int kConsumers = 256;            // consumer threads per block (8 warps)
constexpr int kThreads = kConsumers + 32;  // + one producer warp
constexpr int kConsumerWarps = kConsumers / 32;
// Ring geometry (compile-time; the product builds the defaults).
#ifndef LUTC_RING_STAGES
#define LUTC_RING_STAGES 3
#endif
#ifndef LUTC_ROWS_PER_THREAD
#define LUTC_ROWS_PER_THREAD 4
#endif
constexpr int kStages = LUTC_RING_STAGES;
constexpr int kRowsPerThread = LUTC_ROWS_PER_THREAD;  // rows of a tile each consumer thread processes
constexpr int kTileBytes = kConsumers * 16 * kRowsPerThread;  // 16 KB with the defaults
constexpr int kRingBytes = kStages * kTileBytes;
// mbarriers after the ring (full and empty per stage, one consumer barrier), then the table
constexpr int kBarRegion = ((2 * kStages + 1) * 8 + 127) / 128 * 128;
constexpr int kTableOffset = kRingBytes + kBarRegion;
static_assert((2 * kStages + 1) * 8 + kStages * 12 <= kBarRegion, "barrier region (barriers, per-stage tile units)");
// Work stealing (batch passes): a block claims a.granule units of its own run at a time (planned per
// launch: about a sixteenth of a block's share, one to eight tiles), and a run with fewer than two
// granules left is not stolen from.
constexpr int kStealTries = 8;  // lost compare-and-swap races before a block stops looking for work
static_assert(kTableOffset % 128 == 0, "table alignment");

enum Mode { kHist = kModeHist, kHistGlobal = kModeHistGlobal, kApplyStretch = kModeApplyStretch,
            kApplyDetector = kModeApplyDetector };

__device__ int g_device_status;  // 0, or the first error a kernel of this library recorded

// Single-image launch: everything in the kernel parameters.
struct TmaArgs {
    CUtensorMap map;  // uint16 [bands * H][W], row stride = pitch, box {256, rows per tile}
    JobDesc job;
    BandCoef coef[LUTC_MAX_BANDS];
    int64_t units;
    int64_t units_per_block;
    unsigned long long* hist;
    const uint8_t* S;
    int32_t max_bits;
};

// Batch launch: job table, tensor maps and coefficient arrays in device memory.
struct BatchArgs {
    const JobDesc* jobs;
    const CUtensorMap* maps;
    int32_t njobs;
    int32_t max_bits;
    int64_t unit_offset;  // first unit of this launch (its jobs' unit_begin are absolute)
    int64_t units;
    int64_t units_per_block;
    const int64_t* starts;  // [gridDim.x + 1] block boundaries in units, balanced by cost
    unsigned long long* hist;
    const uint8_t* S;
    unsigned long long* ranges;  // stealing launches only: [gridDim.x] units (next << 32 | end) each block
                                 // has left, set to its static run before the launch
    int32_t granule;             // stealing launches only: units per claim (>= 1)
};

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, TMA (lutc_ptx.cuh); this file's waits record into g_device_status
// ---------------------------------------------------------------------------
using ptx::mbar_arrive;
using ptx::mbar_arrive_expect_tx;
using ptx::mbar_init;
using ptx::mbar_try_wait;
using ptx::smem_addr;
using ptx::tma_load_2d;
using ptx::tma_prefetch_map;

// Wait for the phase of `bar` with the given parity; false after ~2 s (status recorded).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    return ptx::mbar_wait_bounded(bar, parity, &g_device_status);
}

// Barrier among the consumer threads only (the producer runs ahead), bounded like every wait.
__device__ __forceinline__ bool consumer_sync(uint64_t* bar, uint32_t& phase)
{
    mbar_arrive(bar);
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    return ok;
}

// Warp-collective (the producer warp): finds the block whose run has the most units left, takes the
// upper half of that run with one compare-and-swap and makes it this block's run (`mine`).  The
// victim's owner claims from the front of its run with an atomic add on the same word, so the two
// never overlap: either the swap sees the owner's latest claim or it fails.  False when no run has
// `min_left` units left, or after kStealTries lost races.
__device__ bool steal_half(unsigned long long* ranges, unsigned long long* mine, int nblocks, int lane, int64_t min_left)
{
    for (int t = 0; t < kStealTries; ++t) {
        int64_t best = 0;
        int victim = -1;
        for (int v = lane; v < nblocks; v += 32) {
            const unsigned long long w = __ldcg(ranges + v);
            const int64_t rem = (int64_t)(w & 0xffffffffull) - (int64_t)(w >> 32);
            if (rem > best) {
                best = rem;
                victim = v;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ov = __shfl_xor_sync(0xffffffffu, victim, o);
            if (ob > best || (ob == best && ov > victim)) {
                best = ob;
                victim = ov;
            }
        }
        if (best < min_left) return false;
        int won = 0;
        if (lane == 0) {
            const unsigned long long w = __ldcg(ranges + victim);
            const unsigned long long n = w >> 32, e = w & 0xffffffffull;
            if (e > n && (int64_t)(e - n) >= min_left) {
                const unsigned long long cut = n + (e - n + 1) / 2;  // the owner keeps [n, cut)
                if (atomicCAS(ranges + victim, w, (n << 32) | cut) == w) {
                    atomicExch(mine, (cut << 32) | e);
                    won = 1;
                }
            }
        }
        if (__shfl_sync(0xffffffffu, won, 0)) return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// per-pixel arithmetic
// ---------------------------------------------------------------------------
// (P) clamp of raw DN to M, two pixels per 32-bit word
__device__ __forceinline__ void unpack_clamped(const uint4 v, uint32_t M2, uint32_t (&x)[8])
{
    const uint32_t w0 = __vminu2(v.x, M2), w1 = __vminu2(v.y, M2), w2 = __vminu2(v.z, M2), w3 = __vminu2(v.w, M2);
    x[0] = w0 & 0xffffu; x[1] = w0 >> 16;
    x[2] = w1 & 0xffffu; x[3] = w1 >> 16;
    x[4] = w2 & 0xffffu; x[5] = w2 >> 16;
    x[6] = w3 & 0xffffu; x[7] = w3 >> 16;
}

// 8 output bytes (lo: bytes 0-3, hi: bytes 4-7) at any address, with the widest aligned stores
__device__ __forceinline__ void store8(uint8_t* dst, uint32_t lo, uint32_t hi)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
    if ((a & 7) == 0) {
        *reinterpret_cast<uint2*>(dst) = make_uint2(lo, hi);
    } else if ((a & 3) == 0) {
        reinterpret_cast<uint32_t*>(dst)[0] = lo;
        reinterpret_cast<uint32_t*>(dst)[1] = hi;
    } else if ((a & 1) == 0) {
        uint16_t* d = reinterpret_cast<uint16_t*>(dst);
        d[0] = (uint16_t)lo; d[1] = (uint16_t)(lo >> 16);
        d[2] = (uint16_t)hi; d[3] = (uint16_t)(hi >> 16);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = (uint8_t)(lo >> (8 * k));
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[4 + k] = (uint8_t)(hi >> (8 * k));
    }
}

// 8 uint16 outputs at any even address
__device__ __forceinline__ void store8x16(uint8_t* dst, const uint32_t (&d)[8])
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
    const uint32_t w0 = d[0] | (d[1] << 16), w1 = d[2] | (d[3] << 16), w2 = d[4] | (d[5] << 16), w3 = d[6] | (d[7] << 16);
    if ((a & 15) == 0) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(w0, w1, w2, w3);
    } else if ((a & 7) == 0) {
        reinterpret_cast<uint2*>(dst)[0] = make_uint2(w0, w1);
        reinterpret_cast<uint2*>(dst)[1] = make_uint2(w2, w3);
    } else if ((a & 3) == 0) {
        uint32_t* p = reinterpret_cast<uint32_t*>(dst);
        p[0] = w0; p[1] = w1; p[2] = w2; p[3] = w3;
    } else {
        uint16_t* p = reinterpret_cast<uint16_t*>(dst);
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = (uint16_t)d[k];
    }
}

// One row of a thread's 8 pixels through pass MODE.  kFull: all 8 columns exist; otherwise the
// first n do and the rest (TMA zero fill past the image edge) are masked out.
template <int MODE, bool kFull>
__device__ __forceinline__ void row8(const uint4 v, int n, const int32_t (&A)[8], const int32_t (&G)[8],
                                     const int32_t (&O)[8], int32_t M, uint32_t M2, uint32_t* hs,
                                     unsigned long long* hb, const unsigned char* table, uint8_t* dst, int vout)
{
    uint32_t x[8], d[8];
    unpack_clamped(v, M2, x);
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) d[jj] = det_i32(A[jj], G[jj], O[jj], x[jj], M);  // (L)
    if (MODE == kModeHist) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
            if ((kFull || jj < n) && in_bounds(d[jj] <= (uint32_t)M, &g_device_status)) atomicAdd(hs + d[jj], 1u);
    } else if (MODE == kModeHistGlobal) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
            if ((kFull || jj < n) && in_bounds(d[jj] <= (uint32_t)M, &g_device_status)) atomicAdd(hb + d[jj], 1ull);
    } else if (MODE == kModeApplyStretch) {
        uint32_t o[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) o[jj] = in_bounds(d[jj] <= (uint32_t)M, &g_device_status) ? table[d[jj]] : 0u;
        if (kFull) {
            const uint32_t lo = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
            const uint32_t hi = o[4] | (o[5] << 8) | (o[6] << 16) | (o[7] << 24);
            if (vout) *reinterpret_cast<uint2*>(dst) = make_uint2(lo, hi);
            else store8(dst, lo, hi);
        } else {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (jj < n) dst[jj] = (uint8_t)o[jj];
        }
    } else {
        if (kFull) {
            if (vout) {
                uint4 r;
                r.x = d[0] | (d[1] << 16); r.y = d[2] | (d[3] << 16);
                r.z = d[4] | (d[5] << 16); r.w = d[6] | (d[7] << 16);
                *reinterpret_cast<uint4*>(dst) = r;
            } else {
                store8x16(dst, d);
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (jj < n) reinterpret_cast<uint16_t*>(dst)[jj] = (uint16_t)d[jj];
        }
    }
}

// The job's descriptor stays in memory (the job table, or the kernel parameters of a single-image
// launch); the walk keeps only the fields it needs on every tile in registers.
template <bool kBatch, class Args>
__device__ __forceinline__ const JobDesc* job_ptr(const Args& a, int j)
{
    if constexpr (kBatch) return a.jobs + j;
    else return &a.job;
}

template <bool kBatch, class Args>
__device__ __forceinline__ const CUtensorMap* map_of(const Args& a, int j)
{
    if constexpr (kBatch) return a.maps + j;
    else return &a.map;
}

template <bool kBatch, class Args>
__device__ __forceinline__ BandCoef coef_of(const Args& a, const JobDesc* J, int band)
{
    if constexpr (kBatch) return J->coef[band];
    else return a.coef[band];
}

// One persistent kernel for both passes (MODE) and both launch kinds (kBatch).
// The launch's work is the concatenation over its jobs of (band, strip, row)
// units; block k takes units [k q, (k + 1) q) and walks them tile by tile.
// kSteal (batch pass 1): a block starts on its static run as above, but claims it a granule at a
// time from a.ranges[block], and once it is used up takes the upper half of the largest run left
// (steal_half), so that blocks whose rows cost more than the plan priced them are helped by the
// others; the runs stay contiguous, so a block rarely changes band (each change flushes its shared
// histogram).  Each ring stage carries its tile's first unit and row count (unit -1 ends the walk).
template <int TC, int MODE, bool kBatch, class Args, bool kSteal = false>
__global__ void __launch_bounds__(kThreads, 3) k_tma_strip(const __grid_constant__ Args a)
{
    constexpr int SW = 8 * TC;                 // strip width (columns)
    constexpr int P = kConsumers / TC;         // row phases
    constexpr int RT = P * kRowsPerThread;     // rows per tile
    constexpr int NB = TC / 32;                // TMA boxes (256 columns each) per tile row
    static_assert(RT * SW * 2 == kTileBytes, "tile size");

    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* ring = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kRingBytes);
    uint64_t* empty = full + kStages;
    uint64_t* csync = empty + kStages;  // consumer-only barrier (band changes)
    unsigned char* table = smem + kTableOffset;
    uint32_t* hs = reinterpret_cast<uint32_t*>(table);

    const int tid = threadIdx.x;
    // pass 1: the scan behind it may launch now (it waits for this grid's histogram itself)
    if (MODE == kHist || MODE == kHistGlobal) ptx::launch_dependents();

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        mbar_init(csync, kConsumers);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (MODE == kHist)
        for (int i = tid; i < (1 << a.max_bits); i += kThreads) hs[i] = 0;
    __syncthreads();

    // This block's share of the units, walked without divisions after the first.
    int64_t u0, u1;
    if constexpr (kSteal) {
        u0 = 0;  // claimed below
        u1 = 1;
    } else if constexpr (kBatch) {
        u0 = a.starts[blockIdx.x];
        u1 = a.starts[blockIdx.x + 1];
    } else {
        u0 = (int64_t)blockIdx.x * a.units_per_block;
        u1 = min(a.units, u0 + a.units_per_block);
    }
    if (u0 >= u1) return;
    int64_t left = kSteal ? 0 : u1 - u0;
    int j = 0;
    const JobDesc* Jp = job_ptr<kBatch>(a, 0);
    int H = 0, row = 0, band = 0, strip = 0;
    auto seek = [&](int64_t u) {  // the walk's position at unit u
        if constexpr (kBatch) {
            int lo = 0, hi = a.njobs - 1;  // last job whose first unit is <= u
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.jobs[mid].unit_begin <= u) lo = mid;
                else hi = mid - 1;
            }
            j = lo;
        }
        Jp = job_ptr<kBatch>(a, j);
        H = Jp->H;
        const int64_t r = u - Jp->unit_begin;
        const int64_t seg = r / H;
        row = (int)(r - seg * H);
        const int strips = Jp->strips;
        band = (int)(seg / strips);
        strip = (int)(seg - (int64_t)band * strips);
    };
    if constexpr (!kSteal) seek(u0);
    // stealing launches: each stage's first unit (-1: the walk is over) and row count
    int64_t* stage_unit = reinterpret_cast<int64_t*>(csync + 1);
    int* stage_rows = reinterpret_cast<int*>(stage_unit + kStages);
    int stage = 0;
    uint32_t phase = 0;

    if (tid >= kConsumers) {
        // ------------------------------------------------------------ producer
        if (!kSteal && tid != kConsumers) return;
        int issued = 0;
        bool ok = true;
        if constexpr (kSteal) {
            // the whole producer warp looks for runs to steal; its lane 0 claims, issues and publishes
            const int plane = tid - kConsumers;
            unsigned long long* mine = a.ranges + blockIdx.x;
            const int64_t G = a.granule;  // units per claim
            int64_t next_unit = -1;  // lane 0: the unit after the last tile issued
            int W = 0;
            for (;;) {
                unsigned long long old = 0;
                if (plane == 0) old = atomicAdd(mine, (unsigned long long)G << 32);
                old = __shfl_sync(0xffffffffu, old, 0);
                const int64_t n0 = (int64_t)(old >> 32), e0 = (int64_t)(old & 0xffffffffull);
                if (n0 >= e0) {
                    if (!steal_half(a.ranges, mine, (int)gridDim.x, plane, 2 * G)) break;
                    continue;
                }
                int good = 1;
                if (plane == 0) {
                    if (n0 != next_unit) {
                        seek(n0);
                        tma_prefetch_map(map_of<kBatch>(a, j));
                        W = Jp->W;
                    }
                    int64_t u = n0;
                    left = min(n0 + G, e0) - n0;
                    while (left > 0) {
                        const int nrows = (int)min((int64_t)min(RT, H - row), left);
                        if (issued >= kStages && !mbar_wait(&empty[stage], phase ^ 1u)) {
                            good = 0;
                            break;
                        }
                        const int x0 = strip * SW;
                        const int nb = min(NB, (W - x0 + 255) >> 8);
                        stage_unit[stage] = u;  // published by the arrive below
                        stage_rows[stage] = nrows;
                        mbar_arrive_expect_tx(&full[stage], (uint32_t)(nb * 512 * RT));
                        unsigned char* dst = ring + stage * kTileBytes;
                        const int y = band * H + row;
                        const CUtensorMap* map = map_of<kBatch>(a, j);
                        for (int b = 0; b < nb; ++b)
                            tma_load_2d(dst + b * (RT * 512), map, &full[stage], x0 + b * 256, y);
                        ++issued;
                        left -= nrows;
                        u += nrows;
                        row += nrows;
                        if (row == H) {
                            row = 0;
                            if (++strip == Jp->strips) {
                                strip = 0;
                                if (++band == Jp->bands) {
                                    band = 0;
                                    // the walk stands at the next job even when this claim ends here:
                                    // the next claim may continue right there without a seek
                                    if (j + 1 < a.njobs) {
                                        Jp = job_ptr<kBatch>(a, ++j);
                                        tma_prefetch_map(map_of<kBatch>(a, j));
                                        H = Jp->H;
                                        W = Jp->W;
                                    }
                                }
                            }
                        }
                        if (++stage == kStages) { stage = 0; phase ^= 1u; }
                    }
                    next_unit = u;
                }
                if (!__shfl_sync(0xffffffffu, good, 0)) {
                    ok = false;
                    break;
                }
            }
            if (plane != 0) return;
            if (ok) {
                // the end of the walk: a stage without a copy, unit -1
                if (issued >= kStages && !mbar_wait(&empty[stage], phase ^ 1u)) {
                    ok = false;
                } else {
                    stage_unit[stage] = -1;
                    mbar_arrive(&full[stage]);
                }
            }
        } else {
            if constexpr (kBatch) tma_prefetch_map(map_of<kBatch>(a, j));
            int W = Jp->W;
            while (left > 0) {
                const int nrows = (int)min((int64_t)min(RT, H - row), left);
                if (issued >= kStages && !mbar_wait(&empty[stage], phase ^ 1u)) {
                    ok = false;
                    break;
                }
                const int x0 = strip * SW;
                const int nb = min(NB, (W - x0 + 255) >> 8);
                mbar_arrive_expect_tx(&full[stage], (uint32_t)(nb * 512 * RT));
                unsigned char* dst = ring + stage * kTileBytes;
                const int y = band * H + row;
                const CUtensorMap* map = map_of<kBatch>(a, j);
                for (int b = 0; b < nb; ++b) tma_load_2d(dst + b * (RT * 512), map, &full[stage], x0 + b * 256, y);
                ++issued;
                left -= nrows;
                row += nrows;
                if (row == H) {
                    row = 0;
                    if (++strip == Jp->strips) {
                        strip = 0;
                        if (++band == Jp->bands) {
                            band = 0;
                            if (kBatch && left > 0) {
                                Jp = job_ptr<kBatch>(a, ++j);
                                tma_prefetch_map(map_of<kBatch>(a, j));
                                H = Jp->H;
                                W = Jp->W;
                            }
                        }
                    }
                }
                if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok) {
            // let every copy issued land before the block's shared memory goes away
            for (int i = 0; i < kStages && i < issued; ++i) {
                if (--stage < 0) { stage = kStages - 1; phase ^= 1u; }
                mbar_wait(&full[stage], phase);
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    // pass 2 launched right behind the scan (programmatic launch): the producer already streams raw
    // tiles, which no kernel of the step writes; the stretch table is read only after the scan
    if constexpr (MODE == kApplyStretch) ptx::wait_prerequisites();
    const int ct = tid % TC;  // column thread: owns columns strip * SW + ct * 8 .. + 7
    const int ph = tid / TC;  // row phase
    const int lane = tid & 31;
    const unsigned char* my = ring + (ct >> 5) * (RT * 512) + (ct & 31) * 16 + ph * 512;
    uint32_t sync_phase = 0;
    bool new_seg = true;
    bool have_band = false;
    int L = 1 << Jp->bits;
    int32_t M = L - 1;
    uint32_t M2 = (uint32_t)M | ((uint32_t)M << 16);
    unsigned long long* hb = nullptr;  // global histogram of the band being counted
    int hb_len = 0;
    int32_t A[8], G[8], O[8];
    bool fits = true;
    bool masked = false;  // this warp holds the right-edge partial chunk of its strip
    int n = 0, c0 = 0;
    constexpr int64_t esize = MODE == kApplyDetector ? 2 : 1;  // output bytes per pixel
    uint8_t* orow = nullptr;  // output passes: this thread's first byte of row (row + ph) of the segment
    int64_t opitch = 0;
    int vout = 0;
    int64_t expect = -1;  // stealing launches: the unit the walk stands at
    int tab_key = -1;     // stealing launches: (job << 8) | band of the histogram held
    for (;;) {
        int nrows;
        if constexpr (kSteal) {
            if (!mbar_wait(&full[stage], phase)) return;
            const int64_t u = stage_unit[stage];
            if (u < 0) break;  // the walk is over
            nrows = stage_rows[stage];
            if (u != expect) {
                // the first tile of a claim that does not continue the walk: any band of any job
                seek(u);
                new_seg = true;
            }
            expect = u + nrows;
        } else {
            if (left <= 0) break;
            nrows = (int)min((int64_t)min(RT, H - row), left);
        }
        if (new_seg) {
            bool new_band;  // a new band (of this or another job) starts
            if constexpr (kSteal) new_band = ((j << 8) | band) != tab_key;
            else new_band = strip == 0 || !have_band;
            if (new_band) {
                if (MODE == kHist && have_band) {
                    // every consumer is done with the previous band: flush it and clear
                    if (!consumer_sync(csync, sync_phase)) return;
                    for (int i = tid; i < hb_len; i += kConsumers) {
                        const uint32_t c = hs[i];
                        if (c) {
                            atomicAdd(hb + i, (unsigned long long)c);
                            hs[i] = 0;
                        }
                    }
                    if (!consumer_sync(csync, sync_phase)) return;
                }
                L = 1 << Jp->bits;
                if (!in_bounds(Jp->bits <= a.max_bits && band < Jp->bands, &g_device_status)) return;
                M = L - 1;
                M2 = (uint32_t)M | ((uint32_t)M << 16);
                hb = a.hist + Jp->hist_off + (int64_t)band * L;
                hb_len = L;
                if (MODE == kApplyStretch) {
                    if (have_band && !consumer_sync(csync, sync_phase)) return;
                    const uint4* src = reinterpret_cast<const uint4*>(a.S + Jp->S_off + (int64_t)band * L);
                    for (int i = tid; i < L / 16; i += kConsumers) reinterpret_cast<uint4*>(table)[i] = src[i];
                    if (!consumer_sync(csync, sync_phase)) return;
                }
                have_band = true;
                if constexpr (kSteal) tab_key = (j << 8) | band;
            }
            new_seg = false;
            c0 = strip * SW + ct * 8;
            n = min(8, Jp->W - c0);
            if constexpr (MODE >= kApplyStretch) {
                opitch = Jp->out_pitch;
                vout = Jp->vout;
                orow = Jp->out + ((int64_t)band * H + row + ph) * opitch + (int64_t)c0 * esize;
            }
            fits = true;
            const BandCoef cf = coef_of<kBatch>(a, Jp, band);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                if (jj < n) {
                    A[jj] = __ldg(cf.A + c0 + jj);
                    G[jj] = __ldg(cf.G + c0 + jj);
                    O[jj] = __ldg(cf.O + c0 + jj);
                    fits = fits && col_fits_i32(A[jj], G[jj], O[jj], M);
                } else {
                    A[jj] = 0; G[jj] = 0; O[jj] = 0;
                }
            }
            if (fits) {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) O[jj] += 32768;
            }
            // A warp with the partial chunk runs the masked path in every lane: running the full
            // path in 31 lanes and then the masked one in one lane would double the warp's time
            // per tile, and the ring only advances at its slowest warp's pace.
            masked = __any_sync(0xffffffffu, n > 0 && n < 8);
        }
        if constexpr (!kSteal) {
            if (!mbar_wait(&full[stage], phase)) return;
        }
        const unsigned char* tile = my + stage * kTileBytes;
        const bool in_range =
            in_bounds(tile >= ring && tile + (kRowsPerThread - 1) * P * 512 + 16 <= ring + kRingBytes &&
                          row >= 0 && nrows >= 1 && row + nrows <= H && strip < Jp->strips &&
                          (n <= 0 || c0 + n <= Jp->W),
                      &g_device_status);
        if (!in_range) n = 0;  // (checked builds) the tile is skipped
        if (fits && n > 0) {
            // int32-exact columns; a right-edge chunk (n < 8) reads TMA's zero fill past the
            // edge and masks those pixels out, so it stays on this path too
            if (!masked) {
#pragma unroll
                for (int i = 0; i < kRowsPerThread; ++i)
                    if (ph + i * P < nrows)
                        row8<MODE, true>(*reinterpret_cast<const uint4*>(tile + i * P * 512), 8, A, G, O, M, M2,
                                         hs, hb, table, orow + (MODE >= kApplyStretch ? i * P * opitch : 0), vout);
            } else {
#pragma unroll
                for (int i = 0; i < kRowsPerThread; ++i)
                    if (ph + i * P < nrows)
                        row8<MODE, false>(*reinterpret_cast<const uint4*>(tile + i * P * 512), n, A, G, O, M, M2,
                                          hs, hb, table, orow + (MODE >= kApplyStretch ? i * P * opitch : 0), vout);
            }
        } else if (n > 0) {
            // a column that needs int64: exact, slow, few registers
            const BandCoef cf = coef_of<kBatch>(a, Jp, band);
#pragma unroll 1
            for (int i = 0; i < kRowsPerThread; ++i) {
                if (ph + i * P >= nrows) break;
                const uint16_t* px = reinterpret_cast<const uint16_t*>(tile + i * P * 512);
                uint8_t* o = orow + (MODE >= kApplyStretch ? i * P * opitch : 0);
#pragma unroll 1
                for (int jj = 0; jj < n; ++jj) {
                    const uint32_t x = min((uint32_t)px[jj], (uint32_t)M);
                    const uint32_t d =
                        det_i64(__ldg(cf.A + c0 + jj), __ldg(cf.G + c0 + jj), __ldg(cf.O + c0 + jj), x, M);
                    if (!in_bounds(d <= (uint32_t)M, &g_device_status)) continue;
                    if (MODE == kHist) atomicAdd(hs + d, 1u);
                    else if (MODE == kHistGlobal) atomicAdd(hb + d, 1ull);
                    else if (MODE == kApplyStretch) o[jj] = table[d];
                    else reinterpret_cast<uint16_t*>(o)[jj] = (uint16_t)d;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[stage]);
        left -= nrows;
        row += nrows;
        if constexpr (MODE >= kApplyStretch) orow += (int64_t)nrows * opitch;
        if (row == H) {
            row = 0;
            new_seg = true;
            if (++strip == Jp->strips) {
                strip = 0;
                if (++band == Jp->bands) {
                    band = 0;
                    // (stealing: the next tile may not continue the walk, but a next job exists to
                    // stand at; a discontinuity is re-sought at the next stage)
                    bool next_job = left > 0;
                    if constexpr (kSteal) next_job = j + 1 < a.njobs;
                    if (kBatch && next_job) {
                        Jp = job_ptr<kBatch>(a, ++j);
                        H = Jp->H;
                    }
                }
            }
        }
        if (++stage == kStages) { stage = 0; phase ^= 1u; }
    }
    if (MODE == kHist && have_band) {
        if (!consumer_sync(csync, sync_phase)) return;
        for (int i = tid; i < hb_len; i += kConsumers) {
            const uint32_t c = hs[i];
            if (c) atomicAdd(hb + i, (unsigned long long)c);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

int pick_tc(int W, int bits)
{
    const int t = tuning_for(bits).column_threads;
    if (t) return t;
    return W >= 4096 ? 256 : (W >= 1024 ? 128 : 64);
}

size_t table_bytes(int mode, int max_bits)
{
    const size_t L = (size_t)1 << max_bits;
    return mode == kHist ? L * 4 : (mode == kApplyStretch ? L : 0);
}

constexpr size_t kMaxSmem = (size_t)kTableOffset + ((size_t)4 << 15);  // 15-bit histogram
static_assert(kMaxSmem <= 232448, "shared memory per block");

// Grid = SMs x resident blocks (capped by blocks_per_sm when > 0), one wave.  The kernel's
// shared-memory limit is raised once to the largest any launch uses, and the occupancy of each
// (kernel, shared size) is computed once per device: a launch then costs no attribute change
// and no occupancy query.
template <class K>
int grid_for(K k, size_t smem, int blocks_per_sm, int64_t* grid)
{
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> raised;                 // (kernel, device)
    static std::map<std::tuple<const void*, int, size_t>, int> occ;     // (kernel, device, smem) -> blocks/SM
    const void* key = reinterpret_cast<const void*>(k);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LUTC_ECUDA;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!raised.count({key, dev})) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem) != cudaSuccess)
                return LUTC_ECUDA;
            raised.insert({key, dev});
        }
        auto it = occ.find(std::make_tuple(key, dev, smem));
        if (it != occ.end()) {
            per_sm = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess ||
                per_sm < 1)
                return LUTC_ECUDA;
            occ[std::make_tuple(key, dev, smem)] = per_sm;
        }
    }
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    *grid = (int64_t)sm_count() * per_sm;
    return LUTC_OK;
}

template <int TC, int MODE>
int launch_single_tc(TmaArgs& a, cudaStream_t st, bool programmatic)
{
    auto k = k_tma_strip<TC, MODE, false, TmaArgs>;
    const size_t smem = (size_t)kTableOffset + table_bytes(MODE, a.max_bits);
    int64_t grid = 0;
    int rc = grid_for(k, smem, tuning_for(a.job.bits).blocks_per_sm, &grid);
    if (rc) return rc;
    constexpr int SW = 8 * TC;
    a.job.strips = (a.job.W + SW - 1) / SW;
    a.units = (int64_t)a.job.bands * a.job.strips * a.job.H;
    // no more blocks than tiles of work: a block's share is at least one tile of RT rows (a 1024^2
    // detector-only frame: 128 blocks instead of 456, 5.05 -> 3.44 us per call; with the stretch
    // 17.3 -> 12.7 us); rasters with a wave's worth of tiles keep the full wave
    constexpr int64_t RT = (kConsumers / TC) * kRowsPerThread;
    grid = std::max<int64_t>(1, std::min(grid, (a.units + RT - 1) / RT));
    a.units_per_block = (a.units + grid - 1) / grid;
    if (programmatic) return cuda_status(launch_programmatic(k, dim3((unsigned)grid), dim3(kThreads), smem, st, a));
    k<<<(unsigned)grid, kThreads, smem, st>>>(a);
    return cuda_status(cudaGetLastError());
}

template <int MODE>
int launch_single(TmaArgs& a, int tc, cudaStream_t st, bool programmatic = false)
{
    switch (tc) {
    case 256: return launch_single_tc<256, MODE>(a, st, programmatic);
    case 128: return launch_single_tc<128, MODE>(a, st, programmatic);
    default: return launch_single_tc<64, MODE>(a, st, programmatic);
    }
}

template <int TC, int MODE>
int launch_batch_tc(BatchArgs& a, int grid, cudaStream_t st)
{
    auto k = k_tma_strip<TC, MODE, true, BatchArgs>;
    const size_t smem = (size_t)kTableOffset + table_bytes(MODE, a.max_bits);
    int64_t g = 0;
    int rc = grid_for(k, smem, 0, &g);  // raises the shared-memory limit on first use
    if (rc) return rc;
    k<<<(unsigned)grid, kThreads, smem, st>>>(a);
    return cuda_status(cudaGetLastError());
}

template <int TC, int MODE>
int batch_grid_tc(int max_bits, int blocks_per_sm)
{
    auto k = k_tma_strip<TC, MODE, true, BatchArgs>;
    const size_t smem = (size_t)kTableOffset + table_bytes(MODE, max_bits);
    int64_t g = 0;
    return grid_for(k, smem, blocks_per_sm, &g) == LUTC_OK ? (int)g : 0;
}

template <int MODE>
int launch_batch(BatchArgs& a, int tc, int grid, cudaStream_t st)
{
    switch (tc) {
    case 256: return launch_batch_tc<256, MODE>(a, grid, st);
    case 128: return launch_batch_tc<128, MODE>(a, grid, st);
    default: return launch_batch_tc<64, MODE>(a, grid, st);
    }
}

// Launches with work stealing (a.ranges): pass 1 and pass 2 of a batch.
template <int TC, int MODE>
int launch_batch_steal_tc(BatchArgs& a, int grid, cudaStream_t st)
{
    auto k = k_tma_strip<TC, MODE, true, BatchArgs, true>;
    const size_t smem = (size_t)kTableOffset + table_bytes(MODE, a.max_bits);
    int64_t g = 0;
    int rc = grid_for(k, smem, 0, &g);  // raises the shared-memory limit on first use
    if (rc) return rc;
    k<<<(unsigned)grid, kThreads, smem, st>>>(a);
    return cuda_status(cudaGetLastError());
}

template <int MODE>
int launch_batch_steal(BatchArgs& a, int tc, int grid, cudaStream_t st)
{
    switch (tc) {
    case 256: return launch_batch_steal_tc<256, MODE>(a, grid, st);
    case 128: return launch_batch_steal_tc<128, MODE>(a, grid, st);
    default: return launch_batch_steal_tc<64, MODE>(a, grid, st);
    }
}

template <int MODE>
int batch_grid(int tc, int max_bits, int blocks_per_sm)
{
    switch (tc) {
    case 256: return batch_grid_tc<256, MODE>(max_bits, blocks_per_sm);
    case 128: return batch_grid_tc<128, MODE>(max_bits, blocks_per_sm);
    default: return batch_grid_tc<64, MODE>(max_bits, blocks_per_sm);
    }
}

template <int TC>
int preload_tc()
{
    int64_t g = 0;
    int rc = LUTC_OK;
    for (int bits = LUTC_MIN_BITS; bits <= 15 && !rc; ++bits) {
        const size_t h = (size_t)kTableOffset + table_bytes(kHist, bits);
        const size_t t = (size_t)kTableOffset + table_bytes(kApplyStretch, bits);
        const size_t z = (size_t)kTableOffset;
        if (!rc) rc = grid_for(k_tma_strip<TC, kHist, false, TmaArgs>, h, 0, &g);
        if (!rc) rc = grid_for(k_tma_strip<TC, kHist, true, BatchArgs>, h, 0, &g);
        if (!rc) rc = grid_for(k_tma_strip<TC, kHist, true, BatchArgs, true>, h, 0, &g);
        if (!rc) rc = grid_for(k_tma_strip<TC, kApplyStretch, false, TmaArgs>, t, 0, &g);
        if (!rc) rc = grid_for(k_tma_strip<TC, kApplyStretch, true, BatchArgs>, t, 0, &g);
        if (!rc) rc = grid_for(k_tma_strip<TC, kApplyStretch, true, BatchArgs, true>, t, 0, &g);
        if (!rc) rc = grid_for(k_tma_strip<TC, kApplyDetector, false, TmaArgs>, z, 0, &g);
        if (!rc) rc = grid_for(k_tma_strip<TC, kApplyDetector, true, BatchArgs>, z, 0, &g);
    }
    if (!rc) rc = grid_for(k_tma_strip<TC, kHistGlobal, false, TmaArgs>, (size_t)kTableOffset, 0, &g);
    return rc;
}

}  // namespace

// Loads every TMA kernel variant and caches its occupancy, so that no launch pays a first-use
// cost (module loading, attribute change) in the middle of a latency-sensitive stream of work.
int tma_preload()
{
    int rc = preload_tc<64>();
    if (!rc) rc = preload_tc<128>();
    if (!rc) rc = preload_tc<256>();
    return rc;
}

int tma_box_rows(int column_threads) { return kTileBytes / (16 * column_threads); }

bool tma_encode(CUtensorMap* map, const lutc_raster* in, int column_threads)
{
    if (!encode_fn()) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)in->width, (cuuint64_t)in->bands * (cuuint64_t)in->height};
    const cuuint64_t strides[1] = {(cuuint64_t)in->pitch_bytes};
    const cuuint32_t box[2] = {256, (cuuint32_t)tma_box_rows(column_threads)};
    const cuuint32_t estr[2] = {1, 1};
    // Wide strips read 4 KB of each row per tile: letting L2 fill 256-byte blocks helps there.
    // Narrow strips of short, unaligned rows would pull in neighbouring bytes nobody reads.
    const CUtensorMapL2promotion promo =
        column_threads >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE;
    return encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<uint16_t*>(in->data), dims, strides, box,
                       estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_eligible(const lutc_raster* in)
{
    if (tuning_for(in->bits).path == LUTC_PATH_STRIP) return false;
    return in->width >= 256 && ((uintptr_t)in->data % 16 == 0) && (in->pitch_bytes % 16 == 0) &&
           (int64_t)in->bands * in->height < ((int64_t)1 << 31) && encode_fn() != nullptr;
}

// Builds the tensor map and the argument block shared by the passes of one image.
static int tma_args(const lutc_raster* in, const lutc_coeffs* per_band, int tc, TmaArgs& a)
{
    if (!tma_encode(&a.map, in, tc)) return LUTC_ECUDA;
    JobDesc& J = a.job;
    J.W = in->width;
    J.H = in->height;
    J.bits = in->bits;
    J.bands = in->bands;
    J.strips = 0;
    J.vout = 0;
    J.unit_begin = 0;
    J.out = nullptr;
    J.out_pitch = 0;
    J.hist_off = 0;
    J.S_off = 0;
    J.coef = nullptr;
    a.max_bits = in->bits;
    a.S = nullptr;
    a.hist = nullptr;
    for (int b = 0; b < LUTC_MAX_BANDS; ++b)
        a.coef[b] = b < in->bands ? BandCoef{per_band[b].A, per_band[b].G, per_band[b].O} : BandCoef{nullptr, nullptr, nullptr};
    return LUTC_OK;
}

int tma_hist(const lutc_raster* in, const lutc_coeffs* per_band, unsigned long long* hist, cudaStream_t st)
{
    TmaArgs a;
    const int tc = pick_tc(in->width, in->bits);
    int rc = tma_args(in, per_band, tc, a);
    if (rc) return rc;
    a.hist = hist;
    return in->bits <= 15 ? launch_single<kHist>(a, tc, st) : launch_single<kHistGlobal>(a, tc, st);
}

int tma_apply(const lutc_raster* in, const lutc_coeffs* per_band, const uint8_t* S, void* out, int64_t out_pitch,
              bool stretch, cudaStream_t st, bool programmatic)
{
    TmaArgs a;
    const int tc = pick_tc(in->width, in->bits);
    int rc = tma_args(in, per_band, tc, a);
    if (rc) return rc;
    a.job.out = reinterpret_cast<uint8_t*>(out);
    a.job.out_pitch = out_pitch;
    const int64_t vec = stretch ? 8 : 16;
    a.job.vout = ((uintptr_t)out % vec == 0) && (out_pitch % vec == 0);
    a.S = S;
    return stretch ? launch_single<kApplyStretch>(a, tc, st, programmatic) : launch_single<kApplyDetector>(a, tc, st);
}

int tma_batch_grid(int mode, int column_threads, int max_bits, int blocks_per_sm)
{
    switch (mode) {
    case kHist: return batch_grid<kHist>(column_threads, max_bits, blocks_per_sm);
    case kApplyStretch: return batch_grid<kApplyStretch>(column_threads, max_bits, blocks_per_sm);
    case kApplyDetector: return batch_grid<kApplyDetector>(column_threads, max_bits, blocks_per_sm);
    default: return 0;
    }
}

int tma_batch_pass(const BatchLaunch& b, int mode, int column_threads, int blocks_per_sm, cudaStream_t st)
{
    (void)blocks_per_sm;  // folded into b.grid and b.starts when the batch was planned
    if (b.units == 0 || b.grid <= 0) return LUTC_OK;
    BatchArgs a;
    a.jobs = b.jobs;
    a.maps = b.maps;
    a.njobs = b.njobs;
    a.max_bits = b.max_bits;
    a.unit_offset = b.unit_offset;
    a.units = b.units;
    a.units_per_block = 0;
    a.starts = b.starts;
    a.hist = b.hist;
    a.S = b.S;
    a.ranges = b.ranges;
    a.granule = b.granule > 0 ? b.granule : 8 * tma_box_rows(column_threads);
    if (b.ranges && mode == kHist) return launch_batch_steal<kHist>(a, column_threads, b.grid, st);
    if (b.ranges && mode == kApplyStretch) return launch_batch_steal<kApplyStretch>(a, column_threads, b.grid, st);
    switch (mode) {
    case kHist: return launch_batch<kHist>(a, column_threads, b.grid, st);
    case kApplyStretch: return launch_batch<kApplyStretch>(a, column_threads, b.grid, st);
    case kApplyDetector: return launch_batch<kApplyDetector>(a, column_threads, b.grid, st);
    default: return LUTC_EUNSUPPORTED;
    }
}

}  // namespace lutc

namespace lutc {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

// Device address of this library's kernel status word on the current device (for kernels of other files).
int* device_status_ptr()
{
    static int* ptrs[64] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs[dev] = reinterpret_cast<int*>(p);
    }
    return ptrs[dev];
}
}  // namespace lutc

namespace lutc {
namespace {
// one thread waits on a barrier that expects an arrival nobody makes
__global__ void k_selftest_wait(long long cycles)
{
    __shared__ uint64_t bar;
    ptx::mbar_init(&bar, 1);
    ptx::fence_mbar_init();
    ptx::mbar_wait_bounded(&bar, 0, &g_device_status, cycles);
}
}  // namespace
}  // namespace lutc

extern "C" int lutc_selftest_wait_timeout(long long wait_cycles, lutc_stream stream)
{
    if (wait_cycles < 1 || wait_cycles > (1ll << 31)) return LUTC_EINVAL;
    lutc::k_selftest_wait<<<1, 1, 0, (cudaStream_t)stream>>>(wait_cycles);
    return lutc::cuda_status(cudaGetLastError());
}

extern "C" int lutc_device_status(int* status, lutc_stream stream)
{
    if (!status) return LUTC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, lutc::g_device_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LUTC_ECUDA;
    const int zero = 0;
    if (v != 0 && cudaMemcpyToSymbolAsync(lutc::g_device_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) !=
                      cudaSuccess)
        return LUTC_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LUTC_ECUDA;
    *status = v;
    return LUTC_OK;
}
