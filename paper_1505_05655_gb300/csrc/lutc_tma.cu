// TMA-staged, persistent strip kernels of the fused correction (sm_103a).
//
// Section I of the paper names LUT generation and image correction as a task
// the GPU server runs on a client's raster.  This file is the fast path of
// that task for rasters whose base and row pitch are 16-byte aligned and
// whose width is at least 256 columns; other rasters take the plain strip
// kernels of lutc_correct.cu.  Both produce identical results.
//
// Block = 16 consumer warps + 1 producer warp, one block per SM, persistent.
//  * Work: the raster is cut into column strips of 8 * TC columns (TC column
//    threads, each owning 8 adjacent detectors); the (band, strip, row)
//    space is laid out linearly and every block takes an equal contiguous
//    share of it, so the grid is exactly one wave and balanced to a row.
//  * Producer: one thread streams tiles of (1024 / TC) rows x (8 TC) columns
//    (16 KB) into a 6-stage shared-memory ring with 2-D tensor TMA loads
//    (cp.async.bulk.tensor), completion counted on a per-stage mbarrier;
//    96 KB are in flight per SM independent of register pressure.  Columns
//    past the image edge and rows past the raster are zero-filled by TMA and
//    ignored by the consumers.
//  * Consumers: each thread reads its 8 pixels of a row (one 16-byte shared
//    load), clamps them with a packed 16x2 min, evaluates step (L) in
//    wrap-around int32 (Horner form x (A x + G) + O + 2^15, exact when the
//    column bound |A| M^2 + |G| M + |O + 2^15| < 2^31 holds) and then
//      pass 1: increments a shared-memory histogram replicated R times with
//              the copy chosen by lane (copy c holds bin v at word v R + c, so
//              lanes of different copies never collide on an address and
//              rarely on a bank); at each band change and at the end the
//              copies are summed into the band's global uint64 histogram;
//      pass 2: looks up S[D] in the band's stretch table in shared memory and
//              stores 8 output bytes per row (detector-only: 16 bytes of D).
//  * Every wait is bounded (about two seconds of clock); on expiry the block
//    records LUTC_ETIMEOUT in the library's device status word, the producer
//    waits (bounded) for its copies in flight, and the block returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "lutc_internal.cuh"

namespace lutc {

int launch_stretch(const unsigned long long* hist, int bands, int bits, uint8_t* S, int32_t* lohi, cudaStream_t st);

namespace {

constexpr int kConsumers = 256;            // consumer threads per block (8 warps)
constexpr int kThreads = kConsumers + 32;  // + one producer warp
constexpr int kConsumerWarps = kConsumers / 32;
constexpr int kStages = 3;
constexpr int kRowsPerThread = 4;          // rows of a tile each consumer thread processes
constexpr int kTileBytes = kConsumers * 16 * kRowsPerThread;  // 16 KB
constexpr int kRingBytes = kStages * kTileBytes;
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

enum Mode { kHist = 0, kHistGlobal = 1, kApplyStretch = 2, kApplyDetector = 3 };

__device__ int g_device_status;  // 0, or the first error a kernel of this library recorded

struct TmaArgs {
    CUtensorMap map;  // uint16 [bands * H][W], row stride = pitch, box {256, rows per tile}
    int W, H, bits, bands;
    int strips;
    int64_t units;
    int64_t units_per_block;
    uint8_t* out;
    int64_t out_pitch;
    int vout;
    const uint8_t* S;
    unsigned long long* hist;
    BandCoef coef[LUTC_MAX_BANDS];
};

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, TMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity; false after ~2 s (status recorded).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity);

// Barrier among the consumer threads only (the producer runs ahead), bounded like every wait.
__device__ __forceinline__ bool consumer_sync(uint64_t* bar, uint32_t& phase)
{
    mbar_arrive(bar);
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    return ok;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicCAS(&g_device_status, 0, LUTC_ETIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// per-pixel arithmetic
// ---------------------------------------------------------------------------
// (L) in wrap-around int32, Horner form; exact for an int32-exact column (Op = O + 2^15)
__device__ __forceinline__ uint32_t det_horner(int32_t A, int32_t G, int32_t Op, uint32_t x, int32_t M)
{
    const uint32_t t = ((uint32_t)A * x + (uint32_t)G) * x + (uint32_t)Op;
    return (uint32_t)__vimin_s32_relu(((int32_t)t) >> 16, M);  // clamp(floor(t / 2^16), 0, M)
}

// (P) clamp of raw DN to M, two pixels per 32-bit word
__device__ __forceinline__ void unpack_clamped(const uint4 v, uint32_t M2, uint32_t (&x)[8])
{
    const uint32_t w0 = __vminu2(v.x, M2), w1 = __vminu2(v.y, M2), w2 = __vminu2(v.z, M2), w3 = __vminu2(v.w, M2);
    x[0] = w0 & 0xffffu; x[1] = w0 >> 16;
    x[2] = w1 & 0xffffu; x[3] = w1 >> 16;
    x[4] = w2 & 0xffffu; x[5] = w2 >> 16;
    x[6] = w3 & 0xffffu; x[7] = w3 >> 16;
}

template <int TC, int MODE>
__global__ void __launch_bounds__(kThreads) k_tma_strip(const __grid_constant__ TmaArgs a)
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
    unsigned char* table = smem + kRingBytes + 128;
    uint32_t* hs = reinterpret_cast<uint32_t*>(table);

    const int tid = threadIdx.x;
    const int L = 1 << a.bits;
    const int32_t M = L - 1;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        mbar_init(csync, kConsumers);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (MODE == kHist)
        for (int i = tid; i < L; i += kThreads) hs[i] = 0;
    __syncthreads();

    // This block's share of the (band, strip, row) space, walked without divisions.
    const int64_t u0 = (int64_t)blockIdx.x * a.units_per_block;
    const int64_t u1 = min(a.units, u0 + a.units_per_block);
    if (u0 >= u1) return;
    int64_t left = u1 - u0;
    const int64_t seg0 = u0 / a.H;
    int row = (int)(u0 - seg0 * a.H);
    int band = (int)(seg0 / a.strips);
    int strip = (int)(seg0 - (int64_t)band * a.strips);
    int stage = 0;
    uint32_t phase = 0;

    if (tid >= kConsumers) {
        // ------------------------------------------------------------ producer
        if (tid != kConsumers) return;
        int issued = 0;
        bool ok = true;
        while (left > 0) {
            const int nrows = (int)min((int64_t)min(RT, a.H - row), left);
            if (issued >= kStages && !mbar_wait(&empty[stage], phase ^ 1u)) {
                ok = false;
                break;
            }
            const int x0 = strip * SW;
            const int nb = min(NB, (a.W - x0 + 255) >> 8);
            mbar_arrive_expect_tx(&full[stage], (uint32_t)(nb * 512 * RT));
            unsigned char* dst = ring + stage * kTileBytes;
            const int y = band * a.H + row;
            for (int b = 0; b < nb; ++b) tma_load_2d(dst + b * (RT * 512), &a.map, &full[stage], x0 + b * 256, y);
            ++issued;
            left -= nrows;
            row += nrows;
            if (row == a.H) {
                row = 0;
                if (++strip == a.strips) { strip = 0; ++band; }
            }
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
        if (!ok) {
            // let every copy issued land before the block's shared memory goes away
            for (int j = 0; j < kStages && j < issued; ++j) {
                if (--stage < 0) { stage = kStages - 1; phase ^= 1u; }
                mbar_wait(&full[stage], phase);
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ct = tid % TC;  // column thread: owns columns strip * SW + ct * 8 .. + 7
    const int ph = tid / TC;  // row phase
    const int lane = tid & 31;
    const uint32_t M2 = (uint32_t)M | ((uint32_t)M << 16);
    const unsigned char* my = ring + (ct >> 5) * (RT * 512) + (ct & 31) * 16 + ph * 512;
    uint32_t sync_phase = 0;
    bool new_seg = true;
    int cur_band = -1;
    int32_t A[8], G[8], O[8];
    bool fits = true;
    int n = 0, c0 = 0;
    while (left > 0) {
        const int nrows = (int)min((int64_t)min(RT, a.H - row), left);
        if (new_seg) {
            if (band != cur_band) {
                if (MODE == kHist && cur_band >= 0) {
                    // every consumer is done with the previous band: flush it and clear
                    if (!consumer_sync(csync, sync_phase)) return;
                    unsigned long long* hb = a.hist + (int64_t)cur_band * L;
                    for (int i = tid; i < L; i += kConsumers) {
                        const uint32_t c = hs[i];
                        if (c) {
                            atomicAdd(hb + i, (unsigned long long)c);
                            hs[i] = 0;
                        }
                    }
                    if (!consumer_sync(csync, sync_phase)) return;
                }
                if (MODE == kApplyStretch) {
                    if (cur_band >= 0 && !consumer_sync(csync, sync_phase)) return;
                    const uint4* src = reinterpret_cast<const uint4*>(a.S + (int64_t)band * L);
                    for (int i = tid; i < L / 16; i += kConsumers) reinterpret_cast<uint4*>(table)[i] = src[i];
                    if (!consumer_sync(csync, sync_phase)) return;
                }
                cur_band = band;
            }
            new_seg = false;
            c0 = strip * SW + ct * 8;
            n = min(8, a.W - c0);
            fits = true;
            const BandCoef& cf = a.coef[band];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j < n) {
                    A[j] = __ldg(cf.A + c0 + j);
                    G[j] = __ldg(cf.G + c0 + j);
                    O[j] = __ldg(cf.O + c0 + j);
                    fits = fits && col_fits_i32(A[j], G[j], O[j], M);
                } else {
                    A[j] = 0; G[j] = 0; O[j] = 0;
                }
            }
            if (fits) {
#pragma unroll
                for (int j = 0; j < 8; ++j) O[j] += 32768;
            }
        }
        if (!mbar_wait(&full[stage], phase)) return;
        const unsigned char* tile = my + stage * kTileBytes;
        const int64_t orow0 = (int64_t)band * a.H + row + ph;
        if (n == 8 && fits) {
#pragma unroll
            for (int i = 0; i < kRowsPerThread; ++i) {
                if (ph + i * P < nrows) {
                    const uint4 v = *reinterpret_cast<const uint4*>(tile + i * P * 512);
                    uint32_t x[8], d[8];
                    unpack_clamped(v, M2, x);
#pragma unroll
                    for (int j = 0; j < 8; ++j) d[j] = det_horner(A[j], G[j], O[j], x[j], M);
                    if (MODE == kHist) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) atomicAdd(hs + d[j], 1u);
                    } else if (MODE == kHistGlobal) {
                        unsigned long long* hb = a.hist + (int64_t)band * L;
#pragma unroll
                        for (int j = 0; j < 8; ++j) atomicAdd(hb + d[j], 1ull);
                    } else if (MODE == kApplyStretch) {
                        uint32_t o[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) o[j] = table[d[j]];
                        uint8_t* dst = a.out + (orow0 + i * P) * a.out_pitch + c0;
                        uint2 r;
                        r.x = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
                        r.y = o[4] | (o[5] << 8) | (o[6] << 16) | (o[7] << 24);
                        if (a.vout) {
                            *reinterpret_cast<uint2*>(dst) = r;
                        } else {
#pragma unroll
                            for (int j = 0; j < 8; ++j) dst[j] = (uint8_t)o[j];
                        }
                    } else {
                        uint8_t* dst = a.out + (orow0 + i * P) * a.out_pitch + (int64_t)c0 * 2;
                        if (a.vout) {
                            uint4 r;
                            r.x = d[0] | (d[1] << 16); r.y = d[2] | (d[3] << 16);
                            r.z = d[4] | (d[5] << 16); r.w = d[6] | (d[7] << 16);
                            *reinterpret_cast<uint4*>(dst) = r;
                        } else {
#pragma unroll
                            for (int j = 0; j < 8; ++j) reinterpret_cast<uint16_t*>(dst)[j] = (uint16_t)d[j];
                        }
                    }
                }
            }
        } else if (n > 0) {
            // right-edge chunk or a column that needs int64: exact, slow, few registers
            const BandCoef& cf = a.coef[band];
#pragma unroll 1
            for (int i = 0; i < kRowsPerThread; ++i) {
                if (ph + i * P >= nrows) break;
                const uint16_t* px = reinterpret_cast<const uint16_t*>(tile + i * P * 512);
                const int64_t orow = orow0 + i * P;
#pragma unroll 1
                for (int j = 0; j < n; ++j) {
                    const uint32_t x = min((uint32_t)px[j], (uint32_t)M);
                    const uint32_t d = det_i64(__ldg(cf.A + c0 + j), __ldg(cf.G + c0 + j), __ldg(cf.O + c0 + j), x, M);
                    if (MODE == kHist) atomicAdd(hs + d, 1u);
                    else if (MODE == kHistGlobal) atomicAdd(a.hist + (int64_t)band * L + d, 1ull);
                    else if (MODE == kApplyStretch) a.out[orow * a.out_pitch + c0 + j] = table[d];
                    else reinterpret_cast<uint16_t*>(a.out + orow * a.out_pitch)[c0 + j] = (uint16_t)d;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[stage]);
        left -= nrows;
        row += nrows;
        if (row == a.H) {
            row = 0;
            new_seg = true;
            if (++strip == a.strips) { strip = 0; ++band; }
        }
        if (++stage == kStages) { stage = 0; phase ^= 1u; }
    }
    if (MODE == kHist && cur_band >= 0) {
        if (!consumer_sync(csync, sync_phase)) return;
        unsigned long long* hb = a.hist + (int64_t)cur_band * L;
        for (int i = tid; i < L; i += kConsumers) {
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

template <int TC, int MODE>
int launch_tc(TmaArgs& a, cudaStream_t st)
{
    auto k = k_tma_strip<TC, MODE>;
    const size_t L = (size_t)1 << a.bits;
    const size_t table = MODE == kHist ? L * 4 : (MODE == kApplyStretch ? L : 0);
    const size_t smem = (size_t)kRingBytes + 128 + table;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LUTC_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess || per_sm < 1)
        return LUTC_ECUDA;
    constexpr int SW = 8 * TC;
    a.strips = (a.W + SW - 1) / SW;
    a.units = (int64_t)a.bands * a.strips * a.H;
    const int cap = tuning_for(a.bits).blocks_per_sm;
    if (cap > 0 && cap < per_sm) per_sm = cap;
    const int64_t grid = (int64_t)sm_count() * per_sm;
    a.units_per_block = (a.units + grid - 1) / grid;
    k<<<(unsigned)grid, kThreads, smem, st>>>(a);
    return cuda_status(cudaGetLastError());
}

template <int MODE>
int launch_mode(TmaArgs& a, cudaStream_t st)
{
    switch (pick_tc(a.W, a.bits)) {
    case 256: return launch_tc<256, MODE>(a, st);
    case 128: return launch_tc<128, MODE>(a, st);
    default: return launch_tc<64, MODE>(a, st);
    }
}

}  // namespace

bool tma_eligible(const lutc_raster* in)
{
    if (tuning_for(in->bits).path == LUTC_PATH_STRIP) return false;
    return in->width >= 256 && ((uintptr_t)in->data % 16 == 0) && (in->pitch_bytes % 16 == 0) &&
           (int64_t)in->bands * in->height < ((int64_t)1 << 31) && encode_fn() != nullptr;
}

// Builds the tensor map and the argument block shared by the three passes.
static int tma_args(const lutc_raster* in, const lutc_coeffs* per_band, TmaArgs& a)
{
    const int TC = pick_tc(in->width, in->bits);
    const int RT = kTileBytes / (16 * TC);  // rows per tile = (kConsumers / TC) * kRowsPerThread
    const cuuint64_t dims[2] = {(cuuint64_t)in->width, (cuuint64_t)in->bands * (cuuint64_t)in->height};
    const cuuint64_t strides[1] = {(cuuint64_t)in->pitch_bytes};
    const cuuint32_t box[2] = {256, (cuuint32_t)RT};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&a.map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<uint16_t*>(in->data), dims,
                                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return LUTC_ECUDA;
    a.W = in->width;
    a.H = in->height;
    a.bits = in->bits;
    a.bands = in->bands;
    a.out = nullptr;
    a.out_pitch = 0;
    a.vout = 0;
    a.S = nullptr;
    a.hist = nullptr;
    for (int b = 0; b < LUTC_MAX_BANDS; ++b)
        a.coef[b] = b < in->bands ? BandCoef{per_band[b].A, per_band[b].G, per_band[b].O} : BandCoef{nullptr, nullptr, nullptr};
    return LUTC_OK;
}

int tma_hist(const lutc_raster* in, const lutc_coeffs* per_band, unsigned long long* hist, cudaStream_t st)
{
    TmaArgs a;
    int rc = tma_args(in, per_band, a);
    if (rc) return rc;
    a.hist = hist;
    return in->bits <= 15 ? launch_mode<kHist>(a, st) : launch_mode<kHistGlobal>(a, st);
}

int tma_apply(const lutc_raster* in, const lutc_coeffs* per_band, const uint8_t* S, void* out, int64_t out_pitch,
              bool stretch, cudaStream_t st)
{
    TmaArgs a;
    int rc = tma_args(in, per_band, a);
    if (rc) return rc;
    a.out = reinterpret_cast<uint8_t*>(out);
    a.out_pitch = out_pitch;
    const int64_t vec = stretch ? 8 : 16;
    a.vout = ((uintptr_t)out % vec == 0) && (out_pitch % vec == 0);
    a.S = S;
    return stretch ? launch_mode<kApplyStretch>(a, st) : launch_mode<kApplyDetector>(a, st);
}

}  // namespace lutc

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
