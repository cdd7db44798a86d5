// The per-call ("plain") steps with materialised tables: lutgen (L),
// apply_u16 (P), stretch (S), compose (C) and apply_u8 (A).
//
// Section I of the paper names LUT generation and image correction as a task
// a client submits; these entry points expose each step of it on its own, so
// a caller can keep, inspect or reuse the tables.  The fused, table-free path
// lives in lutc_correct.cu.
#include <stdint.h>

#include "lutc_internal.cuh"
#include "lutc_ptx.cuh"

namespace lutc {
namespace {

// ---------------------------------------------------------------------------
// (L): one thread writes 8 consecutive entries (16 bytes) of one column.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_lutgen(BandCoef c, int ncols, int bits, uint16_t* __restrict__ lut)
{
    const int32_t M = (1 << bits) - 1;
    const int64_t chunks = (int64_t)ncols << (bits - 3);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < chunks; i += stride) {
        const int col = (int)(i >> (bits - 3));
        const uint32_t x0 = (uint32_t)(i & ((1 << (bits - 3)) - 1)) << 3;
        const int32_t A = __ldg(c.A + col), G = __ldg(c.G + col), O = __ldg(c.O + col);
        uint32_t d[8];
        if (col_fits_i32(A, G, O, M)) {
            const int32_t Op = O + 32768;
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] = det_i32(A, G, Op, x0 + j, M);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] = det_i64(A, G, O, x0 + j, M);
        }
        uint4 v;
        v.x = d[0] | (d[1] << 16);
        v.y = d[2] | (d[3] << 16);
        v.z = d[4] | (d[5] << 16);
        v.w = d[6] | (d[7] << 16);
        reinterpret_cast<uint4*>(lut)[i] = v;
    }
}

// ---------------------------------------------------------------------------
// (P) and (A) with a table in global memory: one thread per 8-pixel chunk of
// a row; rows of all bands are walked by the grid's y dimension (planar
// layout: row r = b * H + y starts at r * pitch).
// ---------------------------------------------------------------------------
template <typename OutT>
__global__ void __launch_bounds__(128) k_apply_table(const uint8_t* __restrict__ in, int64_t in_pitch, int W, int H,
                                                     int bands, int bits, const OutT* __restrict__ table,
                                                     uint8_t* __restrict__ out, int64_t out_pitch, bool vin, bool vout)
{
    const int64_t L = (int64_t)1 << bits;
    const uint32_t M = (uint32_t)L - 1;
    const int chunk = blockIdx.x * blockDim.x + threadIdx.x;
    const int c0 = chunk * 8;
    if (c0 >= W) return;
    const int n = min(8, W - c0);
    const int64_t rows = (int64_t)bands * H;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const int b = (int)(r / H);
        const OutT* tb = table + ((int64_t)b * W + c0) * L;
        const uint8_t* src = in + r * in_pitch + (int64_t)c0 * 2;
        OutT* dst = reinterpret_cast<OutT*>(out + r * out_pitch) + c0;
        uint32_t x[8];
        if (n == 8 && vin) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
            x[0] = v.x & 0xffff; x[1] = v.x >> 16; x[2] = v.y & 0xffff; x[3] = v.y >> 16;
            x[4] = v.z & 0xffff; x[5] = v.z >> 16; x[6] = v.w & 0xffff; x[7] = v.w >> 16;
        } else {
            const uint16_t* s16 = reinterpret_cast<const uint16_t*>(src);
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = j < n ? (uint32_t)__ldg(s16 + j) : 0u;
        }
        uint32_t o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = j < n ? (uint32_t)__ldg(tb + j * L + min(x[j], M)) : 0u;
        if (n == 8 && vout) {
            if (sizeof(OutT) == 2) {
                uint4 v;
                v.x = o[0] | (o[1] << 16); v.y = o[2] | (o[3] << 16);
                v.z = o[4] | (o[5] << 16); v.w = o[6] | (o[7] << 16);
                *reinterpret_cast<uint4*>(dst) = v;
            } else {
                uint2 v;
                v.x = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
                v.y = o[4] | (o[5] << 8) | (o[6] << 16) | (o[7] << 24);
                *reinterpret_cast<uint2*>(dst) = v;
            }
        } else {
            for (int j = 0; j < n; ++j) dst[j] = (OutT)o[j];
        }
    }
}

// ---------------------------------------------------------------------------
// (S): one block per band.  Each thread owns a contiguous run of bins; a
// block-wide scan of the run totals gives each run its starting cdf, and the
// first bin of each threshold crossing is found by a block-wide minimum.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// (S) for one band's histogram h (2^bits bins): writes S (2^bits bytes) and lohi[0..1].
// Called by all kScanThreads threads of a block; PER = bins per thread (2^bits / kScanThreads, at
// least 1), so a thread's run lies wholly inside [0, 2^bits) or wholly past it.  The run is read by
// independent loads, CH bins at a time, kept in registers when the whole run fits (CH = PER).
template <int PER>
__device__ __forceinline__ void stretch_band(const unsigned long long* __restrict__ h, int bits,
                                             uint8_t* __restrict__ S, int32_t* __restrict__ lohi)
{
    constexpr int CH = PER < 16 ? PER : 16;
    constexpr int NCH = PER / CH;
    __shared__ unsigned long long warp_tot[kScanThreads / 32];
    __shared__ int s_lo, s_hi;
    const int L = 1 << bits;
    const int v0 = (int)threadIdx.x * PER;
    // pairs of bins by 16-byte loads when the histogram allows it (runs start on even bins)
    const bool vec = PER >= 2 && (reinterpret_cast<uintptr_t>(h) & 15) == 0;
    unsigned long long c[CH];
    auto load = [&](int v) {
        if (v >= L) {
#pragma unroll
            for (int k = 0; k < CH; ++k) c[k] = 0;
        } else if (vec) {
#pragma unroll
            for (int k = 0; k < CH; k += 2) {
                const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2*>(h + v + k));
                c[k] = w.x;
                c[k + 1] = w.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < CH; ++k) c[k] = __ldg(h + v + k);
        }
    };
    unsigned long long run = 0;
    for (int ch = 0; ch < NCH; ++ch) {
        load(v0 + ch * CH);
#pragma unroll
        for (int k = 0; k < CH; ++k) run += c[k];
    }
    // block-wide inclusive scan of the run totals
    unsigned long long inc = warp_incl_scan(run);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) warp_tot[warp] = inc;
    if (threadIdx.x == 0) { s_lo = L; s_hi = L; }
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = warp_tot[lane];
        t = warp_incl_scan(t);
        warp_tot[lane] = t;
    }
    __syncthreads();
    const unsigned long long before = (warp > 0 ? warp_tot[warp - 1] : 0ull) + inc - run;
    const unsigned long long N = warp_tot[kScanThreads / 32 - 1];

    // first v of this run with 100 cdf(v) >= 2N (resp. 98N)
    unsigned long long cdf = before;
    int my_lo = L, my_hi = L;
    for (int ch = 0; ch < NCH; ++ch) {
        if (NCH > 1) load(v0 + ch * CH);  // a single chunk is still in c
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            cdf += c[k];
            if (my_lo == L && 100ull * cdf >= 2ull * N) my_lo = v0 + ch * CH + k;
            if (my_hi == L && 100ull * cdf >= 98ull * N) my_hi = v0 + ch * CH + k;
        }
    }
    if (v0 < L) {
        if (my_lo < L) atomicMin(&s_lo, my_lo);
        if (my_hi < L) atomicMin(&s_hi, my_hi);
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi;
    if (threadIdx.x == 0) {
        lohi[0] = lo;
        lohi[1] = hi;
    }
    // S[v] = clamp(((v - lo) 255 + (hi - lo) / 2) / (hi - lo), 0, 255), C division (truncation);
    // |v - lo| < 2^16, so the numerator fits int32 and the 32-bit quotient is the int64 one
    const int span = hi - lo;
    for (int v = threadIdx.x; v < L; v += kScanThreads) {
        int q = 0;
        if (span != 0) {
            q = ((v - lo) * 255 + span / 2) / span;
            q = q < 0 ? 0 : (q > 255 ? 255 : q);
        }
        S[v] = (uint8_t)q;
    }
}

// Runs stretch_band with the run length of `bits`.
__device__ __forceinline__ void stretch_band_bits(const unsigned long long* __restrict__ h, int bits,
                                                  uint8_t* __restrict__ S, int32_t* __restrict__ lohi)
{
    static_assert(kScanThreads == 1024, "run lengths below assume 1024 threads");
    switch (bits) {
    case 16: stretch_band<64>(h, bits, S, lohi); break;
    case 15: stretch_band<32>(h, bits, S, lohi); break;
    case 14: stretch_band<16>(h, bits, S, lohi); break;
    case 13: stretch_band<8>(h, bits, S, lohi); break;
    case 12: stretch_band<4>(h, bits, S, lohi); break;
    case 11: stretch_band<2>(h, bits, S, lohi); break;
    default: stretch_band<1>(h, bits, S, lohi); break;  // 8..10 bits
    }
}

__global__ void __launch_bounds__(kScanThreads) k_stretch(const unsigned long long* __restrict__ hist, int bits,
                                                          uint8_t* __restrict__ S, int32_t* __restrict__ lohi)
{
    // launched right behind pass 1 (programmatic launch): let pass 2 launch behind this grid, then wait
    // for pass 1's histogram
    ptx::launch_dependents();
    ptx::wait_prerequisites();
    const int64_t L = (int64_t)1 << bits;
    const int b = blockIdx.x;
    stretch_band_bits(hist + b * L, bits, S + b * L, lohi + 2 * b);
}

// One block per (image, band) of a batch, each with its own bit depth and table offsets.
__global__ void __launch_bounds__(kScanThreads) k_stretch_batch(const TableDesc* __restrict__ t,
                                                                const unsigned long long* __restrict__ hist,
                                                                uint8_t* __restrict__ S, int32_t* __restrict__ lohi)
{
    const TableDesc d = t[blockIdx.x];
    stretch_band_bits(hist + d.hist_off, d.bits, S + d.S_off, lohi + d.lohi_off);
}

// ---------------------------------------------------------------------------
// (C): clut[i] = S[min(lut[i], M)], 8 entries per thread.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_compose(const uint16_t* __restrict__ lut, const uint8_t* __restrict__ S,
                                                 int64_t chunks, int bits, uint8_t* __restrict__ clut)
{
    const uint32_t M = (1u << bits) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < chunks; i += stride) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(lut) + i);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint32_t o[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[2 * k] = __ldg(S + min(w[k] & 0xffffu, M));
            o[2 * k + 1] = __ldg(S + min(w[k] >> 16, M));
        }
        uint2 r;
        r.x = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
        r.y = o[4] | (o[5] << 8) | (o[6] << 16) | (o[7] << 24);
        reinterpret_cast<uint2*>(clut)[i] = r;
    }
}

int grid_for(int64_t work_items, int threads)
{
    const int64_t want = (work_items + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 16;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

template <typename OutT>
int launch_apply_table(const lutc_raster* in, const OutT* table, void* out, int64_t out_pitch, cudaStream_t st)
{
    int rc = check_raster(in);
    if (rc) return rc;
    if (!table || !out) return LUTC_EINVAL;
    if ((int64_t)in->width * in->height == 0) return LUTC_OK;
    if (out_pitch < (int64_t)sizeof(OutT) * in->width || out_pitch % (int64_t)sizeof(OutT)) return LUTC_EINVAL;
    const bool vin = ((uintptr_t)in->data % 16 == 0) && (in->pitch_bytes % 16 == 0);
    const size_t vec = sizeof(OutT) * 8;
    const bool vout = ((uintptr_t)out % vec == 0) && (out_pitch % (int64_t)vec == 0);
    const int chunks = (in->width + 7) / 8;
    const int threads = 128;
    dim3 grid((chunks + threads - 1) / threads, 1, 1);
    const int64_t rows = (int64_t)in->bands * in->height;
    const int64_t want_y = ((int64_t)sm_count() * 16 + grid.x - 1) / grid.x;
    grid.y = (unsigned)(rows < want_y ? rows : (want_y > 65535 ? 65535 : want_y));
    k_apply_table<OutT><<<grid, threads, 0, st>>>(reinterpret_cast<const uint8_t*>(in->data), in->pitch_bytes,
                                                  in->width, in->height, in->bands, in->bits, table,
                                                  reinterpret_cast<uint8_t*>(out), out_pitch, vin, vout);
    return cuda_status(cudaGetLastError());
}

}  // namespace

int launch_stretch(const unsigned long long* hist, int bands, int bits, uint8_t* S, int32_t* lohi, cudaStream_t st,
                   bool programmatic)
{
    if (!programmatic) {
        k_stretch<<<bands, kScanThreads, 0, st>>>(hist, bits, S, lohi);
        return cuda_status(cudaGetLastError());
    }
    return cuda_status(launch_programmatic(k_stretch, dim3(bands), dim3(kScanThreads), 0, st, hist, bits, S, lohi));
}

int tables_preload()
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_stretch) != cudaSuccess) return LUTC_ECUDA;
    if (cudaFuncGetAttributes(&fa, k_stretch_batch) != cudaSuccess) return LUTC_ECUDA;
    return LUTC_OK;
}

int stretch_batch(const TableDesc* tables, int ntables, const unsigned long long* hist, uint8_t* S, int32_t* lohi,
                  cudaStream_t st)
{
    if (ntables <= 0) return LUTC_OK;
    k_stretch_batch<<<ntables, kScanThreads, 0, st>>>(tables, hist, S, lohi);
    return cuda_status(cudaGetLastError());
}

}  // namespace lutc

using namespace lutc;

extern "C" int lutc_lutgen(const lutc_coeffs* coeffs, int bits, uint16_t* lut, lutc_stream stream)
{
    if (!coeffs || bits < LUTC_MIN_BITS || bits > LUTC_MAX_BITS || coeffs->ncols < 0) return LUTC_EINVAL;
    if (coeffs->ncols == 0) return LUTC_OK;
    if (!lut || !coeffs->A || !coeffs->G || !coeffs->O || ((uintptr_t)lut % 16)) return LUTC_EINVAL;
    const BandCoef c{coeffs->A, coeffs->G, coeffs->O};
    const int64_t chunks = (int64_t)coeffs->ncols << (bits - 3);
    k_lutgen<<<grid_for(chunks, 256), 256, 0, (cudaStream_t)stream>>>(c, coeffs->ncols, bits, lut);
    return cuda_status(cudaGetLastError());
}

extern "C" int lutc_apply_u16(const lutc_raster* in, const uint16_t* lut, uint16_t* out, int64_t out_pitch_bytes,
                              lutc_stream stream)
{
    return launch_apply_table<uint16_t>(in, lut, out, out_pitch_bytes, (cudaStream_t)stream);
}

extern "C" int lutc_apply_u8(const lutc_raster* in, const uint8_t* clut, uint8_t* out, int64_t out_pitch_bytes,
                             lutc_stream stream)
{
    return launch_apply_table<uint8_t>(in, clut, out, out_pitch_bytes, (cudaStream_t)stream);
}

extern "C" int lutc_stretch(const uint64_t* hist, int bands, int bits, uint8_t* S, int32_t* lohi, lutc_stream stream)
{
    if (!hist || !S || !lohi || bands < 1 || bands > LUTC_MAX_BANDS || bits < LUTC_MIN_BITS || bits > LUTC_MAX_BITS)
        return LUTC_EINVAL;
    return launch_stretch(reinterpret_cast<const unsigned long long*>(hist), bands, bits, S, lohi,
                          (cudaStream_t)stream);
}

extern "C" int lutc_compose(const uint16_t* lut, const uint8_t* S, int ncols, int bits, uint8_t* clut,
                            lutc_stream stream)
{
    if (ncols < 0 || bits < LUTC_MIN_BITS || bits > LUTC_MAX_BITS) return LUTC_EINVAL;
    if (ncols == 0) return LUTC_OK;
    if (!lut || !S || !clut || ((uintptr_t)lut % 16) || ((uintptr_t)clut % 8)) return LUTC_EINVAL;
    const int64_t chunks = (int64_t)ncols << (bits - 3);
    k_compose<<<grid_for(chunks, 256), 256, 0, (cudaStream_t)stream>>>(lut, S, chunks, bits, clut);
    return cuda_status(cudaGetLastError());
}
