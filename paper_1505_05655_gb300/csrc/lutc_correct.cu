// The fused, table-free correction: lutc_hist and lutc_correct_image.
//
// Section I of the paper names LUT generation and image correction as one
// task a client ships to the GPU server.  Materialising every detector's LUT
// costs more memory traffic than the image itself at 14 bits (2^14 entries x
// 2 bytes per column against 2 bytes per pixel of a column), so the fused
// path never writes a LUT: each thread owns 8 adjacent columns (detectors),
// keeps their Q16 coefficients in registers and evaluates step (L) per pixel
// with 32-bit integer arithmetic where that is exact (int64 otherwise).
//
//   pass 1  (k_strip_hist)   raw uint16 -> D -> block-private shared-memory
//                            histogram -> merged into the band's global uint64
//                            histogram at block exit                    (H)
//   scan    (k_stretch)      histogram -> lo, hi, S                      (S)
//   pass 2  (k_strip_apply)  raw uint16 -> D -> S[D] in shared memory -> uint8
//                            (steps C and A without the composed table)
//
// Work decomposition: block (strip, rowgroup, band) covers 8 * T columns and a
// contiguous range of rows of one band; a warp reads 512 contiguous bytes per
// row with 16-byte loads.  Without the stretch flag a single pass writes the
// uint16 corrected raster (P).
#include <stdint.h>

#include <new>

#include "lutc_internal.cuh"

namespace lutc {

bool tma_eligible(const lutc_raster* in);
int tma_hist(const lutc_raster* in, const lutc_coeffs* per_band, unsigned long long* hist, cudaStream_t st);
// programmatic: pass 2 launched right behind the scan of the same call (lutc_correct_image only)
int tma_apply(const lutc_raster* in, const lutc_coeffs* per_band, const uint8_t* S, void* out, int64_t out_pitch,
              bool stretch, cudaStream_t st, bool programmatic = false);

namespace {

struct StripArgs {
    const uint8_t* in;
    int64_t in_pitch;
    int W, H, bits;
    int rows_per_group;
    int vin;  // rows 16-byte aligned: data and pitch
    BandCoef coef[LUTC_MAX_BANDS];
};

constexpr int kRowBatch = 4;  // rows loaded before any is processed: 64 bytes in flight per thread

__device__ __forceinline__ void unpack8(const uint4 v, uint32_t M, uint32_t (&x)[8])
{
    x[0] = min(v.x & 0xffffu, M); x[1] = min(v.x >> 16, M);
    x[2] = min(v.y & 0xffffu, M); x[3] = min(v.y >> 16, M);
    x[4] = min(v.z & 0xffffu, M); x[5] = min(v.z >> 16, M);
    x[6] = min(v.w & 0xffffu, M); x[7] = min(v.w >> 16, M);
}

// Coefficients of the thread's 8 columns; returns whether all of them are int32-exact
// (O is then pre-offset by 2^15).  Columns past the image edge get zeros.
__device__ __forceinline__ bool load_coef(const BandCoef& c, int c0, int n, int32_t M, int32_t (&A)[8],
                                          int32_t (&G)[8], int32_t (&O)[8])
{
    bool fits = true;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < n) {
            A[j] = __ldg(c.A + c0 + j);
            G[j] = __ldg(c.G + c0 + j);
            O[j] = __ldg(c.O + c0 + j);
            fits = fits && col_fits_i32(A[j], G[j], O[j], M);
        } else {
            A[j] = 0; G[j] = 0; O[j] = 0;
        }
    }
    if (fits) {
#pragma unroll
        for (int j = 0; j < 8; ++j) O[j] += 32768;
    }
    return fits;
}

// The generic path: any alignment, a partial chunk at the right edge, or a
// column that is not int32-exact.  Scalar loads, int64 evaluation, nothing
// unrolled, coefficients re-read through L1, so that it adds few registers to
// the kernel.  It is exact for every column.
__device__ __forceinline__ uint32_t det_generic(const BandCoef& c, int col, uint32_t raw, int32_t M)
{
    return det_i64(__ldg(c.A + col), __ldg(c.G + col), __ldg(c.O + col), min(raw, (uint32_t)M), M);
}

// ---------------------------------------------------------------------------
// pass 1: histogram of corrected DN
// ---------------------------------------------------------------------------
template <int T, bool kGlobal>
__global__ void __launch_bounds__(T) k_strip_hist(const __grid_constant__ StripArgs a,
                                                   unsigned long long* __restrict__ hist)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* sh = reinterpret_cast<uint32_t*>(smem_raw);
    const int L = 1 << a.bits;
    const int32_t M = L - 1;
    if (!kGlobal)
        for (int i = threadIdx.x; i < L; i += T) sh[i] = 0;
    const int b = blockIdx.z;
    const int c0 = (blockIdx.x * T + threadIdx.x) * 8;
    const int n = min(8, a.W - c0);
    int32_t A[8], G[8], O[8];
    const bool fits = load_coef(a.coef[b], c0, n, M, A, G, O);
    __syncthreads();
    unsigned long long* hb = hist + (int64_t)b * L;
    auto bump = [&](uint32_t d) {
        if (kGlobal) atomicAdd(hb + d, 1ull);
        else atomicAdd(sh + d, 1u);
    };
    const int y0 = blockIdx.y * a.rows_per_group;
    const int y1 = min(a.H, y0 + a.rows_per_group);
    const uint8_t* base = a.in + (int64_t)b * a.H * a.in_pitch + (int64_t)c0 * 2;
    if (n == 8 && a.vin && fits) {
        int y = y0;
        for (; y + kRowBatch <= y1; y += kRowBatch) {
            uint4 v[kRowBatch];
#pragma unroll
            for (int u = 0; u < kRowBatch; ++u)
                v[u] = __ldg(reinterpret_cast<const uint4*>(base + (int64_t)(y + u) * a.in_pitch));
#pragma unroll
            for (int u = 0; u < kRowBatch; ++u) {
                uint32_t x[8];
                unpack8(v[u], (uint32_t)M, x);
#pragma unroll
                for (int j = 0; j < 8; ++j) bump(det_i32(A[j], G[j], O[j], x[j], M));
            }
        }
        for (; y < y1; ++y) {
            uint32_t x[8];
            unpack8(__ldg(reinterpret_cast<const uint4*>(base + (int64_t)y * a.in_pitch)), (uint32_t)M, x);
#pragma unroll
            for (int j = 0; j < 8; ++j) bump(det_i32(A[j], G[j], O[j], x[j], M));
        }
    } else if (n > 0) {
        for (int y = y0; y < y1; ++y) {
            const uint16_t* row = reinterpret_cast<const uint16_t*>(base + (int64_t)y * a.in_pitch);
#pragma unroll 1
            for (int j = 0; j < n; ++j) bump(det_generic(a.coef[b], c0 + j, __ldg(row + j), M));
        }
    }
    if (!kGlobal) {
        __syncthreads();
        for (int i = threadIdx.x; i < L; i += T) {
            const uint32_t c = sh[i];
            if (c) atomicAdd(hb + i, (unsigned long long)c);
        }
    }
}

// ---------------------------------------------------------------------------
// pass 2: out8 = S[D] (kStretch) or out16 = D
// ---------------------------------------------------------------------------
template <int T, bool kStretch>
__global__ void __launch_bounds__(T) k_strip_apply(const __grid_constant__ StripArgs a, const uint8_t* __restrict__ S,
                                                   uint8_t* __restrict__ out, int64_t out_pitch, int vout)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint8_t* sS = smem_raw;
    const int L = 1 << a.bits;
    const int32_t M = L - 1;
    const int b = blockIdx.z;
    if (kStretch) {
        const uint4* src = reinterpret_cast<const uint4*>(S + (int64_t)b * L);
        for (int i = threadIdx.x; i < L / 16; i += T) reinterpret_cast<uint4*>(sS)[i] = src[i];
    }
    const int c0 = (blockIdx.x * T + threadIdx.x) * 8;
    const int n = min(8, a.W - c0);
    int32_t A[8], G[8], O[8];
    const bool fits = load_coef(a.coef[b], c0, n, M, A, G, O);
    __syncthreads();
    const int y0 = blockIdx.y * a.rows_per_group;
    const int y1 = min(a.H, y0 + a.rows_per_group);
    if (n <= 0) return;
    const uint8_t* base = a.in + (int64_t)b * a.H * a.in_pitch + (int64_t)c0 * 2;
    uint8_t* obase = out + (int64_t)b * a.H * out_pitch + (int64_t)c0 * (kStretch ? 1 : 2);
    auto emit8 = [&](int y, const uint4 v) {
        uint32_t x[8], o[8];
        unpack8(v, (uint32_t)M, x);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t d = det_i32(A[j], G[j], O[j], x[j], M);
            o[j] = kStretch ? (uint32_t)sS[d] : d;
        }
        uint8_t* dst = obase + (int64_t)y * out_pitch;
        if (kStretch) {
            uint2 r;
            r.x = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
            r.y = o[4] | (o[5] << 8) | (o[6] << 16) | (o[7] << 24);
            *reinterpret_cast<uint2*>(dst) = r;
        } else {
            uint4 r;
            r.x = o[0] | (o[1] << 16); r.y = o[2] | (o[3] << 16);
            r.z = o[4] | (o[5] << 16); r.w = o[6] | (o[7] << 16);
            *reinterpret_cast<uint4*>(dst) = r;
        }
    };
    if (n == 8 && a.vin && vout && fits) {
        int y = y0;
        for (; y + kRowBatch <= y1; y += kRowBatch) {
            uint4 v[kRowBatch];
#pragma unroll
            for (int u = 0; u < kRowBatch; ++u)
                v[u] = __ldg(reinterpret_cast<const uint4*>(base + (int64_t)(y + u) * a.in_pitch));
#pragma unroll
            for (int u = 0; u < kRowBatch; ++u) emit8(y + u, v[u]);
        }
        for (; y < y1; ++y) emit8(y, __ldg(reinterpret_cast<const uint4*>(base + (int64_t)y * a.in_pitch)));
    } else {
        for (int y = y0; y < y1; ++y) {
            const uint16_t* row = reinterpret_cast<const uint16_t*>(base + (int64_t)y * a.in_pitch);
            uint8_t* dst = obase + (int64_t)y * out_pitch;
#pragma unroll 1
            for (int j = 0; j < n; ++j) {
                const uint32_t d = det_generic(a.coef[b], c0 + j, __ldg(row + j), M);
                if (kStretch) dst[j] = sS[d];
                else reinterpret_cast<uint16_t*>(dst)[j] = (uint16_t)d;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Plan {
    dim3 grid;
    int T;
};

int pick_threads(int W, int bits)
{
    const int t = tuning_for(bits).column_threads;
    if (t) return t;
    return W > 1024 ? 256 : (W > 512 ? 128 : 64);
}

template <typename K>
Plan plan_strips(K kernel, int T, size_t smem, const lutc_raster* in, StripArgs& a)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, T, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int cap = tuning_for(in->bits).blocks_per_sm;
    if (cap > 0 && cap < per_sm) per_sm = cap;
    const int strips = (in->width + 8 * T - 1) / (8 * T);
    const int64_t target = (int64_t)sm_count() * per_sm;
    const int64_t per_band_strip = (int64_t)strips * in->bands;
    // whole row groups that fit one wave (at least one per strip and band)
    int64_t groups = target / per_band_strip;
    if (groups < 1) groups = 1;
    if (groups > in->height) groups = in->height;
    if (groups > 65535) groups = 65535;
    const int rows = (int)((in->height + groups - 1) / groups);
    a.rows_per_group = rows;
    Plan p;
    p.T = T;
    p.grid = dim3((unsigned)strips, (unsigned)((in->height + rows - 1) / rows), (unsigned)in->bands);
    return p;
}

StripArgs make_args(const lutc_raster* in, const lutc_coeffs* per_band)
{
    StripArgs a;
    a.in = reinterpret_cast<const uint8_t*>(in->data);
    a.in_pitch = in->pitch_bytes;
    a.W = in->width;
    a.H = in->height;
    a.bits = in->bits;
    a.rows_per_group = 1;
    a.vin = ((uintptr_t)in->data % 16 == 0) && (in->pitch_bytes % 16 == 0);
    for (int b = 0; b < LUTC_MAX_BANDS; ++b) {
        if (b < in->bands) a.coef[b] = BandCoef{per_band[b].A, per_band[b].G, per_band[b].O};
        else a.coef[b] = BandCoef{nullptr, nullptr, nullptr};
    }
    return a;
}

template <int T>
int launch_hist_T(StripArgs& a, const lutc_raster* in, unsigned long long* hist, cudaStream_t st)
{
    const int L = 1 << in->bits;
    if (in->bits <= 15) {
        const size_t smem = (size_t)L * 4;
        auto k = k_strip_hist<T, false>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return LUTC_ECUDA;
        const Plan p = plan_strips(k, T, smem, in, a);
        k<<<p.grid, T, smem, st>>>(a, hist);
    } else {
        auto k = k_strip_hist<T, true>;
        const Plan p = plan_strips(k, T, 0, in, a);
        k<<<p.grid, T, 0, st>>>(a, hist);
    }
    return cuda_status(cudaGetLastError());
}

int launch_hist(StripArgs& a, const lutc_raster* in, unsigned long long* hist, cudaStream_t st)
{
    switch (pick_threads(in->width, in->bits)) {
    case 64: return launch_hist_T<64>(a, in, hist, st);
    case 128: return launch_hist_T<128>(a, in, hist, st);
    default: return launch_hist_T<256>(a, in, hist, st);
    }
}

template <int T, bool kStretch>
int launch_apply_T(StripArgs& a, const lutc_raster* in, const uint8_t* S, void* out, int64_t out_pitch,
                   cudaStream_t st)
{
    const size_t smem = kStretch ? ((size_t)1 << in->bits) : 0;
    auto k = k_strip_apply<T, kStretch>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LUTC_ECUDA;
    const Plan p = plan_strips(k, T, smem, in, a);
    const size_t vec = kStretch ? 8 : 16;
    const int vout = ((uintptr_t)out % vec == 0) && (out_pitch % (int64_t)vec == 0);
    k<<<p.grid, T, smem, st>>>(a, S, reinterpret_cast<uint8_t*>(out), out_pitch, vout);
    return cuda_status(cudaGetLastError());
}

template <bool kStretch>
int launch_apply(StripArgs& a, const lutc_raster* in, const uint8_t* S, void* out, int64_t out_pitch, cudaStream_t st)
{
    switch (pick_threads(in->width, in->bits)) {
    case 64: return launch_apply_T<64, kStretch>(a, in, S, out, out_pitch, st);
    case 128: return launch_apply_T<128, kStretch>(a, in, S, out, out_pitch, st);
    default: return launch_apply_T<256, kStretch>(a, in, S, out, out_pitch, st);
    }
}

struct Layout {
    size_t hist, S, lohi, total;
};

Layout layout_of(const lutc_raster* in)
{
    const size_t L = (size_t)1 << in->bits;
    Layout l;
    l.hist = 0;
    l.S = align_up(l.hist + (size_t)in->bands * L * 8, 256);
    l.lohi = align_up(l.S + (size_t)in->bands * L, 256);
    l.total = align_up(l.lohi + (size_t)in->bands * 8, 256);
    return l;
}

// ---------------------------------------------------------------------------
// tracing: per-phase events of lutc_correct_image
// ---------------------------------------------------------------------------
struct Trace {
    cudaEvent_t* ev = nullptr;  // [capacity][LUTC_TRACE_PHASES + 1]
    int capacity = 0;
    int used = 0;
};
Trace g_trace;

void trace_release()
{
    for (int i = 0; i < g_trace.capacity * (LUTC_TRACE_PHASES + 1); ++i) cudaEventDestroy(g_trace.ev[i]);
    delete[] g_trace.ev;
    g_trace = Trace();
}

// Kernel family of the calling host thread's last call that enqueued pass kernels (lutc_last_path).
thread_local int t_last_path = LUTC_PATH_AUTO;

}  // namespace

void record_path(bool tma) { t_last_path = tma ? LUTC_PATH_TMA : LUTC_PATH_STRIP; }

// events of the next traced call, or nullptr when tracing is off or full
cudaEvent_t* trace_slot()
{
    if (g_trace.used >= g_trace.capacity) return nullptr;
    return g_trace.ev + (size_t)(g_trace.used++) * (LUTC_TRACE_PHASES + 1);
}
// Pass 1 into an existing histogram (no clear) and pass 2, for the library's own pipelines.
int pass1_accumulate(const lutc_raster* in, const lutc_coeffs* per_band, unsigned long long* hist, cudaStream_t st)
{
    if ((int64_t)in->width * in->height == 0) return LUTC_OK;
    const bool tma = tma_eligible(in);
    record_path(tma);
    if (tma) return tma_hist(in, per_band, hist, st);
    StripArgs a = make_args(in, per_band);
    return launch_hist(a, in, hist, st);
}

int pass2(const lutc_raster* in, const lutc_coeffs* per_band, const uint8_t* S, void* out, int64_t out_pitch,
          bool stretch, cudaStream_t st)
{
    if ((int64_t)in->width * in->height == 0) return LUTC_OK;
    const bool tma = tma_eligible(in);
    record_path(tma);
    if (tma) return tma_apply(in, per_band, S, out, out_pitch, stretch, st);
    StripArgs a = make_args(in, per_band);
    return stretch ? launch_apply<true>(a, in, S, out, out_pitch, st)
                   : launch_apply<false>(a, in, nullptr, out, out_pitch, st);
}

size_t tables_bytes(const lutc_raster* in) { return layout_of(in).total; }

void tables_offsets(const lutc_raster* in, size_t* hist, size_t* S, size_t* lohi)
{
    const Layout l = layout_of(in);
    *hist = l.hist;
    *S = l.S;
    *lohi = l.lohi;
}

}  // namespace lutc

using namespace lutc;

extern "C" int lutc_trace_enable(int capacity)
{
    if (capacity < 0 || capacity > (1 << 20)) return LUTC_EINVAL;
    trace_release();
    if (capacity == 0) return LUTC_OK;
    const int n = capacity * (LUTC_TRACE_PHASES + 1);
    g_trace.ev = new (std::nothrow) cudaEvent_t[n];
    if (!g_trace.ev) return LUTC_ENOMEM;
    for (int i = 0; i < n; ++i) {
        if (cudaEventCreate(&g_trace.ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(g_trace.ev[j]);
            delete[] g_trace.ev;
            g_trace = Trace();
            return LUTC_ECUDA;
        }
    }
    g_trace.capacity = capacity;
    return LUTC_OK;
}

extern "C" int lutc_trace_read(float* ms, int max_calls)
{
    if (!ms || max_calls < 0) return LUTC_EINVAL;
    const int n = g_trace.used < max_calls ? g_trace.used : max_calls;
    for (int c = 0; c < n; ++c) {
        cudaEvent_t* e = g_trace.ev + (size_t)c * (LUTC_TRACE_PHASES + 1);
        if (cudaEventSynchronize(e[LUTC_TRACE_PHASES]) != cudaSuccess) return LUTC_ECUDA;
        for (int p = 0; p < LUTC_TRACE_PHASES; ++p)
            if (cudaEventElapsedTime(&ms[c * LUTC_TRACE_PHASES + p], e[p], e[p + 1]) != cudaSuccess) return LUTC_ECUDA;
    }
    g_trace.used = 0;
    return n;
}

extern "C" int lutc_apply_stretch(const lutc_raster* in, const lutc_coeffs* per_band, const uint8_t* S, uint8_t* out,
                                  int64_t out_pitch_bytes, lutc_stream stream)
{
    int rc = check_raster(in);
    if (rc) return rc;
    if ((rc = check_coeff_set(in, per_band))) return rc;
    if ((int64_t)in->width * in->height == 0) return LUTC_OK;
    if (!S || ((uintptr_t)S % 16) || !out || out_pitch_bytes < in->width) return LUTC_EINVAL;
    const bool tma = tma_eligible(in);
    record_path(tma);
    if (tma) return tma_apply(in, per_band, S, out, out_pitch_bytes, true, (cudaStream_t)stream);
    StripArgs a = make_args(in, per_band);
    return launch_apply<true>(a, in, S, out, out_pitch_bytes, (cudaStream_t)stream);
}

extern "C" int lutc_last_path(int* path)
{
    if (!path) return LUTC_EINVAL;
    *path = t_last_path;
    return LUTC_OK;
}

extern "C" size_t lutc_correct_image_workspace(const lutc_raster* in)
{
    if (check_raster(in)) return 0;
    return layout_of(in).total;
}

extern "C" int lutc_correct_image_tables(const lutc_raster* in, size_t* hist_offset, size_t* S_offset,
                                         size_t* lohi_offset)
{
    if (check_raster(in)) return LUTC_EINVAL;
    const Layout l = layout_of(in);
    if (hist_offset) *hist_offset = l.hist;
    if (S_offset) *S_offset = l.S;
    if (lohi_offset) *lohi_offset = l.lohi;
    return LUTC_OK;
}

extern "C" int lutc_hist(const lutc_raster* in, const lutc_coeffs* per_band, uint64_t* hist, lutc_stream stream)
{
    int rc = check_raster(in);
    if (rc) return rc;
    if ((rc = check_coeff_set(in, per_band))) return rc;
    if (!hist) return LUTC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t L = (size_t)1 << in->bits;
    if ((rc = cuda_status(cudaMemsetAsync(hist, 0, (size_t)in->bands * L * 8, st)))) return rc;
    if ((int64_t)in->width * in->height == 0) return LUTC_OK;
    const bool tma = tma_eligible(in);
    record_path(tma);
    if (tma) return tma_hist(in, per_band, reinterpret_cast<unsigned long long*>(hist), st);
    StripArgs a = make_args(in, per_band);
    return launch_hist(a, in, reinterpret_cast<unsigned long long*>(hist), st);
}

extern "C" int lutc_correct_image(const lutc_raster* in, const lutc_coeffs* per_band, int flags, void* out,
                                  int64_t out_pitch_bytes, void* workspace, size_t workspace_bytes, lutc_stream stream)
{
    int rc = check_raster(in);
    if (rc) return rc;
    if ((rc = check_coeff_set(in, per_band))) return rc;
    if (flags & ~LUTC_STRETCH) return LUTC_EINVAL;
    const bool stretch = (flags & LUTC_STRETCH) != 0;
    const int64_t elem = stretch ? 1 : 2;
    const bool empty = (int64_t)in->width * in->height == 0;
    if (!empty && (!out || out_pitch_bytes < elem * in->width || out_pitch_bytes % elem)) return LUTC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool tma = !empty && tma_eligible(in);
    if (!empty) record_path(tma);
    StripArgs a = make_args(in, per_band);
    if (!stretch) {
        if (empty) return LUTC_OK;
        if (tma) return tma_apply(in, per_band, nullptr, out, out_pitch_bytes, false, st);
        return launch_apply<false>(a, in, nullptr, out, out_pitch_bytes, st);
    }

    const Layout l = layout_of(in);
    if (!workspace || workspace_bytes < l.total) return LUTC_ENOMEM;
    if ((uintptr_t)workspace % 256) return LUTC_EINVAL;
    uint8_t* ws = reinterpret_cast<uint8_t*>(workspace);
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(ws + l.hist);
    uint8_t* S = ws + l.S;
    int32_t* lohi = reinterpret_cast<int32_t*>(ws + l.lohi);
    const size_t L = (size_t)1 << in->bits;
    cudaEvent_t* tr = trace_slot();
    if (tr) cudaEventRecord(tr[0], st);
    if ((rc = cuda_status(cudaMemsetAsync(hist, 0, (size_t)in->bands * L * 8, st)))) return rc;
    if (!empty && (rc = tma ? tma_hist(in, per_band, hist, st) : launch_hist(a, in, hist, st))) return rc;
    // TMA path, untraced: the scan launches behind pass 1 and pass 2 behind the scan (programmatic
    // launch), each waiting on the device for the data it reads -- pass 2's blocks start streaming
    // raw tiles while the scan runs
    const bool chain = tma && !tr;
    if (tr) cudaEventRecord(tr[1], st);
    if ((rc = launch_stretch(hist, in->bands, in->bits, S, lohi, st, chain))) return rc;
    if (tr) cudaEventRecord(tr[2], st);
    if (!empty && (rc = tma ? tma_apply(in, per_band, S, out, out_pitch_bytes, true, st, chain)
                            : launch_apply<true>(a, in, S, out, out_pitch_bytes, st)))
        return rc;
    if (tr) cudaEventRecord(tr[3], st);
    return LUTC_OK;
}
