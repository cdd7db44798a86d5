// Bilinear Bayer demosaicing (paper, Section III.A, case study 1), optionally
// fused with the detector correction (step L applied to every photosite first).
//
// Definition: a pixel keeps its own colour; each missing colour is the
// average of the neighbours of that colour among its 8 direct neighbours
// inside the image, rounded half up in integers, (sum + count/2) / count.
// For the four sites of a Bayer cell that is: at a red or blue site, green
// from the 4 orthogonal and the opposite colour from the 4 diagonal
// neighbours; at a green site, one colour from the left/right pair and the
// other from the up/down pair.
//
// GB300 mapping: frames with 16-byte aligned rows take the TMA-fed persistent
// kernel below (raw frames of at most 4 M pixels excepted); the others a block
// per tile (16 rows raw, 32 rows with correction; see Tile).  The tile and a halo (one row above and below, one
// 8-column chunk left and right, so every load is an aligned vector) is staged
// in shared memory, corrected on the way in when coefficients are given (the
// int32/int64 Horner evaluation of step L).
// Each thread then produces a 2 x 8 patch: reads 4 shared rows of 12 values
// (one 16-byte and two 4-byte loads per row), resolves the Bayer role of each
// pixel at compile time (pattern phase is a template parameter, patch origins
// are even), and writes 16-byte vectors to the three planar outputs.  Blocks
// whose halo lies inside the image take a path with constant neighbour
// counts; border blocks count the neighbours that exist.  HBM traffic per
// pixel: 2 bytes in, 6 bytes out (the halo re-reads hit L2).
#include <stdint.h>

#include <algorithm>

#include "lutc_internal.cuh"
#include "lutc_ptx.cuh"

namespace lutc {
namespace {

// Tile shapes (measured on GB300, 16384 x 16384 frames): the raw path runs
// 128 x 16 tiles in blocks of 128 threads, 8 blocks per SM; the corrected path
// runs 128 x 32 tiles in blocks of 256 threads, 4 per SM, whose loaders hold
// their columns' coefficients in registers.
template <bool kCorrect>
struct Tile {
    static constexpr int W = 128, H = kCorrect ? 32 : 16;
    static constexpr int threads = (W / 8) * (H / 2);   // one 2 x 8 patch per thread
    static constexpr int min_blocks = kCorrect ? 4 : 8;
    static constexpr int SW = W + 16, SH = H + 2;       // staged tile with halo (uint16)
    static constexpr int chunk = kCorrect ? 4 : 8;      // columns per loader load (8 or 16 bytes)
    static constexpr int chunks = SW / chunk;           // loads per staged row
    static constexpr int lanes = threads / chunks;      // row lanes of the loader
};

struct DemosaicArgs {
    const uint8_t* in;
    int64_t in_pitch;
    int W, H, bits;
    BandCoef coef;     // A == nullptr: no correction
    uint8_t* out;
    int64_t out_pitch;
    bool vin, vout;    // 16-byte aligned rows in / out
};

// (sum + cnt/2) / cnt for cnt in 0..4 and sum < 2^18, exactly: multiply by ceil(2^20 / cnt)
__device__ __forceinline__ uint32_t avg_n(uint32_t sum, uint32_t cnt)
{
    const uint32_t mul = cnt == 0 ? 0u : cnt == 1 ? (1u << 20) : cnt == 2 ? (1u << 19) : cnt == 3 ? 349526u : (1u << 18);
    return (uint32_t)(((uint64_t)(sum + (cnt >> 1)) * mul) >> 20);
}

// Stages rows y0-1 .. y0+H and columns x0-8 .. x0+W+7 of the raw frame (zero
// outside it), corrected when kCorrect: a loader thread owns `chunk` adjacent
// staged columns, keeps their coefficients in registers and walks the rows.
template <bool kCorrect>
__device__ __forceinline__ void stage_tile(const DemosaicArgs& a, int x0, int y0,
                                           uint16_t (*s)[Tile<kCorrect>::SW])
{
    using T = Tile<kCorrect>;
    constexpr int CW = T::chunk;
    const int t = threadIdx.x;
    if (t >= T::chunks * T::lanes) return;
    const int ch = t % T::chunks, lane = t / T::chunks;
    const int gx0 = x0 - 8 + ch * CW;
    const int32_t M = (1 << a.bits) - 1;
    int32_t cA[CW], cG[CW], cO[CW];
    bool fits[CW];
    if (kCorrect) {
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const int gx = gx0 + j;
            const bool in = gx >= 0 && gx < a.W;
            cA[j] = in ? __ldg(a.coef.A + gx) : 0;
            cG[j] = in ? __ldg(a.coef.G + gx) : 0;
            cO[j] = in ? __ldg(a.coef.O + gx) : 0;
            fits[j] = col_fits_i32(cA[j], cG[j], cO[j], M);
            if (fits[j]) cO[j] += 32768;
        }
    }
    const bool full = a.vin && gx0 >= 0 && gx0 + CW <= a.W;
    for (int r = lane; r < T::SH; r += T::lanes) {
        const int gy = y0 - 1 + r;
        uint32_t v[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) v[j] = 0;
        if (gy >= 0 && gy < a.H) {
            const uint8_t* row = a.in + (int64_t)gy * a.in_pitch + (int64_t)gx0 * 2;
            if (full) {
                if constexpr (CW == 8) {
                    const uint4 q = __ldg(reinterpret_cast<const uint4*>(row));
                    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int j = 0; j < CW; ++j) v[j] = (w[j / 2] >> (16 * (j & 1))) & 0xffffu;
                } else {
                    const uint2 q = __ldg(reinterpret_cast<const uint2*>(row));
                    const uint32_t w[2] = {q.x, q.y};
#pragma unroll
                    for (int j = 0; j < CW; ++j) v[j] = (w[j / 2] >> (16 * (j & 1))) & 0xffffu;
                }
            } else {
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const int gx = gx0 + j;
                    if (gx >= 0 && gx < a.W) v[j] = __ldg(reinterpret_cast<const uint16_t*>(row) + j);
                }
            }
            if (kCorrect) {
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const int gx = gx0 + j;
                    if (gx >= 0 && gx < a.W) {
                        const uint32_t x = min(v[j], (uint32_t)M);
                        v[j] = fits[j] ? det_i32(cA[j], cG[j], cO[j], x, M) : det_i64(cA[j], cG[j], cO[j], x, M);
                    }
                }
            }
        }
        uint32_t w[CW / 2];
#pragma unroll
        for (int j = 0; j < CW / 2; ++j) w[j] = v[2 * j] | (v[2 * j + 1] << 16);
        if constexpr (CW == 8)
            *reinterpret_cast<uint4*>(&s[r][ch * CW]) = make_uint4(w[0], w[1], w[2], w[3]);
        else
            *reinterpret_cast<uint2*>(&s[r][ch * CW]) = make_uint2(w[0], w[1]);
    }
}

// Bayer role of a pixel under RGGB at parity (py, px): 0 R site, 1 G in a red row, 2 G in a blue row, 3 B site
__host__ __device__ constexpr int role(int py, int px) { return py == 0 ? (px == 0 ? 0 : 1) : (px == 0 ? 2 : 3); }

// One thread's 2 x 8 patch of the tile at (x0, y0): reads 4 staged rows of 12 values (staged
// column c holds frame column x0 - 8 + c, staged row r frame row y0 - 1 + r) and writes the patch's
// rows to the three planes.
template <int PY, int PX, int kTW, int kTH, int kSW>
__device__ __forceinline__ void patch(const uint16_t (*s)[kSW], int x0, int y0, int W, int H, uint8_t* out,
                                      int64_t out_pitch, bool vout)
{
    const int cx = threadIdx.x % (kTW / 8), ry = threadIdx.x / (kTW / 8);
    const int c0 = 8 + cx * 8;   // staged column of the patch's first pixel
    const int r0 = 1 + ry * 2;   // staged row of the patch's first row
    const int gx = x0 + cx * 8, gy = y0 + ry * 2;
    if (gx >= W || gy >= H) return;

    // 4 staged rows x 12 values (columns c0-2 .. c0+9)
    uint32_t v[4][12];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint16_t* row = s[r0 - 1 + i];
        const uint32_t lo = *reinterpret_cast<const uint32_t*>(row + c0 - 2);
        const uint4 mid = *reinterpret_cast<const uint4*>(row + c0);
        const uint32_t hi = *reinterpret_cast<const uint32_t*>(row + c0 + 8);
        v[i][0] = lo & 0xffffu; v[i][1] = lo >> 16;
        v[i][2] = mid.x & 0xffffu; v[i][3] = mid.x >> 16; v[i][4] = mid.y & 0xffffu; v[i][5] = mid.y >> 16;
        v[i][6] = mid.z & 0xffffu; v[i][7] = mid.z >> 16; v[i][8] = mid.w & 0xffffu; v[i][9] = mid.w >> 16;
        v[i][10] = hi & 0xffffu; v[i][11] = hi >> 16;
    }

    // the block's halo is inside the image: every neighbour exists
    const bool interior = x0 > 0 && y0 > 0 && x0 + kTW < W && y0 + kTH < H;
    const bool full = vout && gx + 8 <= W;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int y = gy + i;
        if (y >= H) break;
        const uint32_t nu = interior || y > 0, nd = interior || y + 1 < H;
        uint32_t o[3][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int x = gx + j;
            const uint32_t nl = interior || x > 0, nr = interior || x + 1 < W;
            const uint32_t c = v[i + 1][j + 2];
            const uint32_t hs = v[i + 1][j + 1] + v[i + 1][j + 3];
            const uint32_t vs = v[i][j + 2] + v[i + 2][j + 2];
            const uint32_t ds = v[i][j + 1] + v[i][j + 3] + v[i + 2][j + 1] + v[i + 2][j + 3];
            uint32_t orth, diag, horiz, vert;
            if (interior) {
                orth = (hs + vs + 2) >> 2;
                diag = (ds + 2) >> 2;
                horiz = (hs + 1) >> 1;
                vert = (vs + 1) >> 1;
            } else {
                const uint32_t nh = nl + nr, nv = nu + nd;
                orth = avg_n(hs + vs, nh + nv);
                diag = avg_n(ds, nh * nv);
                horiz = avg_n(hs, nh);
                vert = avg_n(vs, nv);
            }
            switch (role((i + PY) & 1, (j + PX) & 1)) {
            case 0: o[0][j] = c; o[1][j] = orth; o[2][j] = diag; break;
            case 1: o[0][j] = horiz; o[1][j] = c; o[2][j] = vert; break;
            case 2: o[0][j] = vert; o[1][j] = c; o[2][j] = horiz; break;
            default: o[0][j] = diag; o[1][j] = orth; o[2][j] = c; break;
            }
        }
        // this row of the patch in the three planes
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint16_t* row = reinterpret_cast<uint16_t*>(out + ((int64_t)k * H + y) * out_pitch);
            if (full) {
                uint4 q;
                q.x = o[k][0] | (o[k][1] << 16);
                q.y = o[k][2] | (o[k][3] << 16);
                q.z = o[k][4] | (o[k][5] << 16);
                q.w = o[k][6] | (o[k][7] << 16);
                *reinterpret_cast<uint4*>(row + gx) = q;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (gx + j < W) row[gx + j] = (uint16_t)o[k][j];
            }
        }
    }
}

template <int PY, int PX, bool kCorrect>
__global__ void __launch_bounds__(Tile<kCorrect>::threads, Tile<kCorrect>::min_blocks) k_demosaic(DemosaicArgs a)
{
    using T = Tile<kCorrect>;
    __shared__ __align__(16) uint16_t s[T::SH][T::SW];
    const int x0 = blockIdx.x * T::W, y0 = blockIdx.y * T::H;
    stage_tile<kCorrect>(a, x0, y0, s);
    __syncthreads();
    patch<PY, PX, T::W, T::H, T::SW>(s, x0, y0, a.W, a.H, a.out, a.out_pitch, a.vout);
}

// ---------------------------------------------------------------------------
// TMA-fed persistent version (frames with 16-byte aligned rows, at least one
// staged tile in each direction).  A block keeps two 128 x 64 tiles (with
// their halo) in flight through cp.async.bulk.tensor loads into a 2-stage
// ring (zeros outside the frame) while it computes the current one.  The
// grid is one wave and the blocks sweep the frame together: at step k block
// b takes tile k x gridDim + b in row-major tile order, so at any moment all
// blocks work on the same few rows of tiles and share DRAM pages.  (A walk
// where each block took its own contiguous run of tiles was slower than the
// plain kernel, 580 against 474 us at 16384^2, and so was a grid of whole
// blocks per column strip, which leaves SMs unevenly loaded: 465 us.)
// With correction, the block corrects the staged tile in place before the
// interpolation: a thread owns 4 staged columns (their coefficients staged
// with the tile) and a seventh of the rows.  Only the 136 staged columns the
// interpolation reads are corrected (the 8-column alignment halo holds 7
// unused columns on each side); a tile of 64 rows keeps the corrected halo
// rows at 2 in 66, so step L runs 1.10 times per output pixel.
// ---------------------------------------------------------------------------
constexpr int kQW = 128, kQSW = kQW + 16;
constexpr int kQPatchRows = 32;                             // rows one pass of the block's 2 x 8 patches covers
constexpr int kQThreads = (kQW / 8) * (kQPatchRows / 2);
// Two stages: one tile read while the next one loads.  (A third stage, or 64-row tiles whose next
// load is issued as soon as their stage is free, made raw 16384^2 sweeps slower, 401 and 409
// against 357 us: loads issued further ahead of their use slow the memory system down.)
constexpr int kQStages = 2;
// Tile height: 64 rows halve the corrected halo rows (2 in 66); 32 rows for raw frames, whose next
// load then goes out a 32-row tile ahead of its use rather than a 64-row one, and for small frames
// (more tiles).
#ifndef LUTC_DEMOSAIC_CORRECTED_ROWS
#define LUTC_DEMOSAIC_CORRECTED_ROWS 64
#endif
template <int kTH>
struct QTile {
    static constexpr int H = kTH, SH = kTH + 2;
    static constexpr int StageElems = (kQSW * SH + 63) / 64 * 64;  // stages 128-byte aligned
    static constexpr uint32_t BoxBytes = kQSW * SH * 2;
    static_assert(H % kQPatchRows == 0 && SH <= 256 && (StageElems * 2) % 128 == 0, "tile geometry");
};
constexpr int kQQuad0 = 1, kQQuads = kQSW / 4 - 2;          // correction: staged column groups 1 .. 34
constexpr int kQLanes = kQThreads / kQQuads;                // correction: row lanes
// a staged coefficient row: kQSW int32 padded so that every row of every stage starts on the
// 128-byte boundary a tiled tensor copy writes to
constexpr int kQCoefRow = (kQSW * 4 + 127) / 128 * 128 / 4;
static_assert(kQThreads == 256 && kQLanes >= 1, "tile geometry");
static_assert(kQQuad0 * 4 + 3 >= 7 && (kQQuad0 + kQQuads) * 4 <= kQSW && (kQQuad0 + kQQuads) * 4 >= 8 + kQW + 1,
              "the corrected groups cover staged columns 7 .. kQW + 8, all the interpolation reads");
static_assert(kQSW <= 256 && (kQCoefRow * 4) % 128 == 0, "TMA box width, coefficient rows 128-byte aligned");

struct DemosaicTmaArgs {
    CUtensorMap map;      // uint16 [H][W], row stride = pitch, box {kQSW, tile rows + 2}
    CUtensorMap cmap[3];  // int32 [W] coefficient rows A, G, O, box {kQSW} (when coef_tma)
    int W, H, bits;
    BandCoef coef;        // A == nullptr: no correction
    int coef_tma;         // 1: each tile's load also brings its columns' coefficients into the stage
    uint8_t* out;
    int64_t out_pitch;
    int vout;
    int strips;        // column strips of kQW columns (tiles per tile row)
    int64_t ntiles;    // strips x tile rows
    int* status;       // the library's kernel status word
};

// Tile k of a block is tile k x step + first in row-major order over `strips` tiles per row; the
// cursor walks them with one compare per step instead of a 64-bit division.
struct TileCursor {
    int tx, dtx, strips;
    int ty, dty;
    __device__ __forceinline__ void start(int64_t first, int64_t step, int s)
    {
        strips = s;
        ty = (int)(first / s);
        tx = (int)(first - (int64_t)ty * s);
        dty = (int)(step / s);
        dtx = (int)(step - (int64_t)dty * s);
    }
    __device__ __forceinline__ void next()
    {
        tx += dtx;
        ty += dty;
        if (tx >= strips) {
            tx -= strips;
            ++ty;
        }
    }
};

// Step L on the staged columns 4q .. 4q + 3 of one stage, rows lane, lane + kQLanes, ...: the
// coefficients come with the tile (ctma) or from global memory.  The common case (four columns
// inside the frame, all int32-exact) is decided by one bound on the largest |A|, |G| and |O + 2^15|
// of the four, which implies the bound of each column; a group that fails it takes the per-column
// path, exact for any coefficients.
template <int kSH>
__device__ __forceinline__ void correct_stage(const DemosaicTmaArgs& a, uint16_t (*st)[kQSW],
                                              const int32_t (*cb)[kQCoefRow], bool ctma, int x0, int y0, int q,
                                              int lane, int32_t M, uint32_t M2, bool packed)
{
    int32_t cA[4], cG[4], cO[4];
    if (ctma) {
        // staged with the tile (zeros outside the frame)
        const int4 va = *reinterpret_cast<const int4*>(&cb[0][q * 4]);
        const int4 vg = *reinterpret_cast<const int4*>(&cb[1][q * 4]);
        const int4 vo = *reinterpret_cast<const int4*>(&cb[2][q * 4]);
        cA[0] = va.x; cA[1] = va.y; cA[2] = va.z; cA[3] = va.w;
        cG[0] = vg.x; cG[1] = vg.y; cG[2] = vg.z; cG[3] = vg.w;
        cO[0] = vo.x; cO[1] = vo.y; cO[2] = vo.z; cO[3] = vo.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gx = x0 - 8 + q * 4 + j;
            const bool in = gx >= 0 && gx < a.W;
            cA[j] = in ? __ldg(a.coef.A + gx) : 0;
            cG[j] = in ? __ldg(a.coef.G + gx) : 0;
            cO[j] = in ? __ldg(a.coef.O + gx) : 0;
        }
    }
    // rows of the frame only (zeros from the load stay zeros): staged row 0 is frame row y0 - 1,
    // outside the frame on the top tile row
    const int r_lo = (y0 == 0 && lane == 0) ? kQLanes : lane;
    const int r_hi = min(kSH, a.H - y0 + 1);
    const int gx0 = x0 - 8 + q * 4;
    uint32_t ma = 0, mg = 0, mo = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t o = (int64_t)cO[j] + 32768;
        ma = max(ma, cA[j] < 0 ? 0u - (uint32_t)cA[j] : (uint32_t)cA[j]);
        mg = max(mg, cG[j] < 0 ? 0u - (uint32_t)cG[j] : (uint32_t)cG[j]);
        mo = max(mo, (uint32_t)(o < 0 ? -o : o));
    }
    const uint32_t mm = (uint32_t)M * (uint32_t)M;
    const bool all_fit = (uint64_t)ma * mm + (uint64_t)mg * (uint32_t)M + mo < ((uint64_t)1 << 31);
    if (gx0 >= 0 && gx0 + 4 <= a.W && all_fit) {
#pragma unroll
        for (int j = 0; j < 4; ++j) cO[j] += 32768;
        auto pair = [&](uint32_t w, int j) {  // columns j, j + 1 of the thread's four
            w = __vminu2(w, M2);  // both raw DN clamped to M at once
            const uint32_t xa = w & 0xffffu, xb = w >> 16;
            if (packed) {
                // floor(t / 2^16) of an exact int32 t is its high half read as a signed 16-bit value:
                // gather both high halves, clamp both to [0, M] at once
                const uint32_t ta = ((uint32_t)cA[j] * xa + (uint32_t)cG[j]) * xa + (uint32_t)cO[j];
                const uint32_t tb = ((uint32_t)cA[j + 1] * xb + (uint32_t)cG[j + 1]) * xb + (uint32_t)cO[j + 1];
                return __vimin_s16x2_relu(__byte_perm(ta, tb, 0x7632), M2);
            }
            return det_i32(cA[j], cG[j], cO[j], xa, M) | (det_i32(cA[j + 1], cG[j + 1], cO[j + 1], xb, M) << 16);
        };
        auto correct4 = [&](uint2 w) {
            w.x = pair(w.x, 0);
            w.y = pair(w.y, 2);
            return w;
        };
        // four rows per step: sixteen independent evaluations in flight
        int r = r_lo;
        for (; r + 3 * kQLanes < r_hi; r += 4 * kQLanes) {
            uint2* p[4];
            uint2 w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                p[u] = reinterpret_cast<uint2*>(&st[r + u * kQLanes][q * 4]);
                w[u] = *p[u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) *p[u] = correct4(w[u]);
        }
        for (; r < r_hi; r += kQLanes) {
            uint2* p0 = reinterpret_cast<uint2*>(&st[r][q * 4]);
            *p0 = correct4(*p0);
        }
        return;
    }
    bool fits[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        fits[j] = col_fits_i32(cA[j], cG[j], cO[j], M);
        if (fits[j]) cO[j] += 32768;
    }
    for (int r = r_lo; r < r_hi; r += kQLanes) {
        uint2 w = *reinterpret_cast<const uint2*>(&st[r][q * 4]);
        uint32_t v[4] = {w.x & 0xffffu, w.x >> 16, w.y & 0xffffu, w.y >> 16};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gx = gx0 + j;
            if (gx >= 0 && gx < a.W) {
                const uint32_t x = min(v[j], (uint32_t)M);
                v[j] = fits[j] ? det_i32(cA[j], cG[j], cO[j], x, M) : det_i64(cA[j], cG[j], cO[j], x, M);
            }
        }
        w.x = v[0] | (v[1] << 16);
        w.y = v[2] | (v[3] << 16);
        *reinterpret_cast<uint2*>(&st[r][q * 4]) = w;
    }
}

template <int PY, int PX, bool kCorrect, int kTH>
__global__ void __launch_bounds__(kQThreads, 3) k_demosaic_tma(const __grid_constant__ DemosaicTmaArgs a)
{
    constexpr int kS = kQStages;
    using Q = QTile<kTH>;
    constexpr int kQH = Q::H, kQSH = Q::SH;
    __shared__ __align__(128) uint16_t ring[kS][Q::StageElems];
    __shared__ __align__(128) int32_t cbuf[kCorrect ? kS : 1][3][kCorrect ? kQCoefRow : 4];
    __shared__ __align__(8) uint64_t full[kS];
    const int tid = threadIdx.x;
    const int64_t n = (int64_t)blockIdx.x < a.ntiles ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (n == 0) return;  // the whole block, before any barrier exists
    // every tensor copy of this kernel writes to a 128-byte boundary (offsets checked at compile
    // time); a base off that boundary is refused before any copy is issued
    if ((ptx::smem_addr(&ring[0][0]) | ptx::smem_addr(&cbuf[0][0][0])) & 127u) {
        if (tid == 0) atomicCAS(a.status, 0, LUTC_ECUDA);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < kS; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    TileCursor cur, icur;  // the tile being interpolated; the next tile to load (thread 0)
    cur.start(blockIdx.x, gridDim.x, a.strips);
    icur = cur;
    const bool ctma = kCorrect && a.coef_tma;
    int64_t issued = 0;  // thread 0: tiles whose loads it has issued
    auto issue = [&](int64_t k) {  // thread 0: the block's k-th tile (icur) into stage k % kS
        const int s = (int)(k % kS);
        uint64_t* bar = &full[s];
        const int x = icur.tx * kQW - 8;  // a multiple of 8 columns: 16-byte aligned for both maps
        ptx::mbar_arrive_expect_tx(bar, Q::BoxBytes + (ctma ? 3u * kQSW * 4u : 0u));
        ptx::tma_load_2d(ring[s], &a.map, bar, x, icur.ty * kQH - 1);
        if (kCorrect && ctma)
            for (int c = 0; c < 3; ++c) ptx::tma_load_1d(cbuf[s][c], &a.cmap[c], bar, x);
        icur.next();
        ++issued;
    };
    if (tid == 0)
        for (int64_t k = 0; k < n && k < kS; ++k) issue(k);

    const int32_t M = (1 << a.bits) - 1;
    const uint32_t M2 = (uint32_t)M | ((uint32_t)M << 16);
    const bool packed = a.bits <= 15;  // clamps two DN per instruction as signed 16-bit halves
    const int q = kQQuad0 + tid % kQQuads, lane = tid / kQQuads;
    auto stage = [&](int s) { return reinterpret_cast<uint16_t (*)[kQSW]>(ring[s]); };
    // waits (bounded) for the load of the block's tile j and checks (checked builds) that its origin
    // lies in the frame; the same decision in every thread
    auto arrived = [&](int64_t j, const TileCursor& c) {
        const bool ok = ptx::mbar_wait_bounded(&full[j % kS], (uint32_t)((j / kS) & 1), a.status);
        if (!__syncthreads_and(ok)) return false;
        return in_bounds(c.tx >= 0 && c.ty >= 0 && c.tx * kQW < a.W && c.ty * kQH < a.H && c.tx < a.strips, a.status);
    };
    int64_t k = 0;
    for (; k < n; ++k, cur.next()) {
        const int s = (int)(k % kS);
        const int x0 = cur.tx * kQW, y0 = cur.ty * kQH;
        if (!arrived(k, cur)) break;
        if constexpr (kCorrect) {
            if (lane < kQLanes) correct_stage<kQSH>(a, stage(s), cbuf[s], ctma, x0, y0, q, lane, M, M2, packed);
            __syncthreads();
        }
        // one copy of the patch code for every 32-row part of the tile (unrolled, the interpolation's
        // code twice over misses the instruction cache)
#pragma unroll 1
        for (int h = 0; h < kQH; h += kQPatchRows) {
            patch<PY, PX, kQW, kQPatchRows, kQSW>(stage(s) + h, x0, y0 + h, a.W, a.H, a.out, a.out_pitch,
                                                 a.vout != 0);
        }
        __syncthreads();  // every thread is done with stage s
        if (tid == 0 && k + kS < n) {
            ptx::fence_proxy_async_smem();  // this block's generic accesses to the stage come before the reload
            issue(k + kS);
        }
    }
    if (k < n && tid == 0) {
        // a load did not arrive in time: wait (bounded) for the ones still in flight before leaving
        for (int64_t j = k; j < issued; ++j)
            ptx::mbar_wait_bounded(&full[j % kS], (uint32_t)((j / kS) & 1), a.status);
    }
}

// Blocks of the persistent TMA-fed grid: SMs x resident blocks (computed once per device and kernel kind).
template <bool kCorrect, int kTH>
int tma_blocks_per_sm()
{
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cache[dev] == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_demosaic_tma<0, 0, kCorrect, kTH>, kQThreads, 0) !=
                cudaSuccess ||
            b < 1) {
            cudaGetLastError();
            b = 1;
        }
        cache[dev] = b;
    }
    return cache[dev];
}

template <bool kCorrect, int kTH>
int launch_tma(int py, int px, cudaStream_t st, DemosaicTmaArgs& a)
{
    const int per_sm = tma_blocks_per_sm<kCorrect, kTH>();
    if (per_sm < 1) return LUTC_ECUDA;
    // one wave, never more blocks than tiles
    const int64_t blocks = std::min<int64_t>(a.ntiles, (int64_t)sm_count() * per_sm);
    switch (2 * py + px) {
    case 0: k_demosaic_tma<0, 0, kCorrect, kTH><<<(unsigned)blocks, kQThreads, 0, st>>>(a); break;
    case 1: k_demosaic_tma<0, 1, kCorrect, kTH><<<(unsigned)blocks, kQThreads, 0, st>>>(a); break;
    case 2: k_demosaic_tma<1, 0, kCorrect, kTH><<<(unsigned)blocks, kQThreads, 0, st>>>(a); break;
    default: k_demosaic_tma<1, 1, kCorrect, kTH><<<(unsigned)blocks, kQThreads, 0, st>>>(a); break;
    }
    return cuda_status(cudaGetLastError());
}

template <bool kCorrect>
void launch(int py, int px, int W, int H, cudaStream_t st, const DemosaicArgs& a)
{
    using T = Tile<kCorrect>;
    const dim3 grid((unsigned)((W + T::W - 1) / T::W), (unsigned)((H + T::H - 1) / T::H));
    switch (2 * py + px) {
    case 0: k_demosaic<0, 0, kCorrect><<<grid, T::threads, 0, st>>>(a); break;
    case 1: k_demosaic<0, 1, kCorrect><<<grid, T::threads, 0, st>>>(a); break;
    case 2: k_demosaic<1, 0, kCorrect><<<grid, T::threads, 0, st>>>(a); break;
    default: k_demosaic<1, 1, kCorrect><<<grid, T::threads, 0, st>>>(a); break;
    }
}

}  // namespace
}  // namespace lutc

using namespace lutc;

extern "C" int lutc_demosaic(const lutc_raster* in, const lutc_coeffs* coeffs, int pattern, uint16_t* out,
                             int64_t out_pitch_bytes, lutc_stream stream)
{
    if (!in || in->bands != 1) return LUTC_EINVAL;
    int rc = check_raster(in);
    if (rc) return rc;
    if (pattern < LUTC_BAYER_RGGB || pattern > LUTC_BAYER_GBRG) return LUTC_EINVAL;
    if ((int64_t)in->width * in->height == 0) return LUTC_OK;
    if (!out || ((uintptr_t)out % 2) || out_pitch_bytes < 2 * (int64_t)in->width || (out_pitch_bytes % 2))
        return LUTC_EINVAL;
    if (coeffs && (!coeffs->A || !coeffs->G || !coeffs->O || coeffs->ncols != in->width)) return LUTC_EINVAL;
    // pattern -> the row / column shift that turns it into RGGB
    static const int kPY[4] = {0, 1, 0, 1}, kPX[4] = {0, 1, 1, 0};
    DemosaicArgs a;
    a.in = reinterpret_cast<const uint8_t*>(in->data);
    a.in_pitch = in->pitch_bytes;
    a.W = in->width;
    a.H = in->height;
    a.bits = in->bits;
    a.coef = coeffs ? BandCoef{coeffs->A, coeffs->G, coeffs->O} : BandCoef{nullptr, nullptr, nullptr};
    a.out = reinterpret_cast<uint8_t*>(out);
    a.out_pitch = out_pitch_bytes;
    a.vin = ((uintptr_t)in->data % 16) == 0 && (in->pitch_bytes % 16) == 0;
    a.vout = ((uintptr_t)out % 16) == 0 && (out_pitch_bytes % 16) == 0;
    cudaStream_t st = (cudaStream_t)stream;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    int* status = device_status_ptr();
    // tile height: the taller tile for corrected frames with at least two tiles per block of one wave
    constexpr int kTall = LUTC_DEMOSAIC_CORRECTED_ROWS, kShort = 32;
    const int64_t strips = (in->width + kQW - 1) / kQW;
    const bool tall = coeffs && kTall != kShort && in->height >= QTile<kTall>::SH &&
                      strips * ((in->height + kTall - 1) / kTall) >=
                          2 * (int64_t)sm_count() * std::max(1, tma_blocks_per_sm<true, kTall>());
    const int th = tall ? kTall : kShort;
    // a raw frame of at most 4 M pixels (the paper's 2048 x 2048 frame: 8.0 against 9.2 us) takes the
    // block-per-tile kernel: its 16-row tiles spread over more blocks than the persistent grid's
    // 128 x 32 tiles, and the frame stays in L2; corrected frames keep the TMA-fed kernel (12.3 against
    // 12.7 us at that size)
    const bool small = !coeffs && (int64_t)in->width * in->height <= ((int64_t)1 << 22);
    if (!small && enc && status && ((uintptr_t)in->data % 16) == 0 && (in->pitch_bytes % 16) == 0 && in->width >= kQSW &&
        in->height >= th + 2) {
        DemosaicTmaArgs t;
        const cuuint64_t dims[2] = {(cuuint64_t)in->width, (cuuint64_t)in->height};
        const cuuint64_t strides[1] = {(cuuint64_t)in->pitch_bytes};
        const cuuint32_t box[2] = {(cuuint32_t)kQSW, (cuuint32_t)(th + 2)};
        const cuuint32_t estr[2] = {1, 1};
        // a staged row is 288 bytes starting 16 bytes before a 256-byte boundary: promotion to 128-byte
        // lines fetches 512 bytes for it, 256-byte promotion 768 (16384^2 corrected frames 408 -> 399 us,
        // raw 357 -> 354)
        if (enc(&t.map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<uint16_t*>(in->data), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
            t.W = in->width;
            t.H = in->height;
            t.bits = in->bits;
            t.coef = a.coef;
            // coefficient rows as 1-D tensors (their base must be 16-byte aligned); else per-tile loads
            auto coef_map = [&](CUtensorMap* m, const int32_t* p) {
                const cuuint64_t d1[1] = {(cuuint64_t)in->width};
                const cuuint64_t s1[1] = {(cuuint64_t)in->width * 4};  // unused at rank 1
                const cuuint32_t b1[1] = {(cuuint32_t)kQSW};
                const cuuint32_t e1[1] = {1};
                return ((uintptr_t)p % 16) == 0 &&
                       enc(m, CU_TENSOR_MAP_DATA_TYPE_INT32, 1, const_cast<int32_t*>(p), d1, s1, b1, e1,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
            };
            t.coef_tma = coeffs && coef_map(&t.cmap[0], coeffs->A) && coef_map(&t.cmap[1], coeffs->G) &&
                         coef_map(&t.cmap[2], coeffs->O);
            t.out = a.out;
            t.out_pitch = a.out_pitch;
            t.vout = a.vout;
            t.strips = (int)strips;
            t.ntiles = strips * ((in->height + th - 1) / th);
            t.status = status;
            if (!coeffs) return launch_tma<false, kShort>(kPY[pattern], kPX[pattern], st, t);
            return tall ? launch_tma<true, kTall>(kPY[pattern], kPX[pattern], st, t)
                        : launch_tma<true, kShort>(kPY[pattern], kPX[pattern], st, t);
        }
    }
    if ((in->height + 15) / 16 > 65535) return LUTC_EUNSUPPORTED;  // grid rows of the raw path's 16-row tiles
    if (coeffs)
        launch<true>(kPY[pattern], kPX[pattern], in->width, in->height, st, a);
    else
        launch<false>(kPY[pattern], kPX[pattern], in->width, in->height, st, a);
    return cuda_status(cudaGetLastError());
}
