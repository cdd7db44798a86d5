/*
 * CPU oracle for detector LUT generation and LUT-based image correction.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline / reference arm may load it; the
 * product path never calls it and shares no code, header or table with it.
 *
 * The paper (Section I) names LUT generation and image correction as one of
 * the compute-heavy tasks its client-server framework ships to a remote GPU,
 * but prints no formula.  The definitions below are the library's, written
 * out directly in exact integer arithmetic (int64; every intermediate is
 * bounded by 2^63 for bit depths up to 16, see lut_entry):
 *
 *   (L)  D[c][x] = clamp(floor((A[c] x^2 + G[c] x + O[c] + 2^15) / 2^16), 0, M),
 *        M = 2^bits - 1: a per-detector (per-column) response polynomial with
 *        Q16 fixed-point quadratic A, gain G and offset O, rounded half up.
 *        The polynomial-coefficient form follows the paper's least-squares
 *        detector model (Section III-B, the normal equations A X = B).
 *   (P)  corrected pixel d = D[c][min(raw, M)] (raw DN above M reads entry M).
 *   (H)  h[v] = number of pixels of a band whose corrected value is v.
 *   (S)  N = sum_v h[v];  lo = least v with 100 cdf(v) >= 2N, hi = least v
 *        with 100 cdf(v) >= 98N;  S[v] = 0 if hi == lo, else
 *        clamp(trunc(((v - lo) 255 + trunc((hi - lo) / 2)) / (hi - lo)), 0, 255).
 *   (C)  C[c][x] = S[D[c][x]]  (composed per-column 2^bits -> uint8 LUT).
 *   (A)  out8 = C[c][min(raw, M)].
 *
 * Data layout: raster rows are contiguous, row y of a band starts at element
 * y * pitch (pitch in ELEMENTS here); bands are separate calls except in
 * oracle_correct_image, where band b starts at element b * height * pitch.
 * Tables are [column][x] with 2^bits entries per column.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* floor(v / 2^16) written as a plain floor division (C's '/' truncates) */
static int64_t floor_div_65536(int64_t v)
{
    int64_t q = v / 65536;
    if (v % 65536 != 0 && v < 0) q -= 1;
    return q;
}

/* (L): one LUT entry.  |A x^2| <= 2^31 (2^16 - 1)^2 < 2^63 - 2^47 for bits <= 16,
 * so the int64 sum is exact. */
int64_t oracle_lut_entry(int32_t A, int32_t G, int32_t O, int64_t x, int bits)
{
    const int64_t M = ((int64_t)1 << bits) - 1;
    const int64_t sum = (int64_t)A * x * x + (int64_t)G * x + (int64_t)O + 32768;
    int64_t d = floor_div_65536(sum);
    if (d < 0) d = 0;
    if (d > M) d = M;
    return d;
}

/* (L) for every column c < ncols and every x in [0, M]: lut[c * 2^bits + x] */
void oracle_lutgen(const int32_t* A, const int32_t* G, const int32_t* O, int ncols, int bits, uint16_t* lut)
{
    const int64_t L = (int64_t)1 << bits;
    for (int c = 0; c < ncols; ++c)
        for (int64_t x = 0; x < L; ++x)
            lut[(int64_t)c * L + x] = (uint16_t)oracle_lut_entry(A[c], G[c], O[c], x, bits);
}

/* (P): out[y][c] = lut[c][min(in[y][c], M)] */
void oracle_apply_u16(const uint16_t* in, int64_t in_pitch, int width, int height, int bits,
                      const uint16_t* lut, uint16_t* out, int64_t out_pitch)
{
    const int64_t L = (int64_t)1 << bits;
    const int64_t M = L - 1;
    for (int y = 0; y < height; ++y)
        for (int c = 0; c < width; ++c) {
            int64_t x = in[(int64_t)y * in_pitch + c];
            if (x > M) x = M;
            out[(int64_t)y * out_pitch + c] = lut[(int64_t)c * L + x];
        }
}

/* (H): hist[v] = #{(y, c) : lut[c][min(in[y][c], M)] == v}, hist has 2^bits entries */
void oracle_hist(const uint16_t* in, int64_t in_pitch, int width, int height, int bits,
                 const uint16_t* lut, uint64_t* hist)
{
    const int64_t L = (int64_t)1 << bits;
    const int64_t M = L - 1;
    memset(hist, 0, sizeof(uint64_t) * (size_t)L);
    for (int y = 0; y < height; ++y)
        for (int c = 0; c < width; ++c) {
            int64_t x = in[(int64_t)y * in_pitch + c];
            if (x > M) x = M;
            hist[lut[(int64_t)c * L + x]] += 1;
        }
}

/* (S): the 2 % / 98 % percentile stretch of one band's histogram.
 * lohi[0] = lo, lohi[1] = hi.  With an empty histogram (N = 0) every v
 * satisfies 100 cdf(v) >= 0, so lo = hi = 0 and S is all zero. */
void oracle_stretch(const uint64_t* hist, int bits, uint8_t* S, int32_t* lohi)
{
    const int64_t L = (int64_t)1 << bits;
    uint64_t N = 0;
    for (int64_t v = 0; v < L; ++v) N += hist[v];

    int64_t lo = -1, hi = -1;
    uint64_t cdf = 0;
    for (int64_t v = 0; v < L; ++v) {
        cdf += hist[v];
        if (lo < 0 && 100 * cdf >= 2 * N) lo = v;
        if (hi < 0 && 100 * cdf >= 98 * N) hi = v;
    }
    lohi[0] = (int32_t)lo;
    lohi[1] = (int32_t)hi;
    for (int64_t v = 0; v < L; ++v) {
        int64_t s;
        if (hi == lo) {
            s = 0;
        } else {
            s = ((v - lo) * 255 + (hi - lo) / 2) / (hi - lo);
            if (s < 0) s = 0;
            if (s > 255) s = 255;
        }
        S[v] = (uint8_t)s;
    }
}

/* (C): clut[c][x] = S[lut[c][x]]; an entry above M reads S[M] */
void oracle_compose(const uint16_t* lut, const uint8_t* S, int ncols, int bits, uint8_t* clut)
{
    const int64_t L = (int64_t)1 << bits;
    const int64_t M = L - 1;
    for (int c = 0; c < ncols; ++c)
        for (int64_t x = 0; x < L; ++x) {
            int64_t d = lut[(int64_t)c * L + x];
            if (d > M) d = M;
            clut[(int64_t)c * L + x] = S[d];
        }
}

/* (A): out[y][c] = clut[c][min(in[y][c], M)] */
void oracle_apply_u8(const uint16_t* in, int64_t in_pitch, int width, int height, int bits,
                     const uint8_t* clut, uint8_t* out, int64_t out_pitch)
{
    const int64_t L = (int64_t)1 << bits;
    const int64_t M = L - 1;
    for (int y = 0; y < height; ++y)
        for (int c = 0; c < width; ++c) {
            int64_t x = in[(int64_t)y * in_pitch + c];
            if (x > M) x = M;
            out[(int64_t)y * out_pitch + c] = clut[(int64_t)c * L + x];
        }
}

/*
 * The whole correction of a planar multi-band raster, as the chain of the
 * steps above, band by band.  A, G, O are [bands][width].  With stretch == 0
 * the output is the detector-corrected uint16 raster (P); otherwise it is the
 * uint8 raster (A) through the band's own histogram (H), stretch (S) and
 * composed table (C).  hist ([bands][2^bits]), S ([bands][2^bits]) and lohi
 * ([bands][2]) receive the per-band intermediates when not NULL (stretch only).
 * out rows use out_pitch elements of the output type.  Returns 0, or -1 if a
 * table allocation fails.
 */
int oracle_correct_image(const uint16_t* in, int64_t in_pitch, int width, int height, int bands, int bits,
                         const int32_t* A, const int32_t* G, const int32_t* O, int stretch,
                         void* out, int64_t out_pitch, uint64_t* hist_out, uint8_t* S_out, int32_t* lohi_out)
{
    const int64_t L = (int64_t)1 << bits;
    uint16_t* lut = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)(L * (width > 0 ? width : 1)));
    uint8_t* clut = (uint8_t*)malloc((size_t)(L * (width > 0 ? width : 1)));
    uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)L);
    uint8_t* S = (uint8_t*)malloc((size_t)L);
    if (!lut || !clut || !hist || !S) {
        free(lut); free(clut); free(hist); free(S);
        return -1;
    }
    for (int b = 0; b < bands; ++b) {
        const uint16_t* band_in = in + (int64_t)b * height * in_pitch;
        const int32_t* Ab = A + (int64_t)b * width;
        const int32_t* Gb = G + (int64_t)b * width;
        const int32_t* Ob = O + (int64_t)b * width;
        oracle_lutgen(Ab, Gb, Ob, width, bits, lut);
        if (!stretch) {
            uint16_t* band_out = (uint16_t*)out + (int64_t)b * height * out_pitch;
            oracle_apply_u16(band_in, in_pitch, width, height, bits, lut, band_out, out_pitch);
            continue;
        }
        int32_t lohi[2];
        oracle_hist(band_in, in_pitch, width, height, bits, lut, hist);
        oracle_stretch(hist, bits, S, lohi);
        oracle_compose(lut, S, width, bits, clut);
        uint8_t* band_out = (uint8_t*)out + (int64_t)b * height * out_pitch;
        oracle_apply_u8(band_in, in_pitch, width, height, bits, clut, band_out, out_pitch);
        if (hist_out) memcpy(hist_out + (int64_t)b * L, hist, sizeof(uint64_t) * (size_t)L);
        if (S_out) memcpy(S_out + (int64_t)b * L, S, (size_t)L);
        if (lohi_out) { lohi_out[2 * b] = lohi[0]; lohi_out[2 * b + 1] = lohi[1]; }
    }
    free(lut); free(clut); free(hist); free(S);
    return 0;
}
