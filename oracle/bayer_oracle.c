/* CPU oracle of bilinear Bayer demosaicing (paper, Section III.A, case study 1).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, single-threaded C that the CUDA
 * demosaic is checked against.  It shares no code with the CUDA path.
 *
 * A Bayer colour filter array gives each photosite one of red, green, blue:
 * every 2x2 square holds one red, one blue and two greens.  The paper's
 * bilinear method keeps a pixel's own colour and obtains each of its two
 * missing colours as the average of the neighbouring pixels of that colour
 * among its 8 direct neighbours.  Written out for every pixel (y, x) and
 * colour k:
 *
 *   out[k][y][x] = v(y, x)                                   if colour(y, x) == k
 *                = round( sum_{(dy,dx) in N, colour(y+dy, x+dx) == k} v(y+dy, x+dx) / count )
 *
 * where N is the 8-neighbourhood clipped to the image, count the number of
 * summed pixels, and round() is round-half-up in integers:
 * (sum + count / 2) / count.  A colour with no neighbour inside the image
 * (only possible for images 1 pixel wide or high) is 0.  v is the raw value,
 * or the detector-corrected value D[x][raw] when a per-column LUT is given
 * (the correction then precedes the interpolation).
 *
 * CFA patterns name the 2x2 cell row by row: RGGB (R at even row, even
 * column), BGGR, GRBG, GBRG.  Output is planar: R, G, B planes of height rows.
 */
#include <stdint.h>

enum { CH_R = 0, CH_G = 1, CH_B = 2 };

/* colour of the photosite at (y, x) under pattern p */
static int cfa_colour(int pattern, int64_t y, int64_t x)
{
    static const int cell[4][4] = {
        {CH_R, CH_G, CH_G, CH_B}, /* RGGB */
        {CH_B, CH_G, CH_G, CH_R}, /* BGGR */
        {CH_G, CH_R, CH_B, CH_G}, /* GRBG */
        {CH_G, CH_B, CH_R, CH_G}, /* GBRG */
    };
    return cell[pattern][2 * (int)(y & 1) + (int)(x & 1)];
}

/* in: uint16 [height][in_pitch]; lut: NULL or uint16 [width][2^bits] (entry min(raw, 2^bits - 1));
 * out: uint16 [3][height][out_pitch] (out_pitch in elements). */
void oracle_demosaic(const uint16_t* in, int64_t in_pitch, int width, int height, int pattern, const uint16_t* lut,
                     int bits, uint16_t* out, int64_t out_pitch)
{
    const int64_t L = (int64_t)1 << bits;
    for (int64_t y = 0; y < height; ++y) {
        for (int64_t x = 0; x < width; ++x) {
            const int own = cfa_colour(pattern, y, x);
            for (int k = 0; k < 3; ++k) {
                uint32_t result;
                if (k == own) {
                    uint32_t raw = in[y * in_pitch + x];
                    result = lut ? lut[x * L + (raw < (uint32_t)(L - 1) ? raw : (uint32_t)(L - 1))] : raw;
                } else {
                    uint64_t sum = 0;
                    uint32_t count = 0;
                    for (int dy = -1; dy <= 1; ++dy) {
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int64_t yy = y + dy, xx = x + dx;
                            if ((dy == 0 && dx == 0) || yy < 0 || yy >= height || xx < 0 || xx >= width) continue;
                            if (cfa_colour(pattern, yy, xx) != k) continue;
                            uint32_t raw = in[yy * in_pitch + xx];
                            if (lut) raw = lut[xx * L + (raw < (uint32_t)(L - 1) ? raw : (uint32_t)(L - 1))];
                            sum += raw;
                            ++count;
                        }
                    }
                    result = count ? (uint32_t)((sum + count / 2) / count) : 0u;
                }
                out[((int64_t)k * height + y) * out_pitch + x] = (uint16_t)result;
            }
        }
    }
}
