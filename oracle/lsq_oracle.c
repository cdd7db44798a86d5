/* CPU oracle of the per-detector least-squares polynomial fit (paper, Section III.B, case study 2).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, single-threaded fp64 C that the CUDA
 * fit is checked against.  It shares no code with the CUDA path.
 *
 * Each detector (column c) has n calibration samples (x_i, y_i): x_i the raw
 * value the detector read on calibration line i, y_i the value it should have
 * read.  The fit of order m minimises the summed squared error of
 * f(x) = a_0 + a_1 x + ... + a_m x^m over the samples.  The paper sets the
 * first derivatives of that error to zero, which gives the normal equations
 *
 *     sum_k a_k * P[j + k] = Q[j],   j = 0..m,
 *     P[k] = sum_i x_i^k   (P[0] = n),   Q[j] = sum_i x_i^j y_i,
 *
 * and obtains the coefficients as X = A^-1 B with A[j][k] = P[j + k] and
 * B[j] = Q[j].  The steps below follow that order:
 *   F1  power sums P[0..2m] and moments Q[0..m], accumulated over i = 0..n-1
 *   F2  the normal matrix A and right-hand side B
 *   F3  the inverse of A by Gauss-Jordan elimination (A is symmetric positive
 *       definite when the column has at least m+1 distinct abscissae, so the
 *       elimination needs no row exchanges)
 *   F4  X = A^-1 B
 * A column with fewer than m+1 distinct abscissae has a singular A: its
 * coefficients are NaN and its status is 1 (decided by counting distinct x
 * values, exactly).
 *
 * Q16 export (orders 1 and 2): the detector LUT takes D(x) = A x^2 + G x + O
 * in Q16 fixed point, so O = round(a_0 * 2^16), G = round(a_1 * 2^16),
 * A = round(a_2 * 2^16) (0 for order 1), rounding half away from zero
 * (llround).  A code of magnitude above 2^31 - 1 sets status 2 and all three
 * codes to 0.
 *
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define FIT_MAX_ORDER 3

/* number of distinct values among x[0], x[pitch], ..., capped at cap */
static int distinct_upto(const uint16_t* x, int64_t pitch, int n, int cap)
{
    uint16_t seen[FIT_MAX_ORDER + 1];
    int count = 0;
    for (int i = 0; i < n && count < cap; ++i) {
        const uint16_t v = x[(int64_t)i * pitch];
        int fresh = 1;
        for (int k = 0; k < count; ++k)
            if (seen[k] == v) fresh = 0;
        if (fresh) seen[count++] = v;
    }
    return count;
}

/* Fit of one column: x_i = x[i * x_pitch], y_i = y[i * y_pitch] (strides in
 * elements), i = 0..n-1; writes the m+1 coefficients a_0..a_m to coef. */
static int fit_column(const uint16_t* x, int64_t x_pitch, const double* y, int64_t y_pitch, int n, int m,
                      double* coef)
{
    if (distinct_upto(x, x_pitch, n, m + 1) < m + 1) {
        for (int j = 0; j <= m; ++j) coef[j] = NAN;
        return 1;
    }
    /* F1 */
    double P[2 * FIT_MAX_ORDER + 1], Q[FIT_MAX_ORDER + 1];
    for (int k = 0; k <= 2 * m; ++k) P[k] = 0.0;
    for (int j = 0; j <= m; ++j) Q[j] = 0.0;
    for (int i = 0; i < n; ++i) {
        const double xi = (double)x[(int64_t)i * x_pitch];
        const double yi = y[(int64_t)i * y_pitch];
        double pw = 1.0; /* xi^k */
        for (int k = 0; k <= 2 * m; ++k) {
            P[k] += pw;
            if (k <= m) Q[k] += pw * yi;
            pw *= xi;
        }
    }
    /* F2 */
    const int d = m + 1;
    double A[FIT_MAX_ORDER + 1][FIT_MAX_ORDER + 1], inv[FIT_MAX_ORDER + 1][FIT_MAX_ORDER + 1];
    for (int j = 0; j < d; ++j)
        for (int k = 0; k < d; ++k) {
            A[j][k] = P[j + k];
            inv[j][k] = (j == k) ? 1.0 : 0.0;
        }
    /* F3: Gauss-Jordan on [A | I] */
    for (int p = 0; p < d; ++p) {
        const double piv = A[p][p];
        for (int k = 0; k < d; ++k) {
            A[p][k] /= piv;
            inv[p][k] /= piv;
        }
        for (int r = 0; r < d; ++r) {
            if (r == p) continue;
            const double f = A[r][p];
            for (int k = 0; k < d; ++k) {
                A[r][k] -= f * A[p][k];
                inv[r][k] -= f * inv[p][k];
            }
        }
    }
    /* F4 */
    for (int j = 0; j < d; ++j) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += inv[j][k] * Q[k];
        coef[j] = s;
    }
    return 0;
}

/* x: [n][x_pitch] uint16; y: [n][y_pitch] doubles, or one double per line when y_pitch == 0;
 * coef: [ncols][order+1]; status: [ncols] (0 ok, 1 singular, 2 Q16 overflow);
 * q16: NULL or [3][ncols] int32 (A, G, O) for order <= 2. */
void oracle_polyfit(const uint16_t* x, int64_t x_pitch, const double* y, int64_t y_pitch, int n, int ncols,
                    int order, double* coef, int32_t* status, int32_t* q16)
{
    for (int c = 0; c < ncols; ++c) {
        const double* yc = y_pitch ? y + c : y;
        const int64_t ys = y_pitch ? y_pitch : 1;
        double* a = coef + (int64_t)c * (order + 1);
        int st = fit_column(x + c, x_pitch, yc, ys, n, order, a);
        if (q16) {
            int32_t codes[3] = {0, 0, 0}; /* A, G, O */
            if (st == 0) {
                const double scaled[3] = {order >= 2 ? a[2] * 65536.0 : 0.0, a[1] * 65536.0, a[0] * 65536.0};
                for (int k = 0; k < 3; ++k) {
                    if (!(fabs(scaled[k]) < 2147483647.5)) st = 2;
                }
                if (st == 0)
                    for (int k = 0; k < 3; ++k) codes[k] = (int32_t)llround(scaled[k]);
            }
            for (int k = 0; k < 3; ++k) q16[(int64_t)k * ncols + c] = codes[k];
        }
        status[c] = st;
    }
}
