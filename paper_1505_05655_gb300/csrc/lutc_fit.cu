// Per-detector least-squares polynomial fit (paper, Section III.B, case study 2).
//
// Each column c owns n calibration samples (x[i][c], y_i): the raw value the
// detector read on calibration line i and the value it should have read.
// The fit of order m (1..3) minimises sum_i (y_i - f(x_i))^2 over
// f(x) = a_0 + ... + a_m x^m, i.e. solves the normal equations
// sum_k a_k P[j+k] = Q[j] with P[k] = sum_i x_i^k and Q[j] = sum_i x_i^j y_i.
//
// GB300 mapping: one thread per column, the n lines walked in order, so that a
// warp reads 64 contiguous bytes of a calibration line per step (coalesced)
// and the target y_i, when shared by the line, is one broadcast load.  The
// (m+1)x(m+1) system is symmetric positive definite whenever the column has
// at least m+1 distinct abscissae; it is solved in registers by a Cholesky
// factorisation (the paper forms A^-1 B; in exact arithmetic the result is the
// same X, and the factorisation is the better-conditioned route to it).  The
// column's distinct abscissae are counted exactly, so a singular system is
// recognised without a floating-point test.
//
// The power sums P are exact integer sums (x^6 < 2^96, 128-bit accumulators);
// the moments Q and the solve are fp64.  Once n is large the kernel is bound
// by GB300's fp64 issue rate (2m + 1 fp64 instructions per sample); at the
// paper's size (6 lines of 6000 detectors) it is launch- and latency-bound.
#include <math.h>
#include <stdint.h>

#include "lutc_internal.cuh"

namespace lutc {
namespace {

// Exact power sums of one column.  x < 2^16, so x^2 < 2^32, x^3 < 2^48 and
// x^4 < 2^64 are exact in unsigned integers; x^5 and x^6 (< 2^96) and the
// sums from x^4 up are carried in 128 bits.  Only the moments Q[j], which
// involve the fp64 targets, use the fp64 pipe, whose issue rate on GB300 is a
// small fraction of the integer pipe's.
template <int M>
struct PowerSums {
    uint64_t p1 = 0, p2 = 0, p3 = 0;
    unsigned __int128 p4 = 0, p5 = 0, p6 = 0;

    __device__ __forceinline__ void add(uint32_t x)
    {
        const uint32_t x2 = x * x;
        p1 += x;
        p2 += x2;
        if (M >= 2) {
            const uint64_t x3 = (uint64_t)x2 * x;
            const uint64_t x4 = (uint64_t)x2 * x2;
            p3 += x3;
            p4 += x4;
            if (M >= 3) {
                p5 += (unsigned __int128)x4 * x;
                p6 += (unsigned __int128)x3 * x3;
            }
        }
    }
};

__device__ __forceinline__ double u128_to_double(unsigned __int128 v)
{
    // two correctly rounded halves: a relative error of at most one unit in the last place
    return fma((double)(uint64_t)(v >> 64), 18446744073709551616.0, (double)(uint64_t)v);
}

template <int M>
__global__ void __launch_bounds__(64) k_fit(const uint16_t* __restrict__ x, int64_t x_pitch,
                                           const double* __restrict__ y, int64_t y_pitch, int n, int ncols,
                                           double* __restrict__ coef, int32_t* __restrict__ status,
                                           int32_t* __restrict__ q16)
{
    constexpr int D = M + 1;
    constexpr int U = 8;  // lines loaded per step: their loads are in flight together
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const uint16_t* xc = x + c;
    const double* yc = y_pitch ? y + c : y;
    const int64_t ys = y_pitch ? y_pitch : 1;

    PowerSums<M> ps;
    double Q[D];
#pragma unroll
    for (int k = 0; k < D; ++k) Q[k] = 0.0;
    uint32_t seen[D] = {};
    int distinct = 0;
    for (int i0 = 0; i0 < n; i0 += U) {
        uint32_t xv[U];
        double yv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u < n ? i0 + u : n - 1;
            xv[u] = __ldg(xc + (int64_t)i * x_pitch);
            yv[u] = __ldg(yc + (int64_t)i * ys);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u >= n) break;
            const uint32_t xi = xv[u];
            bool fresh = distinct < D;
#pragma unroll
            for (int k = 0; k < D; ++k) fresh = fresh && !(k < distinct && seen[k] == xi);
            if (fresh) {
#pragma unroll
                for (int k = 0; k < D; ++k)
                    if (k == distinct) seen[k] = xi;
                ++distinct;
            }
            ps.add(xi);
            // x^j for j <= 3 is below 2^53: the products are exact
            const double xd = (double)xi;
            double pw = xd;
            Q[0] += yv[u];
#pragma unroll
            for (int k = 1; k < D; ++k) {
                Q[k] = fma(pw, yv[u], Q[k]);
                pw *= xd;
            }
        }
    }
    double P[2 * M + 1];
    P[0] = (double)n;
    P[1] = (double)ps.p1;
    P[2] = (double)ps.p2;
    if (M >= 2) {
        P[3] = (double)ps.p3;
        P[4] = u128_to_double(ps.p4);
    }
    if (M >= 3) {
        P[5] = u128_to_double(ps.p5);
        P[6] = u128_to_double(ps.p6);
    }

    double a[D];
    int st = 0;
    if (distinct < D) {
        st = 1;
#pragma unroll
        for (int k = 0; k < D; ++k) a[k] = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
    } else {
        // Cholesky: normal matrix N[j][k] = P[j+k] = L L^T, lower triangle in L; rinv[k] = 1 / L[k][k]
        // from one reciprocal square root per pivot, so the solve needs no division
        double L[D][D], rinv[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
#pragma unroll
            for (int k = 0; k <= j; ++k) {
                double s = P[j + k];
#pragma unroll
                for (int t = 0; t < k; ++t) s -= L[j][t] * L[k][t];
                if (j == k) {
                    rinv[j] = rsqrt(s);
                    L[j][j] = s * rinv[j];
                } else {
                    L[j][k] = s * rinv[k];
                }
            }
        }
        double z[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double s = Q[j];
#pragma unroll
            for (int t = 0; t < j; ++t) s -= L[j][t] * z[t];
            z[j] = s * rinv[j];
        }
#pragma unroll
        for (int j = D - 1; j >= 0; --j) {
            double s = z[j];
#pragma unroll
            for (int t = j + 1; t < D; ++t) s -= L[t][j] * a[t];
            a[j] = s * rinv[j];
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) coef[(int64_t)c * D + k] = a[k];
    if (q16) {
        // Q16 codes of D(x) = A x^2 + G x + O: round half away from zero, |code| <= 2^31 - 1
        int32_t code[3] = {0, 0, 0};
        if (st == 0) {
            const double v[3] = {M >= 2 ? a[2 < D ? 2 : 0] * 65536.0 : 0.0, a[1] * 65536.0, a[0] * 65536.0};
            bool fits = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) fits = fits && fabs(v[k]) < 2147483647.5;
            if (fits) {
#pragma unroll
                for (int k = 0; k < 3; ++k) code[k] = (int32_t)llround(v[k]);
            } else {
                st = 2;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) q16[(int64_t)k * ncols + c] = code[k];
    }
    status[c] = st;
}

}  // namespace
}  // namespace lutc

using namespace lutc;

extern "C" int lutc_fit(const uint16_t* x, int64_t x_pitch_bytes, const double* y, int64_t y_pitch_bytes, int n,
                        int ncols, int order, double* coef, int32_t* status, int32_t* q16, lutc_stream stream)
{
    if (order < 1 || order > LUTC_FIT_MAX_ORDER || n < order + 1 || n > LUTC_FIT_MAX_LINES || ncols < 0)
        return LUTC_EINVAL;
    if (q16 && order > 2) return LUTC_EINVAL;
    if (ncols == 0) return LUTC_OK;
    if (!x || !y || !coef || !status) return LUTC_EINVAL;
    if (((uintptr_t)x % 2) || ((uintptr_t)y % 8) || ((uintptr_t)coef % 8) || ((uintptr_t)status % 4) ||
        ((uintptr_t)q16 % 4))
        return LUTC_EINVAL;
    if (x_pitch_bytes < 2 * (int64_t)ncols || (x_pitch_bytes % 2)) return LUTC_EINVAL;
    if (y_pitch_bytes != 0 && (y_pitch_bytes < 8 * (int64_t)ncols || (y_pitch_bytes % 8))) return LUTC_EINVAL;
    const int64_t xp = x_pitch_bytes / 2, yp = y_pitch_bytes / 8;
    const int threads = 64;
    const int blocks = (ncols + threads - 1) / threads;
    cudaStream_t st = (cudaStream_t)stream;
    switch (order) {
    case 1: k_fit<1><<<blocks, threads, 0, st>>>(x, xp, y, yp, n, ncols, coef, status, q16); break;
    case 2: k_fit<2><<<blocks, threads, 0, st>>>(x, xp, y, yp, n, ncols, coef, status, q16); break;
    default: k_fit<3><<<blocks, threads, 0, st>>>(x, xp, y, yp, n, ncols, coef, status, q16); break;
    }
    return cuda_status(cudaGetLastError());
}
