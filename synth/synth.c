/*
 * Seeded synthetic inputs for detector LUT generation and LUT-based image
 * correction: raw uint16 scenes and per-column Q16 coefficient triples.
 *
 * This module only draws inputs.  It holds none of the correction arithmetic
 * (no LUT, histogram, percentile or stretch), so the CPU oracle and the CUDA
 * path can both consume its buffers without sharing any of the method.
 *
 * The paper (Section I) names LUT generation and image correction as a task
 * and says nothing of the detector data beyond it arriving in scan lines
 * (Section III-B); the scene recipe below is this library's stand-in for such
 * data: a smooth radiance field, per-detector stripes and sensor noise.
 *
 * Randomness is counter based: every variate is a pure function of
 * (seed, stream, index) through the SplitMix64 finaliser (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so
 * the output does not depend on the number of threads used.  Transcendental
 * functions come from the host libm, so two different machines may differ in
 * the last DN of a few pixels; parity never regenerates inputs on two sides,
 * both sides read the same host buffers.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define SYNTH_TWO_PI 6.283185307179586476925286766559

/* stream kinds; the stream id of a band is (band << 8) | kind */
enum {
    K_WAVES = 1,   /* sinusoid parameters of the scene */
    K_STRIPE = 2,  /* per-column additive stripe */
    K_NOISE = 3,   /* per-pixel Gaussian noise (two uniforms per pixel) */
    K_SAT = 4,     /* per-pixel saturation draw */
    K_DEAD = 5,    /* per-column dead-detector draw */
    K_GAIN = 6,
    K_OFFS = 7,
    K_QUAD = 8,
    K_BATCH = 9,   /* image specification of a batch (band argument = 0) */
    K_CAL = 10     /* calibration scan lines: per-column response and per-sample noise */
};

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t synth_hash(uint64_t seed, uint64_t stream, uint64_t index)
{
    uint64_t key = mix64(seed * 0x9e3779b97f4a7c15ULL + 0x632be59bd9b4e019ULL);
    key = mix64(key ^ (stream * 0xd1b54a32d192ed03ULL));
    return mix64(key + (index + 1) * 0x9e3779b97f4a7c15ULL);
}

/* uniform in [0, 1) with 53 random bits */
double synth_u01(uint64_t seed, uint64_t stream, uint64_t index)
{
    return (double)(synth_hash(seed, stream, index) >> 11) * (1.0 / 9007199254740992.0);
}

static inline uint64_t sid(int band, int kind) { return ((uint64_t)band << 8) | (uint64_t)kind; }

/* ------------------------------------------------------------------------ */
/* scene */

typedef struct {
    uint64_t seed;
    int band, width, height, bits;
    double dead_frac, sat_frac;
    uint16_t* out;
    int64_t pitch;          /* elements */
    /* separable sinusoid tables: sin/cos(alpha_k x) per column, sin/cos(beta_k y + phi_k) per row */
    const double* cx;       /* [4][width] cos */
    const double* sx;       /* [4][width] sin */
    const double* cy;       /* [4][height] */
    const double* sy;       /* [4][height] */
    const double* amp;      /* [4] a_k / sum a */
    const double* stripe;   /* [width] */
    const unsigned char* dead; /* [width] */
    double m0, r;
    int y0, y1;
} scene_job;

static void* scene_rows(void* arg)
{
    const scene_job* j = (const scene_job*)arg;
    const int32_t maxdn = (int32_t)((1u << j->bits) - 1u);
    const int W = j->width;
    for (int y = j->y0; y < j->y1; ++y) {
        uint16_t* row = j->out + (int64_t)y * j->pitch;
        double cyk[4], syk[4];
        for (int k = 0; k < 4; ++k) {
            cyk[k] = j->cy[k * j->height + y];
            syk[k] = j->sy[k * j->height + y];
        }
        for (int x = 0; x < W; ++x) {
            if (j->dead[x]) { row[x] = 0; continue; }
            double s = 0.0;
            for (int k = 0; k < 4; ++k)  /* sin(a + b) = sin a cos b + cos a sin b */
                s += j->amp[k] * (j->sx[k * W + x] * cyk[k] + j->cx[k * W + x] * syk[k]);
            const uint64_t i = (uint64_t)y * (uint64_t)W + (uint64_t)x;
            const double u1 = 1.0 - synth_u01(j->seed, sid(j->band, K_NOISE), 2 * i);
            const double u2 = synth_u01(j->seed, sid(j->band, K_NOISE), 2 * i + 1);
            const double z = sqrt(-2.0 * log(u1)) * cos(SYNTH_TWO_PI * u2);  /* Box-Muller */
            double v = j->m0 + j->r * s + j->stripe[x] + 20.0 * z;
            long long dn = llround(v);
            if (dn < 0) dn = 0;
            if (dn > maxdn) dn = maxdn;
            if (j->sat_frac > 0.0 && synth_u01(j->seed, sid(j->band, K_SAT), i) < j->sat_frac)
                dn = maxdn;
            row[x] = (uint16_t)dn;
        }
    }
    return NULL;
}

/*
 * One band of a scene, H rows x W columns, DN in [0, 2^bits - 1], written to
 * out[y * pitch + x].  Scene = M0 + R * sum_k a_k sin(2 pi (x cos t_k + y sin t_k)/P_k + p_k) / sum_k a_k
 * with 4 waves, P_k log-uniform in [32, 512] px, t_k ~ U(0, pi), p_k ~ U(0, 2 pi),
 * a_k ~ U(0.5, 1), M0 = 2000 * 2^(bits-12), R = 1500 * 2^(bits-12); plus a
 * per-column stripe ~ U(-50, 50) and Gaussian noise of sigma 20; rounded and
 * clipped.  Then a fraction sat_frac of pixels is set to 2^bits - 1 and a
 * fraction dead_frac of columns (Bernoulli per column) is constant 0.
 * nthreads <= 0 uses every online core.  Returns 0, or -1 on bad arguments.
 */
int synth_scene(uint64_t seed, int band, int width, int height, int bits,
                double dead_frac, double sat_frac, uint16_t* out, int64_t pitch, int nthreads)
{
    if (width < 0 || height < 0 || bits < 1 || bits > 16 || pitch < width || !out) return -1;
    if (width == 0 || height == 0) return 0;
    const double scale = ldexp(1.0, bits - 12);
    double amp[4], alpha[4], beta[4], phi[4], asum = 0.0;
    for (int k = 0; k < 4; ++k) {
        const double up = synth_u01(seed, sid(band, K_WAVES), 4 * k + 0);
        const double ut = synth_u01(seed, sid(band, K_WAVES), 4 * k + 1);
        const double uf = synth_u01(seed, sid(band, K_WAVES), 4 * k + 2);
        const double ua = synth_u01(seed, sid(band, K_WAVES), 4 * k + 3);
        const double period = 32.0 * pow(16.0, up);
        const double theta = M_PI * ut;
        phi[k] = SYNTH_TWO_PI * uf;
        amp[k] = 0.5 + 0.5 * ua;
        alpha[k] = SYNTH_TWO_PI * cos(theta) / period;
        beta[k] = SYNTH_TWO_PI * sin(theta) / period;
        asum += amp[k];
    }
    for (int k = 0; k < 4; ++k) amp[k] /= asum;

    double* cx = (double*)malloc(sizeof(double) * 4 * (size_t)width);
    double* sx = (double*)malloc(sizeof(double) * 4 * (size_t)width);
    double* cy = (double*)malloc(sizeof(double) * 4 * (size_t)height);
    double* sy = (double*)malloc(sizeof(double) * 4 * (size_t)height);
    double* stripe = (double*)malloc(sizeof(double) * (size_t)width);
    unsigned char* dead = (unsigned char*)malloc((size_t)width);
    if (!cx || !sx || !cy || !sy || !stripe || !dead) {
        free(cx); free(sx); free(cy); free(sy); free(stripe); free(dead);
        return -1;
    }
    for (int k = 0; k < 4; ++k) {
        for (int x = 0; x < width; ++x) {
            cx[k * width + x] = cos(alpha[k] * x);
            sx[k * width + x] = sin(alpha[k] * x);
        }
        for (int y = 0; y < height; ++y) {
            cy[k * height + y] = cos(beta[k] * y + phi[k]);
            sy[k * height + y] = sin(beta[k] * y + phi[k]);
        }
    }
    for (int x = 0; x < width; ++x) {
        stripe[x] = -50.0 + 100.0 * synth_u01(seed, sid(band, K_STRIPE), (uint64_t)x);
        dead[x] = (unsigned char)(dead_frac > 0.0 && synth_u01(seed, sid(band, K_DEAD), (uint64_t)x) < dead_frac);
    }

    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > height) nthreads = height;
    if (nthreads > 256) nthreads = 256;
    scene_job jobs[256];
    pthread_t tids[256];
    int started[256];
    for (int t = 0; t < nthreads; ++t) {
        scene_job* j = &jobs[t];
        j->seed = seed; j->band = band; j->width = width; j->height = height; j->bits = bits;
        j->dead_frac = dead_frac; j->sat_frac = sat_frac; j->out = out; j->pitch = pitch;
        j->cx = cx; j->sx = sx; j->cy = cy; j->sy = sy; j->amp = amp; j->stripe = stripe; j->dead = dead;
        j->m0 = 2000.0 * scale; j->r = 1500.0 * scale;
        j->y0 = (int)((int64_t)height * t / nthreads);
        j->y1 = (int)((int64_t)height * (t + 1) / nthreads);
    }
    for (int t = 1; t < nthreads; ++t)
        started[t] = pthread_create(&tids[t], NULL, scene_rows, &jobs[t]) == 0;
    scene_rows(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (started[t]) pthread_join(tids[t], NULL);
        else scene_rows(&jobs[t]);
    }
    free(cx); free(sx); free(cy); free(sy); free(stripe); free(dead);
    return 0;
}

/*
 * Per-column Q16 coefficients of one band: gain g ~ U(0.9, 1.1), offset
 * o ~ U(-20, 20), quadratic a ~ U(-2e-5, 2e-5), each stored as llround(r * 2^16).
 */
void synth_coeffs(uint64_t seed, int band, int width, int32_t* A, int32_t* G, int32_t* O)
{
    for (int c = 0; c < width; ++c) {
        const double g = 0.9 + 0.2 * synth_u01(seed, sid(band, K_GAIN), (uint64_t)c);
        const double o = -20.0 + 40.0 * synth_u01(seed, sid(band, K_OFFS), (uint64_t)c);
        const double a = -2e-5 + 4e-5 * synth_u01(seed, sid(band, K_QUAD), (uint64_t)c);
        G[c] = (int32_t)llround(g * 65536.0);
        O[c] = (int32_t)llround(o * 65536.0);
        A[c] = (int32_t)llround(a * 65536.0);
    }
}

/*
 * Image specifications of a batch of n independent images: width
 * round(512 * 16^u) in [512, 8192], height round(256 * 32^u) in [256, 8192],
 * bits uniform over {10, 12, 14}, bands uniform over {1, 3, 4}.
 */
void synth_batch_spec(uint64_t seed, int n, int32_t* width, int32_t* height, int32_t* bits, int32_t* bands)
{
    static const int32_t bit_set[3] = {10, 12, 14};
    static const int32_t band_set[3] = {1, 3, 4};
    for (int i = 0; i < n; ++i) {
        const uint64_t b = 4 * (uint64_t)i;
        width[i] = (int32_t)llround(512.0 * pow(16.0, synth_u01(seed, K_BATCH, b + 0)));
        height[i] = (int32_t)llround(256.0 * pow(32.0, synth_u01(seed, K_BATCH, b + 1)));
        int kb = (int)(3.0 * synth_u01(seed, K_BATCH, b + 2));
        int kn = (int)(3.0 * synth_u01(seed, K_BATCH, b + 3));
        bits[i] = bit_set[kb > 2 ? 2 : kb];
        bands[i] = band_set[kn > 2 ? 2 : kn];
    }
}

/*
 * Flat-field calibration scan lines for the per-detector polynomial fit.
 * Line i (0 <= i < n) images a uniform target of level
 *     L_i = M * (0.05 + 0.9 * (i + 0.5) / n),  M = 2^bits - 1,
 * and detector c reads x = clamp(round(b_c + h_c L_i + q_c L_i^2 + e), 0, M)
 * with gain h_c ~ U(0.9, 1.1), offset b_c ~ U(-20, 20), curvature
 * q_c ~ U(-2e-5, 2e-5) (scaled by 2^(12 - bits) so that its effect at full
 * scale is the same at every bit depth) and e ~ N(0, 2) per sample.  A
 * fraction dead_frac of the columns read 0 on every line.  x is [n][pitch]
 * uint16, y receives the n levels.
 */
void synth_calib(uint64_t seed, int n, int width, int bits, double dead_frac, uint16_t* x, int64_t pitch, double* y)
{
    const double M = (double)((1u << bits) - 1u);
    const double qscale = ldexp(1.0, 12 - bits);
    for (int i = 0; i < n; ++i) y[i] = M * (0.05 + 0.9 * (i + 0.5) / n);
    for (int c = 0; c < width; ++c) {
        const uint64_t st = sid(0, K_CAL);
        const double h = 0.9 + 0.2 * synth_u01(seed, st, 4 * (uint64_t)c + 0);
        const double b = -20.0 + 40.0 * synth_u01(seed, st, 4 * (uint64_t)c + 1);
        const double q = (-2e-5 + 4e-5 * synth_u01(seed, st, 4 * (uint64_t)c + 2)) * qscale;
        const int dead = synth_u01(seed, st, 4 * (uint64_t)c + 3) < dead_frac;
        for (int i = 0; i < n; ++i) {
            uint16_t v = 0;
            if (!dead) {
                const uint64_t k = 2 * ((uint64_t)i * (uint64_t)width + (uint64_t)c);
                const double u1 = synth_u01(seed, sid(1, K_CAL), k);
                const double u2 = synth_u01(seed, sid(1, K_CAL), k + 1);
                const double e = 2.0 * sqrt(-2.0 * log(1.0 - u1)) * cos(SYNTH_TWO_PI * u2);
                double r = llround(b + h * y[i] + q * y[i] * y[i] + e);
                v = (uint16_t)(r < 0 ? 0 : (r > M ? M : r));
            }
            x[(int64_t)i * pitch + c] = v;
        }
    }
}
