/*
 * Seeded synthetic temporal graphs (R-MAT structure, configurable departure-time and
 * duration laws) shared by the oracle tests, the GPU parity tests and the benchmark.
 *
 * This file holds none of the temporal-path arithmetic: it only draws edge lists.
 *
 * Determinism: every random number is a pure function of (seed, edge index, draw number)
 * through the SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014), so the output does
 * not depend on the thread count.  The only floating point used is IEEE add/mul/div/sqrt
 * plus a logarithm and an exponential written out below (no libm transcendental), so
 * x86-64 and AArch64 builds produce identical graphs when compiled with
 * -ffp-contract=off (no fused multiply-add contraction).
 *
 * Edge model (Sec. 2.1 of the paper): a temporal edge (u, v, t, lambda) is valid over the
 * interval [t, t + lambda]; t is the departure (start) time, lambda the duration.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define SYNTH_TIME_UNIFORM 0
#define SYNTH_TIME_BURSTY 1
#define SYNTH_TIME_ZIPF 2
#define SYNTH_LAM_UNIFORM 0
#define SYNTH_LAM_GEOMETRIC 1

typedef struct {
    uint64_t seed;
    int64_t m;          /* number of edges */
    int32_t scale;      /* vertices = 2^scale */
    int32_t time_model; /* SYNTH_TIME_* */
    double a, b, c;     /* R-MAT quadrant probabilities (d = 1 - a - b - c) */
    uint64_t t_span;    /* departure times lie in [0, t_span) */
    int32_t n_bursts;   /* bursty model: number of Gaussian bursts */
    double burst_frac;  /* bursty model: fraction of edges drawn from a burst */
    double burst_sigma; /* bursty model: burst standard deviation */
    double zipf_s;      /* Zipf model: exponent */
    int32_t lam_model;  /* SYNTH_LAM_* */
    int32_t lam_bits;   /* 16 or 32: width of the output duration array */
    uint32_t lam_lo, lam_hi; /* uniform model: lambda in [lam_lo, lam_hi] */
    double lam_mean;    /* geometric model: mean of lambda on {1,2,...} */
} synth_params;

/* ---- counter-based random numbers ------------------------------------------------ */

uint64_t synth_sm64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw number d (< 256) of item i under `seed`. */
uint64_t synth_draw(uint64_t seed, uint64_t i, uint32_t d) {
    return synth_sm64(seed ^ synth_sm64((i << 8) | (uint64_t)(d & 0xFF)));
}

/* Uniform double in (0, 1): (k + 0.5) * 2^-53 with k the top 53 bits, never 0 or 1. */
static double u01(uint64_t r) { return ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/* Uniform integer in [0, n) for n <= 2^32, by a 32x32 multiply-high (exact integer). */
static uint64_t below(uint64_t r, uint64_t n) { return ((r >> 32) * n) >> 32; }

/* Natural logarithm for finite x > 0 with a normal exponent: x = f 2^e, f in
 * [sqrt(1/2), sqrt(2)), ln f = 2 artanh(s) with s = (f-1)/(f+1), |s| < 0.172, summed to
 * s^41 (truncation far below one ulp). */
static double det_log(double x) {
    uint64_t bits;
    memcpy(&bits, &x, 8);
    int e = (int)((bits >> 52) & 0x7FF) - 1023;
    bits = (bits & 0x000FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL;
    double f;
    memcpy(&f, &bits, 8);
    if (f > 1.4142135623730951) {
        f *= 0.5;
        e += 1;
    }
    double s = (f - 1.0) / (f + 1.0), s2 = s * s, term = s, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) {
        sum += term / (double)k;
        term *= s2;
    }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}

/* Exponential for |x| < 700: x = k ln2 + r with |r| <= ln2/2, e^r by its Taylor series
 * to r^24, then scaled by 2^k through the exponent field. */
static double det_exp(double x) {
    double kf = floor(x / 0.69314718055994530942 + 0.5);
    double r = x - kf * 0.69314718055994530942;
    double sum = 1.0, term = 1.0;
    for (int k = 1; k <= 24; ++k) {
        term *= r / (double)k;
        sum += term;
    }
    int k = (int)kf;
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double scale;
    memcpy(&scale, &bits, 8);
    return sum * scale;
}

/* Standard normal by Marsaglia's polar method, draws d0, d0+1, ... of item i. */
static double normal(uint64_t seed, uint64_t i, uint32_t d0, uint32_t dmax) {
    for (uint32_t d = d0; d + 1 < dmax; d += 2) {
        double x = 2.0 * u01(synth_draw(seed, i, d)) - 1.0;
        double y = 2.0 * u01(synth_draw(seed, i, d + 1)) - 1.0;
        double s = x * x + y * y;
        if (s < 1.0 && s > 0.0) return x * sqrt(-2.0 * det_log(s) / s);
    }
    return 0.0; /* unreachable in practice: 0.215^n rejection tail */
}

/* Zipf(s) on ranks {1..N} by rejection-inversion (Hormann & Derflinger, ACM TOMACS 1996),
 * with H(x) = ((x)^(1-s) - 1)/(1-s) the integral of x^-s.  Returns rank - 1. */
static double zipf_h(double x, double s) { return (det_exp((1.0 - s) * det_log(x)) - 1.0) / (1.0 - s); }
static double zipf_hinv(double y, double s) { return det_exp(det_log(1.0 + y * (1.0 - s)) / (1.0 - s)); }
/* The constants of one (N, s): H(3/2) - h(1), H(N + 1/2) and the squeeze bound. */
typedef struct {
    double hx0, hn, ss;
} zipf_consts;
static zipf_consts zipf_setup(uint64_t n, double s) {
    zipf_consts z;
    z.hx0 = zipf_h(1.5, s) - 1.0;
    z.hn = zipf_h((double)n + 0.5, s);
    z.ss = 2.0 - zipf_hinv(zipf_h(2.5, s) - det_exp(-s * det_log(2.0)), s);
    return z;
}
static uint64_t zipf(const zipf_consts *zc, uint64_t seed, uint64_t i, uint32_t d0, uint32_t dmax, uint64_t n,
                     double s) {
    const double hx0 = zc->hx0, hn = zc->hn, ss = zc->ss;
    for (uint32_t d = d0; d < dmax; ++d) {
        double u = hn + u01(synth_draw(seed, i, d)) * (hx0 - hn);
        double x = zipf_hinv(u, s);
        double k = floor(x + 0.5);
        if (k < 1.0) k = 1.0;
        if (k > (double)n) k = (double)n;
        if (k - x <= ss || u >= zipf_h(k + 0.5, s) - det_exp(-s * det_log(k))) return (uint64_t)k - 1;
    }
    return 0;
}

/* ---- the generator ---------------------------------------------------------------- */

/* Draw numbers: 0..31 R-MAT levels; 32..127 departure time; 128..255 duration. */
enum { D_TIME = 32, D_TIME_END = 128, D_LAM = 128, D_LAM_END = 256 };

typedef struct {
    const synth_params *p;
    int64_t lo, hi;
    int32_t *src, *dst;
    uint32_t *t;
    void *lam;
    const uint64_t *burst_centre;
} job;

/* Seeded bijection on [0, 2^scale) (multiply by an odd constant, xorshift, multiply),
 * so that R-MAT hubs are not all at small vertex ids. */
static uint64_t scramble(uint64_t x, int scale, uint64_t seed) {
    uint64_t mask = (scale >= 64) ? ~0ULL : ((1ULL << scale) - 1);
    uint64_t k1 = synth_sm64(seed ^ 0x5C4A31ULL) | 1ULL, k2 = synth_sm64(seed ^ 0x7B13ULL) | 1ULL;
    int sh = scale / 2 > 0 ? scale / 2 : 1;
    x = (x * k1) & mask;
    x ^= x >> sh;
    x = (x * k2) & mask;
    return x;
}

static void *run(void *arg) {
    job *J = (job *)arg;
    const synth_params *p = J->p;
    const double ab = p->a + p->b, abc = p->a + p->b + p->c;
    const uint64_t sd = p->seed;
    const zipf_consts zc = zipf_setup(p->t_span, p->zipf_s); /* used by the Zipf model only */
    for (int64_t i = J->lo; i < J->hi; ++i) {
        uint64_t u = 0, v = 0;
        for (int l = 0; l < p->scale; ++l) {
            /* quadrant of level l: [0, a) none, [a, a+b) v, [a+b, a+b+c) u, else both
             * (selected without branches: the draws are independent across levels) */
            double r = u01(synth_draw(sd, (uint64_t)i, (uint32_t)l));
            const uint64_t ge_a = r >= p->a, ge_ab = r >= ab, ge_abc = r >= abc;
            const int sh = p->scale - 1 - l;
            u |= ge_ab << sh;
            v |= ((ge_a & (ge_ab ^ 1u)) | ge_abc) << sh;
        }
        J->src[i] = (int32_t)scramble(u, p->scale, sd);
        J->dst[i] = (int32_t)scramble(v, p->scale, sd);

        uint64_t tt;
        if (p->time_model == SYNTH_TIME_UNIFORM) {
            tt = below(synth_draw(sd, (uint64_t)i, D_TIME), p->t_span);
        } else if (p->time_model == SYNTH_TIME_BURSTY) {
            if (u01(synth_draw(sd, (uint64_t)i, D_TIME)) < p->burst_frac) {
                uint64_t k = below(synth_draw(sd, (uint64_t)i, D_TIME + 1), (uint64_t)p->n_bursts);
                double z = normal(sd, (uint64_t)i, D_TIME + 2, D_TIME_END);
                double x = floor((double)J->burst_centre[k] + p->burst_sigma * z + 0.5);
                if (x < 0.0) x = 0.0;
                if (x > (double)(p->t_span - 1)) x = (double)(p->t_span - 1);
                tt = (uint64_t)x;
            } else {
                tt = below(synth_draw(sd, (uint64_t)i, D_TIME + 1), p->t_span);
            }
        } else {
            tt = zipf(&zc, sd, (uint64_t)i, D_TIME, D_TIME_END, p->t_span, p->zipf_s);
        }
        J->t[i] = (uint32_t)tt;

        uint64_t lam;
        if (p->lam_model == SYNTH_LAM_UNIFORM) {
            lam = p->lam_lo + below(synth_draw(sd, (uint64_t)i, D_LAM), (uint64_t)(p->lam_hi - p->lam_lo) + 1);
        } else {
            /* geometric on {1,2,...} with mean mu: 1 + floor(ln U / ln(1 - 1/mu)) */
            double q = det_log(1.0 - 1.0 / p->lam_mean);
            double g = floor(det_log(u01(synth_draw(sd, (uint64_t)i, D_LAM))) / q);
            lam = 1 + (uint64_t)g;
        }
        if (p->lam_bits == 16) {
            if (lam > 0xFFFF) lam = 0xFFFF;
            ((uint16_t *)J->lam)[i] = (uint16_t)lam;
        } else {
            ((uint32_t *)J->lam)[i] = (uint32_t)lam;
        }
    }
    return NULL;
}

/* Fill src/dst/t/lam[0..m).  lam is uint16_t* when lam_bits == 16, else uint32_t*.
 * nthreads <= 0 uses every online core.  Returns 0, or -1 on a bad parameter. */
int synth_rmat(const synth_params *p, int32_t *src, int32_t *dst, uint32_t *t, void *lam, int nthreads) {
    if (!p || p->scale < 1 || p->scale > 31 || p->m < 0 || p->t_span < 1 || p->t_span > (1ULL << 32)) return -1;
    if (p->time_model == SYNTH_TIME_BURSTY && (p->n_bursts < 1 || p->n_bursts > 1024)) return -1;
    if (p->lam_bits != 16 && p->lam_bits != 32) return -1;
    uint64_t centre[1024];
    if (p->time_model == SYNTH_TIME_BURSTY)
        for (int k = 0; k < p->n_bursts; ++k) centre[k] = below(synth_draw(p->seed ^ 0xB0B5ULL, (uint64_t)k, 0), p->t_span);
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > p->m / 4096 + 1) nthreads = (int)(p->m / 4096 + 1);
    pthread_t th[256];
    job jobs[256];
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].p = p;
        jobs[k].lo = p->m * k / nthreads;
        jobs[k].hi = p->m * (k + 1) / nthreads;
        jobs[k].src = src;
        jobs[k].dst = dst;
        jobs[k].t = t;
        jobs[k].lam = lam;
        jobs[k].burst_centre = centre;
    }
    int started = 0;
    for (int k = 1; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, run, &jobs[k]) != 0) break;
        started = k;
    }
    run(&jobs[0]);
    for (int k = started + 1; k < nthreads; ++k) run(&jobs[k]); /* threads that failed to start */
    for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    return 0;
}

/* Exposed for tests of the deterministic elementary functions. */
double synth_det_log(double x) { return det_log(x); }
double synth_det_exp(double x) { return det_exp(x); }
uint64_t synth_zipf_rank(uint64_t seed, uint64_t i, uint64_t n, double s) {
    const zipf_consts zc = zipf_setup(n, s);
    return zipf(&zc, seed, i, 0, 128, n, s);
}
