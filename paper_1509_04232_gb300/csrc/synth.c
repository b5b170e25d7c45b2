/*
 * Seeded synthetic test images: Voronoi colour regions, a global linear
 * colour gradient and Gaussian noise, optionally animated as a video
 * (regions translating at a constant per-region velocity, region colours
 * drifting as a Gaussian random walk).
 *
 * This file produces INPUTS only. It contains none of SLIC's arithmetic and
 * is shared by the CUDA path, the FP64 oracle's tests and the benchmark so
 * that every side reads identical bytes.
 *
 * Random numbers: every draw is a pure function of (seed, stream, index),
 * computed with the SplitMix64 output function (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014). The output
 * therefore does not depend on the number of threads used.
 *
 * Normal variates: Box-Muller transform of two uniforms in (0,1).
 * Rounding: values are clipped to [0,255] and rounded half-to-even.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* SplitMix64 finaliser applied to a 64-bit counter value. */
static inline uint64_t sm64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of draw `idx` of stream `stream` under `seed`. */
static inline uint64_t key3(uint64_t seed, uint64_t stream, uint64_t idx) {
    return sm64(sm64(seed ^ (stream * 0xD1B54A32D192ED03ULL)) + idx);
}

/* Uniform in (0,1) from 32 bits. */
static inline double u32_open(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

/* Uniform in [0,1) from the top 53 bits. */
static inline double u53(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* Two standard normals from one 64-bit draw (Box-Muller). */
static inline void normal2(uint64_t r, double *n0, double *n1) {
    double u1 = u32_open((uint32_t)(r >> 32));
    double u2 = u32_open((uint32_t)(r & 0xFFFFFFFFu));
    double rad = sqrt(-2.0 * log(u1));
    *n0 = rad * cos(2.0 * M_PI * u2);
    *n1 = rad * sin(2.0 * M_PI * u2);
}

enum { ST_SITE = 1, ST_COLOUR = 2, ST_VEL = 3, ST_GRAD = 4, ST_DRIFT = 5, ST_NOISE = 6 };

typedef struct {
    int width, height, channels; /* channels 3 (RGB) or 4 (RGBA, alpha = 255) */
    int regions;                 /* number of Voronoi sites, >= 1 */
    double noise_sigma;          /* per-channel Gaussian noise, grey levels */
    double grad_max;             /* per-channel gradient amplitude ~ U[0, grad_max] */
    double vmax;                 /* per-region speed ~ U[0, vmax] px/frame */
    double drift_sigma;          /* per-region colour random-walk step, grey levels */
    uint64_t seed;
} synth_spec;

static uint8_t round_clip(double v) {
    if (v < 0.0) v = 0.0;
    if (v > 255.0) v = 255.0;
    return (uint8_t)nearbyint(v); /* default rounding mode: half to even */
}

/*
 * Render frame `t` (t = 0 is the still image) into out[H][W][channels].
 * Returns 0 on success, -1 on invalid arguments, -2 on allocation failure.
 */
int synth_frame(const synth_spec *sp, int t, uint8_t *out) {
    if (!sp || !out || sp->width <= 0 || sp->height <= 0 || sp->regions <= 0 ||
        (sp->channels != 3 && sp->channels != 4) || t < 0)
        return -1;
    const int W = sp->width, H = sp->height, R = sp->regions, C = sp->channels;
    double *sx = (double *)malloc(sizeof(double) * R * 5);
    if (!sx) return -2;
    double *sy = sx + R, *col = sx + 2 * R; /* col: R x 3 */

    /* Sites, velocities and colours at frame t. */
    for (int i = 0; i < R; ++i) {
        double x0 = u53(key3(sp->seed, ST_SITE, 2 * (uint64_t)i)) * W;
        double y0 = u53(key3(sp->seed, ST_SITE, 2 * (uint64_t)i + 1)) * H;
        double speed = u53(key3(sp->seed, ST_VEL, 2 * (uint64_t)i)) * sp->vmax;
        double ang = u53(key3(sp->seed, ST_VEL, 2 * (uint64_t)i + 1)) * 2.0 * M_PI;
        sx[i] = x0 + t * speed * cos(ang);
        sy[i] = y0 + t * speed * sin(ang);
        for (int c = 0; c < 3; ++c) {
            double v = u53(key3(sp->seed, ST_COLOUR, 3 * (uint64_t)i + c)) * 255.0;
            for (int s = 1; s <= t && sp->drift_sigma > 0.0; ++s) {
                double n0, n1;
                normal2(key3(sp->seed, ST_DRIFT, ((uint64_t)s * R + i) * 3 + c), &n0, &n1);
                v += sp->drift_sigma * n0;
            }
            col[3 * i + c] = v;
        }
    }

    /* One global linear gradient: direction theta, per-channel amplitude;
       g(x,y) runs from -1/2 to +1/2 across the image along theta. */
    double theta = u53(key3(sp->seed, ST_GRAD, 0)) * 2.0 * M_PI;
    double amp[3];
    for (int c = 0; c < 3; ++c) amp[c] = u53(key3(sp->seed, ST_GRAD, 1 + c)) * sp->grad_max;
    double ct = cos(theta), st = sin(theta);
    double extent = fabs((W - 1) * ct) + fabs((H - 1) * st);
    if (extent <= 0.0) extent = 1.0;

    /* Bucket grid over the image for an exact nearest-site search. */
    double B = sqrt((double)W * H / R);
    if (B < 1.0) B = 1.0;
    int gx = (int)ceil(W / B), gy = (int)ceil(H / B);
    if (gx < 1) gx = 1;
    if (gy < 1) gy = 1;
    int *head = (int *)malloc(sizeof(int) * ((size_t)gx * gy + R));
    if (!head) { free(sx); return -2; }
    int *next = head + (size_t)gx * gy;
    for (int b = 0; b < gx * gy; ++b) head[b] = -1;
    /* Insert in descending index order so each bucket lists ascending indices. */
    for (int i = R - 1; i >= 0; --i) {
        int bx = (int)floor(sx[i] / B), by = (int)floor(sy[i] / B);
        bx = bx < 0 ? 0 : (bx >= gx ? gx - 1 : bx);
        by = by < 0 ? 0 : (by >= gy ? gy - 1 : by);
        next[i] = head[by * gx + bx];
        head[by * gx + bx] = i;
    }
    int maxring = gx > gy ? gx : gy;

#pragma omp parallel for schedule(dynamic, 8)
    for (int y = 0; y < H; ++y) {
        int pby = (int)floor(y / B);
        if (pby >= gy) pby = gy - 1;
        for (int x = 0; x < W; ++x) {
            int pbx = (int)floor(x / B);
            if (pbx >= gx) pbx = gx - 1;
            double best = INFINITY;
            int bi = -1;
            for (int r = 0; r <= maxring; ++r) {
                /* Sites clamped into border buckets may lie outside them, so
                   the ring bound uses (r-1) buckets of guaranteed separation. */
                double lb = (r - 1) * B;
                if (bi >= 0 && lb > 0.0 && best < lb * lb) break;
                for (int by = pby - r; by <= pby + r; ++by) {
                    if (by < 0 || by >= gy) continue;
                    for (int bx = pbx - r; bx <= pbx + r; ++bx) {
                        if (bx < 0 || bx >= gx) continue;
                        if (by != pby - r && by != pby + r && bx != pbx - r && bx != pbx + r) continue;
                        for (int i = head[by * gx + bx]; i >= 0; i = next[i]) {
                            double dx = x - sx[i], dy = y - sy[i];
                            double d = dx * dx + dy * dy;
                            if (d < best || (d == best && i < bi)) { best = d; bi = i; }
                        }
                    }
                }
            }
            double g = ((x - 0.5 * (W - 1)) * ct + (y - 0.5 * (H - 1)) * st) / extent;
            uint64_t pix = ((uint64_t)t * H + y) * (uint64_t)W + x;
            double n[4];
            normal2(key3(sp->seed, ST_NOISE, 2 * pix), &n[0], &n[1]);
            normal2(key3(sp->seed, ST_NOISE, 2 * pix + 1), &n[2], &n[3]);
            uint8_t *o = out + ((size_t)y * W + x) * C;
            for (int c = 0; c < 3; ++c)
                o[c] = round_clip(col[3 * bi + c] + amp[c] * g + sp->noise_sigma * n[c]);
            if (C == 4) o[3] = 255;
        }
    }
    free(head);
    free(sx);
    return 0;
}
