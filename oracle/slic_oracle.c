/*
 * FP64 CPU oracle for SLIC superpixels as gSLICr (Ren, Prisacariu and Reid,
 * "gSLICr: SLIC superpixels at over 250Hz", arXiv 1509.04232) defines it.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this code:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * and reference legs use it. It shares no code, header, table or constant
 * generator with the CUDA implementation.
 *
 * Every step is written as plainly as possible, in the paper's order and
 * notation, in double precision, with no blocking, fusion or reordering:
 *   grid            Sec. 2 (S = sqrt(N/K))                  oracle_grid
 *   colour convert  Sec. 2 (CIELAB), Sec. 3 "Image space conversion"
 *                                                           oracle_convert
 *   init            Sec. 3 "Cluster center initialisation"  oracle_init_centres
 *   seed perturbation  Sec. 2 (original SLIC's first step)  oracle_perturb_seeds
 *   stopping test   Sec. 2 (L1 change of the centres)       oracle_residual
 *   assign          Eq. (1), Sec. 3 "Finding the cluster associations"
 *                                                           oracle_assign
 *   update          Sec. 3 "Updating the cluster center"    oracle_update
 *   connectivity    Sec. 3 "Enforce connectivity"           oracle_connectivity_pass
 *   connectivity, original SLIC's components (Sec. 2)      oracle_connectivity_components
 *   driver          Sec. 4 Perform_Segmentation order       oracle_slic
 *
 * Readings where the paper is silent or garbled (each one is listed in the
 * design notes with its reason):
 *   - S is an integer; when K is given, S = max(1, round(sqrt(N/K))).
 *   - The grid has ns_c = ceil(W/S) columns and ns_r = ceil(H/S) rows; the
 *     last column/row may be a partial cell. Label k = r*ns_c + c.
 *   - sRGB (IEC 61966-2-1) gamma, the sRGB D65 matrix, white point = the
 *     matrix row sums, CIE 1976 L*a*b* with eps = 216/24389, kappa = 24389/27.
 *   - Pixel coordinates are integer indices (x, y).
 *   - Initial centre: midpoint of the in-image part of its cell, colour of
 *     the pixel at (floor(x_k), floor(y_k)); no gradient perturbation
 *     (the paper's GPU listing has none).
 *   - Eq. (1)'s "n_k" is read as b_k; D_s = d_lab + (m/S) d_xy literally.
 *   - Assignment ties go to the first candidate in scan order (dy outer,
 *     dx inner, each -1..1).
 *   - An empty cluster keeps its previous centre and gets count 0.
 *   - "iterations" counts centre updates; each is followed by an assignment.
 *   - Connectivity: two double-buffered passes; a pixel whose every in-image
 *     4-neighbour has a different label adopts the most frequent neighbour
 *     label, ties to the earliest in the order left, up, right, down.
 *     Centres are not recomputed afterwards.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_CIELAB 0
#define ORACLE_RGB 1
#define ORACLE_XYZ 2

/* Sec. 2: "there would be a superpixel center at every grid interval
   S = sqrt(N/K)". Returns 0, or -1 on invalid arguments. */
int oracle_grid(int W, int H, int K, int S_in, int *S, int *ns_c, int *ns_r) {
    if (W <= 0 || H <= 0) return -1;
    int s;
    if (S_in > 0) {
        s = S_in;
    } else {
        if (K <= 0) return -1;
        s = (int)lround(sqrt((double)W * (double)H / (double)K));
        if (s < 1) s = 1;
    }
    *S = s;
    *ns_c = (W + s - 1) / s;
    *ns_r = (H + s - 1) / s;
    return 0;
}

/* sRGB electro-optical transfer function (IEC 61966-2-1), v in [0,1]. */
static double srgb_to_linear(double v) {
    if (v <= 0.04045) return v / 12.92;
    return pow((v + 0.055) / 1.055, 2.4);
}

/* CIE 1976 companding function f(t). */
static double lab_f(double t) {
    const double eps = 216.0 / 24389.0;
    const double kappa = 24389.0 / 27.0;
    if (t > eps) return cbrt(t);
    return (kappa * t + 16.0) / 116.0;
}

/* Linear sRGB -> XYZ (D65), rows of the sRGB matrix. */
static const double M_RGB_XYZ[3][3] = {
    {0.4124564, 0.3575761, 0.1804375},
    {0.2126729, 0.7151522, 0.0721750},
    {0.0193339, 0.1191920, 0.9503041},
};

/* Sec. 3 "Image space conversion": one pixel, R,G,B bytes -> 3 features.
   CIELAB: L in [0,100], a, b. RGB: raw bytes. XYZ: X, Y, Z times 100. */
static void convert_pixel(const uint8_t *p, int color_space, double out[3]) {
    if (color_space == ORACLE_RGB) {
        out[0] = p[0];
        out[1] = p[1];
        out[2] = p[2];
        return;
    }
    double lin[3];
    for (int c = 0; c < 3; ++c) lin[c] = srgb_to_linear(p[c] / 255.0);
    double xyz[3];
    for (int r = 0; r < 3; ++r)
        xyz[r] = M_RGB_XYZ[r][0] * lin[0] + M_RGB_XYZ[r][1] * lin[1] + M_RGB_XYZ[r][2] * lin[2];
    if (color_space == ORACLE_XYZ) {
        for (int r = 0; r < 3; ++r) out[r] = 100.0 * xyz[r];
        return;
    }
    /* White point: the XYZ of linear (1,1,1), i.e. the row sums. */
    double white[3];
    for (int r = 0; r < 3; ++r) white[r] = M_RGB_XYZ[r][0] + M_RGB_XYZ[r][1] + M_RGB_XYZ[r][2];
    double fx = lab_f(xyz[0] / white[0]);
    double fy = lab_f(xyz[1] / white[1]);
    double fz = lab_f(xyz[2] / white[2]);
    out[0] = 116.0 * fy - 16.0;
    out[1] = 500.0 * (fx - fy);
    out[2] = 200.0 * (fy - fz);
}

/* Whole image: rgb[H][W][C] (C = 3 or 4, alpha ignored) -> feat[H*W][3]. */
int oracle_convert(const uint8_t *rgb, int W, int H, int C, int color_space, double *feat) {
    if (W <= 0 || H <= 0 || (C != 3 && C != 4) || color_space < 0 || color_space > 2) return -1;
    for (long i = 0; i < (long)W * H; ++i) convert_pixel(rgb + i * C, color_space, feat + 3 * i);
    return 0;
}

/* Sec. 3 "Cluster center initialisation": one centre per grid cell, stored
   in an ns_r x ns_c map; centre = (l, a, b, x, y, count). */
int oracle_init_centres(const double *feat, int W, int H, int S, double *centres) {
    int ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
    for (int r = 0; r < ns_r; ++r) {
        for (int c = 0; c < ns_c; ++c) {
            int x_first = c * S, x_last = ((c + 1) * S < W ? (c + 1) * S : W) - 1;
            int y_first = r * S, y_last = ((r + 1) * S < H ? (r + 1) * S : H) - 1;
            double xk = (x_first + x_last) / 2.0;
            double yk = (y_first + y_last) / 2.0;
            long pix = (long)floor(yk) * W + (long)floor(xk);
            double *ck = centres + 6 * ((long)r * ns_c + c);
            ck[0] = feat[3 * pix + 0];
            ck[1] = feat[3 * pix + 1];
            ck[2] = feat[3 * pix + 2];
            ck[3] = xk;
            ck[4] = yk;
            ck[5] = 0.0;
        }
    }
    return 0;
}

/* Sec. 2, first step of the original SLIC: "the cluster centers are
   perturbed to the lowest gradient position from a local neighborhood".
   Readings (the paper names neither the gradient nor the neighbourhood):
   the neighbourhood is the 3x3 pixels around the seed pixel
   (floor(x_k), floor(y_k)); the gradient is the squared central
   differences of the features, G(x,y) = |I(x+1,y) - I(x-1,y)|^2 +
   |I(x,y+1) - I(x,y-1)|^2, with coordinates clamped into the image. The
   seed pixel is the first candidate and a later one (dy outer, dx inner,
   each -1..1, in-image only) replaces the best only when its G is strictly
   lower; a seed that moves takes that pixel's features and integer
   coordinates, one that stays keeps its initial centre. */
static double gradient_G(const double *feat, int W, int H, int x, int y) {
    int xl = x > 0 ? x - 1 : 0, xr = x < W - 1 ? x + 1 : W - 1;
    int yu = y > 0 ? y - 1 : 0, yd = y < H - 1 ? y + 1 : H - 1;
    double g = 0.0;
    for (int c = 0; c < 3; ++c) {
        double gx = feat[3 * ((long)y * W + xr) + c] - feat[3 * ((long)y * W + xl) + c];
        double gy = feat[3 * ((long)yd * W + x) + c] - feat[3 * ((long)yu * W + x) + c];
        g += gx * gx + gy * gy;
    }
    return g;
}

/* Applies the perturbation to grid-initialised centres in place.
   g_best [K_eff] (optional): G at the chosen pixel; margin [K_eff]
   (optional): (smallest G among the other candidates - g_best) /
   max(g_best, 1e-12), +inf with a single candidate. */
int oracle_perturb_seeds(const double *feat, int W, int H, int S, double *centres, double *g_best,
                         double *margin) {
    if (W <= 0 || H <= 0 || S <= 0) return -1;
    int ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
    for (int k = 0; k < ns_c * ns_r; ++k) {
        double *ck = centres + 6 * (long)k;
        int px = (int)floor(ck[3]), py = (int)floor(ck[4]);
        int bx = px, by = py;
        const double g0 = gradient_G(feat, W, H, px, py);
        double best = g0;
        double gv[9];
        int gx[9], gy[9], n = 0;
        for (int dy = -1; dy <= 1; ++dy) {
            for (int dx = -1; dx <= 1; ++dx) {
                int x = px + dx, y = py + dy;
                if (x < 0 || x >= W || y < 0 || y >= H) continue;
                double g = (dx == 0 && dy == 0) ? g0 : gradient_G(feat, W, H, x, y);
                gv[n] = g;
                gx[n] = x;
                gy[n] = y;
                ++n;
                if (!(dx == 0 && dy == 0) && g < best) {
                    best = g;
                    bx = x;
                    by = y;
                }
            }
        }
        if (g_best) g_best[k] = best;
        if (margin) {
            double second = INFINITY;
            for (int i = 0; i < n; ++i)
                if (!(gx[i] == bx && gy[i] == by) && gv[i] < second) second = gv[i];
            margin[k] = isinf(second) ? INFINITY : (second - best) / (best > 1e-12 ? best : 1e-12);
        }
        if (bx != px || by != py) {
            const double *f = feat + 3 * ((long)by * W + bx);
            ck[0] = f[0];
            ck[1] = f[1];
            ck[2] = f[2];
            ck[3] = bx;
            ck[4] = by;
        }
    }
    return 0;
}

/* Sec. 2: the iteration stops "when the cluster centers stabilise", the
   L1 distance between centres of consecutive iterations falling below a
   threshold. Reading: E = (1/K_eff) sum_k (|x_k - x'_k| + |y_k - y'_k|),
   the mean L1 move of the centre positions over one update. */
double oracle_residual(const double *prev, const double *cur, int K_eff) {
    double e = 0.0;
    for (int k = 0; k < K_eff; ++k) e += fabs(cur[6 * k + 3] - prev[6 * k + 3]) + fabs(cur[6 * k + 4] - prev[6 * k + 4]);
    return K_eff > 0 ? e / K_eff : 0.0;
}

/* Eq. (1): D_s = d_lab + (m/S) d_xy for pixel i against centre k. */
static double distance_Ds(const double *fi, double xi, double yi, const double *ck, double m, int S) {
    double dl = ck[0] - fi[0], da = ck[1] - fi[1], db = ck[2] - fi[2];
    double d_lab = sqrt(dl * dl + da * da + db * db);
    double dx = ck[3] - xi, dy = ck[4] - yi;
    double d_xy = sqrt(dx * dx + dy * dy);
    return d_lab + (m / S) * d_xy;
}

/* Sec. 3 "Finding the cluster associations": each pixel examines at most
   nine centres, those of its own grid cell and the 8 around it, and takes
   the one with the smallest D_s (first in scan order on exact ties).
   margin (optional) = (second best - best) / max(best, 1e-12), +inf when
   there is a single candidate. */
int oracle_assign(const double *feat, int W, int H, int S, double m, const double *centres,
                  int32_t *labels, double *margin) {
    int ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            int cx = x / S, cy = y / S;
            double best = INFINITY, second = INFINITY;
            int best_k = -1;
            for (int dy = -1; dy <= 1; ++dy) {
                for (int dx = -1; dx <= 1; ++dx) {
                    int nx = cx + dx, ny = cy + dy;
                    if (nx < 0 || nx >= ns_c || ny < 0 || ny >= ns_r) continue;
                    int k = ny * ns_c + nx;
                    double D = distance_Ds(feat + 3 * i, x, y, centres + 6 * k, m, S);
                    if (D < best) {
                        second = best;
                        best = D;
                        best_k = k;
                    } else if (D < second) {
                        second = D;
                    }
                }
            }
            labels[i] = best_k;
            if (margin) {
                double denom = best > 1e-12 ? best : 1e-12;
                margin[i] = isinf(second) ? INFINITY : (second - best) / denom;
            }
        }
    }
    return 0;
}

/* Sec. 3 "Updating the cluster center": each centre becomes the mean labxy
   of the pixels assigned to it; a centre with no pixels keeps its previous
   value and gets count 0. */
int oracle_update(const double *feat, int W, int H, const int32_t *labels, int K_eff, double *centres) {
    double *sum = (double *)calloc((size_t)K_eff * 6, sizeof(double));
    if (!sum) return -2;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            int k = labels[i];
            if (k < 0 || k >= K_eff) { free(sum); return -1; }
            sum[6 * k + 0] += feat[3 * i + 0];
            sum[6 * k + 1] += feat[3 * i + 1];
            sum[6 * k + 2] += feat[3 * i + 2];
            sum[6 * k + 3] += x;
            sum[6 * k + 4] += y;
            sum[6 * k + 5] += 1.0;
        }
    }
    for (int k = 0; k < K_eff; ++k) {
        double n = sum[6 * k + 5];
        if (n > 0.0) {
            for (int j = 0; j < 5; ++j) centres[6 * k + j] = sum[6 * k + j] / n;
            centres[6 * k + 5] = n;
        } else {
            centres[6 * k + 5] = 0.0;
        }
    }
    free(sum);
    return 0;
}

/* Sec. 3 "Enforce connectivity", one pass: reads `in`, writes `out`. A
   pixel whose every in-image 4-neighbour carries a different label takes
   the most frequent neighbour label (ties: earliest of left, up, right,
   down); otherwise it keeps its label. */
int oracle_connectivity_pass(const int32_t *in, int W, int H, int32_t *out) {
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            int32_t own = in[i];
            int32_t nb[4];
            int n = 0;
            if (x > 0) nb[n++] = in[i - 1];
            if (y > 0) nb[n++] = in[i - W];
            if (x < W - 1) nb[n++] = in[i + 1];
            if (y < H - 1) nb[n++] = in[i + W];
            int all_differ = (n > 0);
            for (int j = 0; j < n; ++j)
                if (nb[j] == own) all_differ = 0;
            if (!all_differ) {
                out[i] = own;
                continue;
            }
            int best_j = 0, best_count = 0;
            for (int j = 0; j < n; ++j) {
                int count = 0;
                for (int q = 0; q < n; ++q)
                    if (nb[q] == nb[j]) ++count;
                if (count > best_count) {
                    best_count = count;
                    best_j = j;
                }
            }
            out[i] = nb[best_j];
        }
    }
    return 0;
}

/* Component-based connectivity, the original SLIC's notion of "connectivity
 * is enforced" (Sec. 2), offered as an alternative to the paper's local rule.
 * Readings: a segment is a 4-connected set of pixels with equal labels;
 * segments are visited in scan order of their first pixel; one of at most
 * min_size pixels (the caller passes S*S/4) is merged into the segment of
 * its first pixel's left neighbour, or of its upper neighbour in column 0,
 * taking that segment's final label; the segment of pixel (0, 0) is always
 * kept; kept segments are numbered 0, 1, ... in the order visited.
 * out[H*W] receives the new labels. Returns the number of segments kept,
 * -1 on invalid arguments, -2 on allocation failure. */
int oracle_connectivity_components(const int32_t *in, int W, int H, int min_size, int32_t *out) {
    if (W <= 0 || H <= 0 || min_size < 0) return -1;
    long N = (long)W * H;
    long *queue = (long *)malloc(sizeof(long) * N);
    if (!queue) return -2;
    for (long i = 0; i < N; ++i) out[i] = -1;
    int kept = 0;
    for (long start = 0; start < N; ++start) {
        if (out[start] >= 0) continue;
        /* breadth-first search of the segment, marking its pixels with a
           provisional label (kept) */
        long head = 0, tail = 0;
        queue[tail++] = start;
        out[start] = kept;
        while (head < tail) {
            long i = queue[head++];
            int x = (int)(i % W), y = (int)(i / W);
            long nb[4];
            int n = 0;
            if (x > 0) nb[n++] = i - 1;
            if (y > 0) nb[n++] = i - W;
            if (x < W - 1) nb[n++] = i + 1;
            if (y < H - 1) nb[n++] = i + W;
            for (int j = 0; j < n; ++j) {
                if (out[nb[j]] < 0 && in[nb[j]] == in[start]) {
                    out[nb[j]] = kept;
                    queue[tail++] = nb[j];
                }
            }
        }
        long size = tail;
        int sx = (int)(start % W);
        long adj = start == 0 ? -1 : (sx > 0 ? start - 1 : start - W);
        if (size <= min_size && adj >= 0) {
            /* merged: the neighbour's segment was visited earlier, so its
               final label is already written */
            for (long q = 0; q < size; ++q) out[queue[q]] = out[adj];
        } else {
            ++kept;
        }
    }
    free(queue);
    return kept;
}

/*
 * Sec. 4, Perform_Segmentation: convert; initialise centres (or take
 * init_centres when given, e.g. the previous video frame's), perturbed
 * when perturb_seeds is set (Sec. 2); assign; then up to `iterations` times
 * {update; assign}, ending after the first iteration whose update moved
 * the centres by E < convergence (Sec. 2; convergence 0: never); then, with
 * enforce_connectivity 1, two connectivity passes, or with 2 the
 * component-based relabelling (minimum size S*S/4).
 *   labels   [H*W]      final labels
 *   centres  [K_eff*6]  centres the final labels were assigned against
 *   labels_pre [H*W]    optional: labels before connectivity
 *   margin   [H*W]      optional: tie margin of the final assignment
 *   iterations_run      optional: updates performed
 * Returns 0, -1 on invalid arguments, -2 on allocation failure.
 */
int oracle_slic(const uint8_t *rgb, int W, int H, int C, int K, int S_in, double m, int iterations,
                int color_space, int enforce_connectivity, const double *init_centres, int perturb_seeds,
                double convergence, int32_t *labels, double *centres, int32_t *labels_pre, double *margin,
                int *iterations_run) {
    int S, ns_c, ns_r;
    if (oracle_grid(W, H, K, S_in, &S, &ns_c, &ns_r) != 0 || iterations < 0 || !(m >= 0.0) ||
        !(convergence >= 0.0))
        return -1;
    int K_eff = ns_c * ns_r;
    long N = (long)W * H;
    double *feat = (double *)malloc(sizeof(double) * 3 * N);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * N);
    double *prev = (double *)malloc(sizeof(double) * 6 * K_eff);
    if (!feat || !tmp || !prev) { free(feat); free(tmp); free(prev); return -2; }
    if (oracle_convert(rgb, W, H, C, color_space, feat) != 0) { free(feat); free(tmp); free(prev); return -1; }
    if (init_centres) {
        memcpy(centres, init_centres, sizeof(double) * 6 * K_eff);
    } else {
        oracle_init_centres(feat, W, H, S, centres);
        if (perturb_seeds) oracle_perturb_seeds(feat, W, H, S, centres, NULL, NULL);
    }
    oracle_assign(feat, W, H, S, m, centres, labels, margin);
    int done = 0;
    for (int it = 0; it < iterations; ++it) {
        memcpy(prev, centres, sizeof(double) * 6 * K_eff);
        oracle_update(feat, W, H, labels, K_eff, centres);
        oracle_assign(feat, W, H, S, m, centres, labels, margin);
        ++done;
        if (convergence > 0.0 && oracle_residual(prev, centres, K_eff) < convergence) break;
    }
    if (iterations_run) *iterations_run = done;
    free(prev);
    if (labels_pre) memcpy(labels_pre, labels, sizeof(int32_t) * N);
    if (enforce_connectivity == 1) {
        oracle_connectivity_pass(labels, W, H, tmp);
        oracle_connectivity_pass(tmp, W, H, labels);
    } else if (enforce_connectivity == 2) {
        memcpy(tmp, labels, sizeof(int32_t) * N);
        if (oracle_connectivity_components(tmp, W, H, S * S / 4, labels) < 0) {
            free(feat);
            free(tmp);
            return -2;
        }
    }
    free(feat);
    free(tmp);
    return 0;
}
