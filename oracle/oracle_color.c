/*
 * FP64 oracle: histogram equalisation of the frames in HSV (Sec. 4.2, the
 * paper's illumination experiment: equalise the image pair in HSV and run the
 * unchanged method on the result).  Test infrastructure, never the product.
 *
 * Reading (the paper gives no detail): each frame separately; the V channel
 * (V = max(R, G, B), Smith's hexcone model) is equalised over 256 bins of
 * [0, 1], bin = min(255, floor(256 V)); a pixel in bin b gets
 * V' = (cdf(b) - cdf_min) / (n - cdf_min), where cdf_min is the count of the
 * lowest occupied bin; H and S are kept.  A frame whose pixels all share one
 * bin is left unchanged.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* Smith's hexcone RGB -> HSV, h in [0, 1), everything in [0, 1] for inputs in [0, 1]. */
void orc_rgb_to_hsv(double r, double g, double b, double* h, double* s, double* v) {
    double mx = r, mn = r;
    if (g > mx) mx = g;
    if (b > mx) mx = b;
    if (g < mn) mn = g;
    if (b < mn) mn = b;
    *v = mx;
    if (mx == mn) {
        *h = 0.0;
        *s = 0.0;
        return;
    }
    const double c = mx - mn;
    *s = c / mx;
    double hh;
    if (mx == r)
        hh = (g - b) / c;          /* between yellow and magenta */
    else if (mx == g)
        hh = 2.0 + (b - r) / c;    /* between cyan and yellow */
    else
        hh = 4.0 + (r - g) / c;    /* between magenta and cyan */
    hh /= 6.0;
    if (hh < 0) hh += 1.0;
    *h = hh;
}

/* The inverse: sector i = floor(6 h), fraction f, and the three levels
   v (1 - s), v (1 - s f), v (1 - s (1 - f)). */
void orc_hsv_to_rgb(double h, double s, double v, double* r, double* g, double* b) {
    if (s == 0.0) {
        *r = *g = *b = v;
        return;
    }
    const double h6 = h * 6.0;
    int i = (int)floor(h6);
    const double f = h6 - i;
    const double p = v * (1.0 - s), q = v * (1.0 - s * f), t = v * (1.0 - s * (1.0 - f));
    i %= 6;
    if (i < 0) i += 6;
    switch (i) {
        case 0: *r = v; *g = t; *b = p; break;
        case 1: *r = q; *g = v; *b = p; break;
        case 2: *r = p; *g = v; *b = t; break;
        case 3: *r = p; *g = q; *b = v; break;
        case 4: *r = t; *g = p; *b = v; break;
        default: *r = v; *g = p; *b = q; break;
    }
}

static int v_bin(double v) {
    double x = floor(256.0 * v);
    if (!(x >= 0)) x = 0;
    if (x > 255) x = 255;
    return (int)x;
}

/* Equalised V of each bin (lut[256]); returns 0 when the frame is left unchanged. */
int orc_v_lut(const orc_params* P, const double* rgb, double* lut) {
    const int n = P->W * P->H;
    long long cnt[256];
    memset(cnt, 0, sizeof cnt);
    for (int i = 0; i < n; ++i) {
        double h, s, v;
        orc_rgb_to_hsv(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], &h, &s, &v);
        cnt[v_bin(v)]++;
    }
    long long cdf = 0, cmin = -1;
    for (int b = 0; b < 256; ++b) {
        cdf += cnt[b];
        if (cmin < 0 && cnt[b] > 0) cmin = cnt[b];
        lut[b] = (double)cdf; /* cumulative count, mapped below */
    }
    if (cmin < 0 || cmin == n) return 0;
    for (int b = 0; b < 256; ++b) lut[b] = (lut[b] - (double)cmin) / (double)(n - cmin);
    return 1;
}

void orc_hsv_equalize(const orc_params* P, const double* in, double* out) {
    const int n = P->W * P->H;
    double lut[256];
    if (!orc_v_lut(P, in, lut)) {
        memcpy(out, in, sizeof(double) * 3 * (size_t)n);
        return;
    }
    for (int i = 0; i < n; ++i) {
        double h, s, v;
        orc_rgb_to_hsv(in[3 * i], in[3 * i + 1], in[3 * i + 2], &h, &s, &v);
        orc_hsv_to_rgb(h, s, lut[v_bin(v)], &out[3 * i], &out[3 * i + 1], &out[3 * i + 2]);
    }
}

/*
 * Census transform data term (Sec. 6 names census as an illumination-robust
 * data term for the framework).  Reading: grey = R + G + B (FP64); the code
 * of a pixel has one bit per neighbour of its 5x5 window in raster order
 * without the centre (24 bits, neighbour coordinates clamped into the frame),
 * set iff the neighbour's grey is strictly below the centre's.  Codes come
 * from the frames as given: census is unchanged by a global gain.  Written as
 * a "code frame" (code, 0, 0 per pixel) that the PatchMatch routines read
 * when P->census is set: the patch cost is then the sum over taps of the
 * Hamming distance of the two codes, over 24 T.
 */
#define ORC_CENSUS_R 2
#define ORC_CENSUS_BITS 24

static double grey(const double* rgb, int W, int x, int y) {
    const double* p = rgb + ((size_t)y * W + x) * 3;
    return (p[0] + p[1]) + p[2];
}

void orc_census(const orc_params* P, const double* rgb, double* codes) {
    const int W = P->W, H = P->H;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double c = grey(rgb, W, x, y);
            uint32_t code = 0;
            int bit = 0;
            for (int dy = -ORC_CENSUS_R; dy <= ORC_CENSUS_R; ++dy)
                for (int dx = -ORC_CENSUS_R; dx <= ORC_CENSUS_R; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    int nx = x + dx, ny = y + dy;
                    nx = nx < 0 ? 0 : (nx > W - 1 ? W - 1 : nx);
                    ny = ny < 0 ? 0 : (ny > H - 1 ? H - 1 : ny);
                    if (grey(rgb, W, nx, ny) < c) code |= 1u << bit;
                    ++bit;
                }
            double* o = codes + ((size_t)y * W + x) * 3;
            o[0] = (double)code;
            o[1] = 0.0;
            o[2] = 0.0;
        }
}

int orc_popcount32(uint32_t v) {
    int n = 0;
    while (v) {
        v &= v - 1;
        ++n;
    }
    return n;
}

/*
 * Edge-aware fill of the pixels left without a plane (stands in for the
 * EpicFlow interpolation the paper applies after MSGPM, Sec. 3.4.1 / 4).
 * Reading: each such pixel takes the plane of the assigned pixel nearest to
 * it in geodesic distance, where a step between 4-neighbours costs
 * 256 + |q_i - q_j| with q = floor(1024 (R + G + B)) of the frame as given
 * (FP64).  Distances are integers, computed by fast sweeping: ORC_INTERP_ROUNDS
 * rounds of four in-place scans (rows left to right, rows right to left,
 * columns top to bottom, columns bottom to top); a neighbour's offer replaces
 * the current one if its distance is lower, or equal with a lower seed index.
 */
#define ORC_INTERP_ROUNDS 4

void orc_grey_q(const orc_params* P, const double* rgb, int32_t* q) {
    const int n = P->W * P->H;
    for (int i = 0; i < n; ++i) q[i] = (int32_t)floor(1024.0 * ((rgb[3 * i] + rgb[3 * i + 1]) + rgb[3 * i + 2]));
}

static void relax(const int32_t* q, long long* dist, int32_t* seed, int j, int i) {
    if (seed[j] < 0) return;
    const long long c = dist[j] + 256 + llabs((long long)q[i] - q[j]);
    if (c < dist[i] || (c == dist[i] && seed[j] < seed[i])) {
        dist[i] = c;
        seed[i] = seed[j];
    }
}

void orc_interp_seeds(const orc_params* P, const int32_t* q, const int32_t* am, int32_t* seed) {
    const int W = P->W, H = P->H, n = W * H;
    long long* dist = (long long*)malloc(sizeof(long long) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        dist[i] = am[i] >= 0 ? 0 : (long long)1 << 62;
        seed[i] = am[i] >= 0 ? i : -1;
    }
    for (int r = 0; r < ORC_INTERP_ROUNDS; ++r) {
        for (int y = 0; y < H; ++y)
            for (int x = 1; x < W; ++x) relax(q, dist, seed, y * W + x - 1, y * W + x);
        for (int y = 0; y < H; ++y)
            for (int x = W - 2; x >= 0; --x) relax(q, dist, seed, y * W + x + 1, y * W + x);
        for (int x = 0; x < W; ++x)
            for (int y = 1; y < H; ++y) relax(q, dist, seed, (y - 1) * W + x, y * W + x);
        for (int x = 0; x < W; ++x)
            for (int y = H - 2; y >= 0; --y) relax(q, dist, seed, (y + 1) * W + x, y * W + x);
    }
    free(dist);
}
