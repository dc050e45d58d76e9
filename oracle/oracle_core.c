/*
 * FP64 oracle, part 1: random numbers, window grid, warped patch cost and
 * PatchMatch.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the definition in Salmon, Moraes, Dror and    */
/* Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11: ten rounds of */
/* two 32x32->64 multiplications whose halves are xor-ed with the other two  */
/* counter words and the key; the key is bumped by the Weyl constants        */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Counter layout shared (as a specification, not as code) with the GPU:
   c0 = element (pixel or cell) index, c1 = sub-index, c2 = stream tag,
   c3 = pair id; key = the 64-bit seed split into two words. */
static uint32_t stream_tag(int purpose, int dir, int level, int stage) {
    return ((uint32_t)purpose << 24) | ((uint32_t)dir << 16) | ((uint32_t)level << 8) | (uint32_t)stage;
}

/* Uniform integer in [0, n) from a 32-bit random word: floor(u * n / 2^32). */
static inline uint32_t bounded_u32(uint32_t u, uint32_t n) { return (uint32_t)(((uint64_t)u * n) >> 32); }

static void rng4(const orc_params* P, uint32_t c0, uint32_t c1, uint32_t tag, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, tag, P->pair_id};
    uint32_t key[2] = {(uint32_t)(P->seed & 0xFFFFFFFFu), (uint32_t)(P->seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Window grid.  Sec. 3.1.2: each window overlaps the previous one by half.  */
/* Side s, stride s/2, starting at 0; one more window flush with the far     */
/* border when the regular ones stop short of it.                           */
/* ------------------------------------------------------------------------ */
int orc_grid_axis(int n, int s, int32_t* pos) {
    int h = s / 2, cnt = 0, last = -1;
    if (s <= 0 || n < s) return 0;
    for (int p = 0; p + s <= n; p += h) {
        if (pos) pos[cnt] = p;
        last = p;
        ++cnt;
    }
    if (last + s < n) {
        if (pos) pos[cnt] = n - s;
        ++cnt;
    }
    return cnt;
}

int orc_total_cells(const orc_params* P, int32_t* cell_base) {
    int total = 0;
    for (int l = 0; l < P->num_scales; ++l) {
        if (cell_base) cell_base[l] = total;
        total += orc_grid_axis(P->W, P->cell[l], NULL) * orc_grid_axis(P->H, P->cell[l], NULL);
    }
    if (cell_base) cell_base[P->num_scales] = total;
    return total;
}

/* ------------------------------------------------------------------------ */
/* Bilinear sample with the coordinates clamped to the frame (a continuous   */
/* function of (X, Y)).                                                     */
/* ------------------------------------------------------------------------ */
void orc_sample_bilinear(const double* img, int W, int H, double X, double Y, double out[3]) {
    if (X < 0.0) X = 0.0;
    if (X > W - 1) X = W - 1;
    if (Y < 0.0) Y = 0.0;
    if (Y > H - 1) Y = H - 1;
    int x0 = (int)floor(X), y0 = (int)floor(Y);
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
    int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    double fx = X - x0, fy = Y - y0;
    for (int c = 0; c < 3; ++c) {
        double a = img[((size_t)y0 * W + x0) * 3 + c], b = img[((size_t)y0 * W + x1) * 3 + c];
        double d = img[((size_t)y1 * W + x0) * 3 + c], e = img[((size_t)y1 * W + x1) * 3 + c];
        out[c] = (1.0 - fy) * ((1.0 - fx) * a + fx * b) + fy * ((1.0 - fx) * d + fx * e);
    }
}

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static inline void apply_h(const double* G, double x, double y, double* X, double* Y) {
    double w = G[6] * x + G[7] * y + G[8];
    *X = (G[0] * x + G[1] * y + G[2]) / w;
    *Y = (G[3] * x + G[4] * y + G[5]) / w;
}

/* ------------------------------------------------------------------------ */
/* Warped patch cost.  The colour-consistency error of eq. 3, averaged over  */
/* a (2r+1)^2 patch and the three channels.  Tap d of the patch of p reads   */
/* I1 at s = clamp(p + d) and the target frame at p + v + G(s) - G(p): the   */
/* square patch moved by the candidate offset v and distorted by the plane G */
/* (identity: the ordinary square patch of PatchMatch).                     */
/* ------------------------------------------------------------------------ */
/* Patch costs evaluated since the last reset (instrumentation for the timed
   CPU baseline; not part of the method). */
static long long orc_evals_;
long long orc_eval_count(int reset) {
    long long v;
#pragma omp atomic read
    v = orc_evals_;
    if (reset) {
#pragma omp atomic write
        orc_evals_ = 0;
    }
    return v;
}

double orc_patch_cost(const orc_params* P, const double* src, const double* tgt,
                      int px, int py, int vx, int vy, const double* G) {
    const int W = P->W, H = P->H, r = P->r;
#pragma omp atomic
    orc_evals_++;
    if (P->census && !G) { /* census code frames: Hamming distance per tap (Sec. 6) */
        long long sum = 0;
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                int sx = clampi(px + dx, 0, W - 1), sy = clampi(py + dy, 0, H - 1);
                int tx = clampi(sx + vx, 0, W - 1), ty = clampi(sy + vy, 0, H - 1);
                uint32_t a = (uint32_t)src[((size_t)sy * W + sx) * 3], b = (uint32_t)tgt[((size_t)ty * W + tx) * 3];
                sum += orc_popcount32(a ^ b);
            }
        return (double)sum / (24.0 * (2 * r + 1) * (2 * r + 1));
    }
    double gpx = 0, gpy = 0, sum = 0.0, s[3];
    if (G) apply_h(G, px, py, &gpx, &gpy);
    for (int dy = -r; dy <= r; ++dy) {
        for (int dx = -r; dx <= r; ++dx) {
            int sx = clampi(px + dx, 0, W - 1), sy = clampi(py + dy, 0, H - 1);
            double X, Y;
            if (G) {
                double gx, gy;
                apply_h(G, sx, sy, &gx, &gy);
                X = px + vx + (gx - gpx);
                Y = py + vy + (gy - gpy);
            } else {
                X = sx + vx;
                Y = sy + vy;
            }
            orc_sample_bilinear(tgt, W, H, X, Y, s);
            const double* a = src + ((size_t)sy * W + sx) * 3;
            sum += fabs(a[0] - s[0]) + fabs(a[1] - s[1]) + fabs(a[2] - s[2]);
        }
    }
    return sum / (3.0 * (2 * r + 1) * (2 * r + 1));
}

/* ------------------------------------------------------------------------ */
/* PatchMatch.  Sec. 3.1: the baseline NNF comes from PatchMatch (Barnes et  */
/* al. 2009) with 7x7 patches (Sec. 4).  The schedule is red-black: pixels   */
/* with (x+y) even update first from the state before the half-step, then   */
/* the odd ones.  Per pixel: incumbent, the four neighbours' offsets, the    */
/* plane candidates (levels >= 1), then random search around the best offset */
/* found so far; a candidate replaces the best only if strictly cheaper.     */
/* Sec. 3.3.2: at levels >= 1 only pixels without an assigned plane update;  */
/* assigned ones still lend their offsets as candidates.                    */
/* ------------------------------------------------------------------------ */
void orc_pm_init(const orc_params* P, const double* src, const double* tgt, int dir,
                 int32_t* vx, int32_t* vy, double* cost) {
    const int W = P->W, H = P->H;
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            uint32_t w[4];
            int i = y * W + x;
            rng4(P, (uint32_t)i, 0u, stream_tag(1, dir, 0, 0), w);
            int tx = (int)(w[0] % (uint32_t)W), ty = (int)(w[1] % (uint32_t)H);
            vx[i] = tx - x;
            vy[i] = ty - y;
            cost[i] = orc_patch_cost(P, src, tgt, x, y, vx[i], vy[i], NULL);
        }
    }
}

/* Window index ranges covering coordinate x on one axis. */
static int covering(const int32_t* pos, int n, int s, int x, int* idx) {
    int k = 0;
    for (int i = 0; i < n; ++i)
        if (pos[i] <= x && x < pos[i] + s) idx[k++] = i;
    return k;
}

/* Home window on one axis: the window whose central half holds x. */
static int home_index(int x, int s, int n) {
    int h = s / 2;
    int i = (int)floor((double)(x - s / 4) / h);
    return clampi(i, 0, n - 1);
}

typedef struct {
    int ncx, ncy, s, base;
    int32_t xs[4096], ys[4096];
} grid_t;

static void make_grid(const orc_params* P, int level, grid_t* g) {
    int32_t cb[ORC_MAX_SCALES + 1];
    orc_total_cells(P, cb);
    g->s = P->cell[level - 1];
    g->ncx = orc_grid_axis(P->W, g->s, g->xs);
    g->ncy = orc_grid_axis(P->H, g->s, g->ys);
    g->base = cb[level - 1];
}

/* Distortion plane of a pixel's patch at level >= 1: the home window's
   residual-stage model if valid, else its first-stage model if valid, else
   none (identity). */
static const double* home_plane(const grid_t* g, const double* mh, const int32_t* mi, int x, int y) {
    int cx = home_index(x, g->s, g->ncx), cy = home_index(y, g->s, g->ncy);
    int cell = cy * g->ncx + cx;
    int id2 = (g->base + cell) * 2 + 1, id1 = (g->base + cell) * 2;
    if (mi[id2 * ORC_MI + ORC_MI_VALID]) return mh + (size_t)id2 * 9;
    if (mi[id1 * ORC_MI + ORC_MI_VALID]) return mh + (size_t)id1 * 9;
    return NULL;
}

void orc_pm_recost(const orc_params* P, const double* src, const double* tgt, int level,
                   const double* mh, const int32_t* mi, const uint8_t* frozen,
                   const int32_t* vx, const int32_t* vy, double* cost) {
    const int W = P->W, H = P->H;
    grid_t* g = NULL;
    if (level >= 1) {
        g = (grid_t*)malloc(sizeof(grid_t));
        make_grid(P, level, g);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int i = y * W + x;
            if (level >= 1 && frozen && frozen[i]) continue;
            const double* G = g ? home_plane(g, mh, mi, x, y) : NULL;
            cost[i] = orc_patch_cost(P, src, tgt, x, y, vx[i], vy[i], G);
        }
    free(g);
}

static inline double rel_gap(double a, double b) {
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (m < 1e-7) m = 1e-7;
    return fabs(a - b) / m;
}

/* round(x) = floor(x + 0.5); logs how close x + 0.5 is to an integer */
static inline int round_logged(double x, double* gap) {
    double t = x + 0.5, f = floor(t);
    double d = fmin(t - f, f + 1.0 - t) / fmax(1.0, fabs(x));
    if (d < *gap) *gap = d;
    return (int)f;
}

void orc_pm_sweep(const orc_params* P, const double* src, const double* tgt, int dir, int level,
                  int it, int phase, const double* mh, const int32_t* mi, const uint8_t* frozen,
                  int32_t* vx, int32_t* vy, double* cost, double* amb) {
    const int W = P->W, H = P->H;
    grid_t* g = NULL;
    if (level >= 1) {
        g = (grid_t*)malloc(sizeof(grid_t));
        make_grid(P, level, g);
    }
    int R0 = W > H ? W : H, nrad = 0;
    while ((R0 >> nrad) >= 1) ++nrad;
    /* Pixels of the other colour are not written during this half-step, and
       all neighbours of a pixel have the other colour, so reading vx/vy in
       place is the same as reading the state before the half-step. */
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            if (((x + y) & 1) != phase) continue;
            int i = y * W + x;
            if (level >= 1 && frozen && frozen[i]) continue;
            const double* G = g ? home_plane(g, mh, mi, x, y) : NULL;
            int bx = vx[i], by = vy[i];
            double bc = cost[i], gap = 1e300;
#define TRY(cx_, cy_)                                                          \
    do {                                                                       \
        int cx__ = (cx_), cy__ = (cy_);                                        \
        if (!(cx__ == bx && cy__ == by)) {                                     \
            double c__ = orc_patch_cost(P, src, tgt, x, y, cx__, cy__, G);     \
            double g__ = rel_gap(c__, bc);                                     \
            if (g__ < gap) gap = g__;                                          \
            if (c__ < bc) {                                                    \
                bc = c__;                                                      \
                bx = cx__;                                                     \
                by = cy__;                                                     \
            }                                                                  \
        }                                                                      \
    } while (0)
            /* propagation: left, right, up, down */
            static const int NX[4] = {-1, 1, 0, 0}, NY[4] = {0, 0, -1, 1};
            for (int k = 0; k < 4; ++k) {
                int nx = x + NX[k], ny = y + NY[k];
                if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
                int j = ny * W + nx, cx = vx[j], cy = vy[j];
                int tx = x + cx, ty = y + cy;
                if (tx < 0 || tx >= W || ty < 0 || ty >= H) continue;
                TRY(cx, cy);
            }
            /* plane candidates: models of the windows covering p, in cell order */
            if (g) {
                int ix[8], iy[8];
                int nxw = covering(g->xs, g->ncx, g->s, x, ix), nyw = covering(g->ys, g->ncy, g->s, y, iy);
                for (int a = 0; a < nyw; ++a)
                    for (int b = 0; b < nxw; ++b) {
                        int cell = iy[a] * g->ncx + ix[b];
                        for (int st = 0; st < 2; ++st) {
                            int id = (g->base + cell) * 2 + st;
                            if (!mi[id * ORC_MI + ORC_MI_VALID]) continue;
                            const double* Hm = mh + (size_t)id * 9;
                            double w = Hm[6] * x + Hm[7] * y + Hm[8];
                            if (!(w > 0)) continue;
                            double X = (Hm[0] * x + Hm[1] * y + Hm[2]) / w;
                            double Y = (Hm[3] * x + Hm[4] * y + Hm[5]) / w;
                            int cx = round_logged(X - x, &gap), cy = round_logged(Y - y, &gap);
                            int tx = x + cx, ty = y + cy;
                            if (tx < 0 || tx >= W || ty < 0 || ty >= H) continue;
                            TRY(cx, cy);
                        }
                    }
            }
            /* random search around the best offset after propagation */
            int v0x = bx, v0y = by;
            for (int k = 0; k < nrad; ++k) {
                int R = R0 >> k;
                uint32_t w[4];
                rng4(P, (uint32_t)i, ((uint32_t)it << 8) | (uint32_t)(k >> 1), stream_tag(2, dir, level, 0), w);
                uint32_t ux = (k & 1) ? w[2] : w[0], uy = (k & 1) ? w[3] : w[1];
                int ox = (int)bounded_u32(ux, (uint32_t)(2 * R + 1)) - R;
                int oy = (int)bounded_u32(uy, (uint32_t)(2 * R + 1)) - R;
                int tx = clampi(x + v0x + ox, 0, W - 1), ty = clampi(y + v0y + oy, 0, H - 1);
                TRY(tx - x, ty - y);
            }
#undef TRY
            vx[i] = bx;
            vy[i] = by;
            cost[i] = bc;
            if (amb) amb[i] = gap;
        }
    }
    free(g);
}
