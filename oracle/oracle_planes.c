/*
 * FP64 oracle, part 2: homography solvers, robust plane fit per window,
 * plane assignment, occlusion cues, cross-level merge, fill and the final
 * occlusion map.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static inline double rel_gap(double a, double b) {
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (m < 1e-7) m = 1e-7;
    return fabs(a - b) / m;
}

/* a and b (colour errors, eq. 3, or values compared with one) are within the
   near-tie band: relative ORC_TIE_REL, at least ORC_L_ATOL absolute */
static inline int near_colour(double a, double b) {
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    return fabs(a - b) < fmax(ORC_TIE_REL * m, ORC_L_ATOL);
}

static void rng4(const orc_params* P, uint32_t c0, uint32_t c1, uint32_t tag, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, tag, P->pair_id};
    uint32_t key[2] = {(uint32_t)(P->seed & 0xFFFFFFFFu), (uint32_t)(P->seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform integer in [0, n) from a 32-bit random word: floor(u * n / 2^32). */
static inline uint32_t bounded_u32(uint32_t u, uint32_t n) { return (uint32_t)(((uint64_t)u * n) >> 32); }

static uint32_t stream_tag(int purpose, int dir, int level, int stage) {
    return ((uint32_t)purpose << 24) | ((uint32_t)dir << 16) | ((uint32_t)level << 8) | (uint32_t)stage;
}

/* ------------------------------------------------------------------------ */
/* Homography solvers.  Sec. 3.1.1: a plane is a homography, obtained by     */
/* least squares from 4 correspondences.  Both solvers use the normalised    */
/* direct linear transform: points are moved to zero mean and scaled to mean */
/* distance sqrt(2) (Hartley), each pair gives two rows of A h = 0, and h is */
/* the (unit) null vector of A.                                             */
/* ------------------------------------------------------------------------ */
static int hartley(int n, const double* p, double T[9], double* out) {
    double mx = 0, my = 0, d = 0;
    for (int i = 0; i < n; ++i) {
        mx += p[2 * i];
        my += p[2 * i + 1];
    }
    mx /= n;
    my /= n;
    for (int i = 0; i < n; ++i) d += hypot(p[2 * i] - mx, p[2 * i + 1] - my);
    d /= n;
    if (!(d > 1e-12)) return 0;
    double s = sqrt(2.0) / d;
    T[0] = s; T[1] = 0; T[2] = -s * mx;
    T[3] = 0; T[4] = s; T[5] = -s * my;
    T[6] = 0; T[7] = 0; T[8] = 1;
    for (int i = 0; i < n; ++i) {
        out[2 * i] = s * (p[2 * i] - mx);
        out[2 * i + 1] = s * (p[2 * i + 1] - my);
    }
    return 1;
}

/* the two DLT rows of the pair (x, y) -> (u, v) */
static void dlt_rows(double x, double y, double u, double v, double a[2][9]) {
    double r0[9] = {0, 0, 0, -x, -y, -1, v * x, v * y, v};
    double r1[9] = {x, y, 1, 0, 0, 0, -u * x, -u * y, -u};
    memcpy(a[0], r0, sizeof r0);
    memcpy(a[1], r1, sizeof r1);
}

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j];
}

static void inv_similarity(const double T[9], double Ti[9]) {
    /* T = [s 0 tx; 0 s ty; 0 0 1] */
    double s = T[0];
    Ti[0] = 1 / s; Ti[1] = 0; Ti[2] = -T[2] / s;
    Ti[3] = 0; Ti[4] = 1 / s; Ti[5] = -T[5] / s;
    Ti[6] = 0; Ti[7] = 0; Ti[8] = 1;
}

static void denormalise(const double Hn[9], const double Ts[9], const double Td[9], double H[9]) {
    double Tdi[9], tmp[9];
    inv_similarity(Td, Tdi);
    mat3_mul(Tdi, Hn, tmp);
    mat3_mul(tmp, Ts, H);
    double f = 0;
    for (int k = 0; k < 9; ++k) f += H[k] * H[k];
    f = sqrt(f);
    for (int k = 0; k < 9; ++k) H[k] /= f;
}

/* Minimal solver: 4 pairs give 8 equations in 9 unknowns; the null vector is
   found by Gaussian elimination with complete pivoting (the one column left
   without a pivot is the free unknown, set to 1). */
int orc_h_minimal(const double* src, const double* dst, double H[9]) {
    double Ts[9], Td[9], ps[8], pd[8];
    if (!hartley(4, src, Ts, ps) || !hartley(4, dst, Td, pd)) return 0;
    double A[8][9];
    for (int i = 0; i < 4; ++i) {
        double a[2][9];
        dlt_rows(ps[2 * i], ps[2 * i + 1], pd[2 * i], pd[2 * i + 1], a);
        memcpy(A[2 * i], a[0], sizeof a[0]);
        memcpy(A[2 * i + 1], a[1], sizeof a[1]);
    }
    int col[9];
    for (int j = 0; j < 9; ++j) col[j] = j;
    double amax = 0;
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 9; ++j) amax = fmax(amax, fabs(A[i][j]));
    for (int k = 0; k < 8; ++k) {
        int bi = k, bj = k;
        double best = -1;
        for (int i = k; i < 8; ++i)
            for (int j = k; j < 9; ++j)
                if (fabs(A[i][j]) > best) {
                    best = fabs(A[i][j]);
                    bi = i;
                    bj = j;
                }
        if (!(best > 1e-12 * amax)) return 0;
        if (bi != k)
            for (int j = 0; j < 9; ++j) {
                double t = A[k][j]; A[k][j] = A[bi][j]; A[bi][j] = t;
            }
        if (bj != k) {
            for (int i = 0; i < 8; ++i) {
                double t = A[i][k]; A[i][k] = A[i][bj]; A[i][bj] = t;
            }
            int t = col[k]; col[k] = col[bj]; col[bj] = t;
        }
        for (int i = k + 1; i < 8; ++i) {
            double f = A[i][k] / A[k][k];
            for (int j = k; j < 9; ++j) A[i][j] -= f * A[k][j];
        }
    }
    double z[9];
    z[8] = 1.0;
    for (int k = 7; k >= 0; --k) {
        double s = 0;
        for (int j = k + 1; j < 9; ++j) s += A[k][j] * z[j];
        z[k] = -s / A[k][k];
    }
    double h[9];
    for (int j = 0; j < 9; ++j) h[col[j]] = z[j];
    denormalise(h, Ts, Td, H);
    return 1;
}

/* Smallest-eigenvalue eigenvector of a symmetric 9x9 matrix by the cyclic
   Jacobi method. */
static void jacobi_min_vector_gap(double A[9][9], double v[9], double* gap);
static void jacobi_min_vector(double A[9][9], double v[9]) { jacobi_min_vector_gap(A, v, NULL); }

/* eigenvector of the smallest eigenvalue of the symmetric A (destroyed); with
   gap != NULL also (lambda_2 - lambda_1) / lambda_max, the relative gap that
   bounds how far the eigenvector moves under a perturbation of A */
static void jacobi_min_vector_gap(double A[9][9], double v[9], double* gap) {
    double V[9][9];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) V[i][j] = (i == j);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, diag = 0;
        for (int p = 0; p < 9; ++p) {
            diag += A[p][p] * A[p][p];
            for (int q = p + 1; q < 9; ++q) off += A[p][q] * A[p][q];
        }
        if (off <= 1e-32 * diag || off == 0) break;
        for (int p = 0; p < 8; ++p)
            for (int q = p + 1; q < 9; ++q) {
                if (A[p][q] == 0) continue;
                double theta = (A[q][q] - A[p][p]) / (2 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
                double c = 1 / sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < 9; ++k) { /* columns p, q */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 9; ++k) { /* rows p, q */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 9; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int m = 0;
    for (int i = 1; i < 9; ++i)
        if (A[i][i] < A[m][m]) m = i;
    for (int i = 0; i < 9; ++i) v[i] = V[i][m];
    if (gap) {
        double l1 = DBL_MAX, lmax = 0;
        for (int i = 0; i < 9; ++i) {
            lmax = fmax(lmax, fabs(A[i][i]));
            if (i != m) l1 = fmin(l1, A[i][i]);
        }
        *gap = lmax > 0 ? (l1 - A[m][m]) / lmax : 0.0;
    }
}

static int h_dlt_gap(int n, const double* src, const double* dst, double H[9], double* gap);
/* Least-squares refit over n >= 4 pairs: normalised DLT, h = eigenvector of
   A^T A with the smallest eigenvalue. */
int orc_h_dlt(int n, const double* src, const double* dst, double H[9]) { return h_dlt_gap(n, src, dst, H, NULL); }

static int h_dlt_gap(int n, const double* src, const double* dst, double H[9], double* gap) {
    if (n < 4) return 0;
    double Ts[9], Td[9];
    double* ps = (double*)malloc(sizeof(double) * 4 * n);
    double* pd = ps + 2 * n;
    int ok = hartley(n, src, Ts, ps) && hartley(n, dst, Td, pd);
    if (ok) {
        double M[9][9];
        memset(M, 0, sizeof M);
        for (int i = 0; i < n; ++i) {
            double a[2][9];
            dlt_rows(ps[2 * i], ps[2 * i + 1], pd[2 * i], pd[2 * i + 1], a);
            for (int r = 0; r < 2; ++r)
                for (int p = 0; p < 9; ++p)
                    for (int q = 0; q < 9; ++q) M[p][q] += a[r][p] * a[r][q];
        }
        double h[9];
        jacobi_min_vector_gap(M, h, gap);
        denormalise(h, Ts, Td, H);
    }
    free(ps);
    return ok;
}

/* ------------------------------------------------------------------------ */
/* Window geometry                                                           */
/* ------------------------------------------------------------------------ */
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

static int covering(const int32_t* pos, int n, int s, int x, int* idx) {
    int k = 0;
    for (int i = 0; i < n; ++i)
        if (pos[i] <= x && x < pos[i] + s) idx[k++] = i;
    return k;
}

/* colour-consistency error of eq. 3 for one pixel, with the three channels
   averaged: delta = mean_c |I_src,c(p) - I~_tgt,c(X, Y)| */
static double delta_at(const orc_params* P, const double* src, const double* tgt, int x, int y, double X,
                       double Y) {
    double s[3];
    orc_sample_bilinear(tgt, P->W, P->H, X, Y, s);
    const double* a = src + ((size_t)y * P->W + x) * 3;
    return (fabs(a[0] - s[0]) + fabs(a[1] - s[1]) + fabs(a[2] - s[2])) / 3.0;
}

/* maps p through H; returns 0 if the denominator is not positive */
static inline int map_h(const double* H, double x, double y, double* X, double* Y) {
    double w = H[6] * x + H[7] * y + H[8];
    if (!(w > 0)) return 0;
    *X = (H[0] * x + H[1] * y + H[2]) / w;
    *Y = (H[3] * x + H[4] * y + H[5]) / w;
    return 1;
}

static inline int in_frame(const orc_params* P, double X, double Y) {
    return X >= -ORC_FRAME_TOL && X <= P->W - 1 + ORC_FRAME_TOL && Y >= -ORC_FRAME_TOL && Y <= P->H - 1 + ORC_FRAME_TOL;
}

/* near the in-frame boundary (for the ambiguity logs) */
static inline int near_frame_edge(const orc_params* P, double X, double Y) {
    const double t = ORC_TIE_REL;
    return fabs(X + ORC_FRAME_TOL) < t * fmax(1, fabs(X)) || fabs(X - (P->W - 1 + ORC_FRAME_TOL)) < t * fabs(X) ||
           fabs(Y + ORC_FRAME_TOL) < t * fmax(1, fabs(Y)) || fabs(Y - (P->H - 1 + ORC_FRAME_TOL)) < t * fabs(Y);
}

/* ------------------------------------------------------------------------ */
/* Robust plane detection per window.  Sec. 3.1.2: RANSAC (Chum et al.)      */
/* keeps the hypothesis with the largest inlier support among random         */
/* 4-samples of the window's NNF matches.  Sec. 3.2: the second stage runs    */
/* on the window's residual (still unassigned) pixels only.  The winning     */
/* hypothesis (most inliers; lowest index on ties) is refitted once by least */
/* squares on its inliers; the refit is kept unless it has fewer inliers.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    double* p; /* n x 2 source points */
    double* q; /* n x 2 target points */
    int32_t* pix;
    double cx, cy; /* window centre */
} matches_t;

/* A refit whose normal matrix has a relative eigen-gap below this is not
   determined to the 1e-6 a model is compared at (its eigenvector moves by
   about 1e-16 / gap under rounding of the matrix): a property of the
   least-squares problem, logged as a near tie. */
#define ORC_REFIT_GAP 1e-8

/* Exact test that the 4-point homography of a sample has a zero
   denominator at the window centre.  With the projective bases
   P_s = [s1 s2 s3] diag(adj([s1 s2 s3]) s4) of the source points and weights
   mu = adj([t1 t2 t3]) t4 of the target points (homogeneous, z = 1), H is
   proportional to P_t adj(P_s), and P_t's third row is mu; so the
   denominator at p is proportional to mu^T adj(P_s) (p, 1).  Source points
   relative to an integer origin o near the centre (|coordinates| <= 48 for
   windows up to 96 px) and the centre doubled keep every product below
   2^110.  Such a hypothesis cannot be oriented (positive denominator at the
   centre) and is rejected like a degenerate sample. */
static int den_zero_at_centre(const int* sx, const int* sy, const int* tx, const int* ty, int ox, int oy,
                              int cx2, int cy2) {
    typedef __int128 i128;
    long long u[4], v[4];
    for (int j = 0; j < 4; ++j) {
        u[j] = sx[j] - ox;
        v[j] = sy[j] - oy;
    }
    /* M = [s1 s2 s3] (columns), lambda = adj(M) s4 */
    const long long M[9] = {u[0], u[1], u[2], v[0], v[1], v[2], 1, 1, 1};
    long long aM[9];
    aM[0] = M[4] * M[8] - M[5] * M[7];
    aM[1] = M[2] * M[7] - M[1] * M[8];
    aM[2] = M[1] * M[5] - M[2] * M[4];
    aM[3] = M[5] * M[6] - M[3] * M[8];
    aM[4] = M[0] * M[8] - M[2] * M[6];
    aM[5] = M[2] * M[3] - M[0] * M[5];
    aM[6] = M[3] * M[7] - M[4] * M[6];
    aM[7] = M[1] * M[6] - M[0] * M[7];
    aM[8] = M[0] * M[4] - M[1] * M[3];
    const long long s4[3] = {u[3], v[3], 1};
    long long lam[3];
    for (int r = 0; r < 3; ++r) lam[r] = aM[3 * r] * s4[0] + aM[3 * r + 1] * s4[1] + aM[3 * r + 2] * s4[2];
    i128 Ps[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ps[3 * r + c] = (i128)M[3 * r + c] * lam[c];
    i128 aP[9];
    aP[0] = Ps[4] * Ps[8] - Ps[5] * Ps[7];
    aP[1] = Ps[2] * Ps[7] - Ps[1] * Ps[8];
    aP[2] = Ps[1] * Ps[5] - Ps[2] * Ps[4];
    aP[3] = Ps[5] * Ps[6] - Ps[3] * Ps[8];
    aP[4] = Ps[0] * Ps[8] - Ps[2] * Ps[6];
    aP[5] = Ps[2] * Ps[3] - Ps[0] * Ps[5];
    aP[6] = Ps[3] * Ps[7] - Ps[4] * Ps[6];
    aP[7] = Ps[1] * Ps[6] - Ps[0] * Ps[7];
    aP[8] = Ps[0] * Ps[4] - Ps[1] * Ps[3];
    /* mu = adj(T) t4, T = [t1 t2 t3] (columns) */
    const long long T[9] = {tx[0], tx[1], tx[2], ty[0], ty[1], ty[2], 1, 1, 1};
    long long aT[9];
    aT[0] = T[4] * T[8] - T[5] * T[7];
    aT[1] = T[2] * T[7] - T[1] * T[8];
    aT[2] = T[1] * T[5] - T[2] * T[4];
    aT[3] = T[5] * T[6] - T[3] * T[8];
    aT[4] = T[0] * T[8] - T[2] * T[6];
    aT[5] = T[2] * T[3] - T[0] * T[5];
    aT[6] = T[3] * T[7] - T[4] * T[6];
    aT[7] = T[1] * T[6] - T[0] * T[7];
    aT[8] = T[0] * T[4] - T[1] * T[3];
    const long long t4[3] = {tx[3], ty[3], 1};
    long long mu[3];
    for (int r = 0; r < 3; ++r) mu[r] = aT[3 * r] * t4[0] + aT[3 * r + 1] * t4[1] + aT[3 * r + 2] * t4[2];
    /* (2c - 2o, 2) doubled centre */
    const long long p2[3] = {cx2 - 2LL * ox, cy2 - 2LL * oy, 2};
    i128 den = 0;
    for (int c = 0; c < 3; ++c) {
        const i128 row = (i128)mu[0] * aP[c] + (i128)mu[1] * aP[3 + c] + (i128)mu[2] * aP[6 + c];
        den += row * p2[c];
    }
    return den == 0;
}

int orc_den_zero_at_centre(const int32_t* sx, const int32_t* sy, const int32_t* tx, const int32_t* ty, int x0, int y0,
                           int s) {
    int a[4], b[4], c[4], d[4];
    for (int j = 0; j < 4; ++j) {
        a[j] = sx[j];
        b[j] = sy[j];
        c[j] = tx[j];
        d[j] = ty[j];
    }
    return den_zero_at_centre(a, b, c, d, x0 + s / 2, y0 + s / 2, 2 * x0 + s - 1, 2 * y0 + s - 1);
}

static int collinear_int(const int* x, const int* y, int a, int b, int c) {
    long long cr = (long long)(x[b] - x[a]) * (y[c] - y[a]) - (long long)(y[b] - y[a]) * (x[c] - x[a]);
    return cr == 0;
}

/* counts inliers ||H p - q||^2 < t^2 and the comparisons inside the near-tie band */
static int score_h(const double* H, const matches_t* M, double t2, int* amb, uint8_t* flags) {
    int cnt = 0, a = 0;
    for (int j = 0; j < M->n; ++j) {
        double X, Y;
        int in = 0;
        const double px = M->p[2 * j], py = M->p[2 * j + 1];
        if (map_h(H, px, py, &X, &Y)) {
            double dx = X - M->q[2 * j], dy = Y - M->q[2 * j + 1];
            double r2 = dx * dx + dy * dy;
            in = r2 < t2;
            if (rel_gap(r2, t2) < ORC_TIE_REL) ++a;
        }
        cnt += in;
        if (flags) flags[j] = (uint8_t)in;
    }
    if (amb) *amb = a;
    return cnt;
}

static void normalise_sign(double H[9], double cx, double cy) {
    double w = H[6] * cx + H[7] * cy + H[8];
    double f = 0;
    for (int k = 0; k < 9; ++k) f += H[k] * H[k];
    f = sqrt(f);
    if (w < 0) f = -f;
    for (int k = 0; k < 9; ++k) H[k] /= f;
}

static void fit_cell(const orc_params* P, const double* src, const double* tgt, int dir, int level, int stage,
                     int cell, int x0, int y0, int s, const int32_t* vx, const int32_t* vy, const uint8_t* resid,
                     double* Hout, int32_t* mi) {
    const int W = P->W, K = P->num_hyp;
    const double t2 = P->ransac_px * P->ransac_px;
    memset(mi, 0, sizeof(int32_t) * ORC_MI);
    mi[ORC_MI_BESTK] = -1;
    matches_t M;
    M.p = (double*)malloc(sizeof(double) * 4 * s * s);
    M.q = M.p + 2 * s * s;
    int* ix = (int*)malloc(sizeof(int) * 4 * s * s);
    int *iy = ix + s * s, *jx = iy + s * s, *jy = jx + s * s;
    uint8_t* fl = (uint8_t*)malloc((size_t)s * s);
    M.n = 0;
    /* the window's matches (p, p + v(p)) in raster order */
    for (int y = y0; y < y0 + s; ++y)
        for (int x = x0; x < x0 + s; ++x) {
            int i = y * W + x;
            if (stage == 2 && !resid[i]) continue;
            ix[M.n] = x;
            iy[M.n] = y;
            jx[M.n] = x + vx[i];
            jy[M.n] = y + vy[i];
            M.p[2 * M.n] = x;
            M.p[2 * M.n + 1] = y;
            M.q[2 * M.n] = x + vx[i];
            M.q[2 * M.n + 1] = y + vy[i];
            ++M.n;
        }
    const int N = M.n;
    const double cxw = x0 + 0.5 * (s - 1), cyw = y0 + 0.5 * (s - 1);
    M.cx = cxw;
    M.cy = cyw;
    mi[ORC_MI_NIN] = N;
    for (int k = 0; k < 9; ++k) Hout[k] = 0;
    if (N < P->min_inliers || N < 4) goto done;
    {
        int best = -1, bscore = -1, bamb = 0;
        double Hb[9];
        int* scores = (int*)malloc(sizeof(int) * 2 * K);
        int* ambs = scores + K;
        for (int k = 0; k < K; ++k) {
            uint32_t w[4];
            rng4(P, (uint32_t)cell, (uint32_t)k, stream_tag(3, dir, level, stage), w);
            int id[4];
            for (int j = 0; j < 4; ++j) id[j] = (int)bounded_u32(w[j], (uint32_t)N);
            scores[k] = -1;
            ambs[k] = 0;
            /* degenerate sample: three of the four source (or target) points on one line */
            int degen = 0;
            int sx[4], sy[4], tx[4], ty[4];
            for (int j = 0; j < 4; ++j) {
                sx[j] = ix[id[j]]; sy[j] = iy[id[j]];
                tx[j] = jx[id[j]]; ty[j] = jy[id[j]];
            }
            static const int TRI[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
            for (int t = 0; t < 4 && !degen; ++t)
                degen = collinear_int(sx, sy, TRI[t][0], TRI[t][1], TRI[t][2]) ||
                        collinear_int(tx, ty, TRI[t][0], TRI[t][1], TRI[t][2]);
            if (degen) continue;
            if (den_zero_at_centre(sx, sy, tx, ty, x0 + s / 2, y0 + s / 2, 2 * x0 + s - 1, 2 * y0 + s - 1)) continue;
            double ps[8], pd[8], Hk[9];
            for (int j = 0; j < 4; ++j) {
                ps[2 * j] = sx[j]; ps[2 * j + 1] = sy[j];
                pd[2 * j] = tx[j]; pd[2 * j + 1] = ty[j];
            }
            if (!orc_h_minimal(ps, pd, Hk)) continue;
            normalise_sign(Hk, cxw, cyw); /* denominator positive at the window centre */
            int a;
            scores[k] = score_h(Hk, &M, t2, &a, NULL);
            ambs[k] = a;
            if (scores[k] > bscore) {
                bscore = scores[k];
                best = k;
                bamb = a;
                memcpy(Hb, Hk, sizeof Hb);
            }
        }
        /* the winner's own inlier decisions fix its recorded score and the refit's input set */
        int ambig = bamb > 0;
        for (int k = 0; k < K && best >= 0; ++k) {
            if (k == best || scores[k] < 0) continue;
            if (k < best && scores[k] + ambs[k] >= bscore - bamb) ambig = 1;
            if (k > best && scores[k] + ambs[k] > bscore - bamb) ambig = 1;
        }
        free(scores);
        mi[ORC_MI_BESTK] = best;
        mi[ORC_MI_BESTSCORE] = bscore;
        if (best < 0 || bscore < 4) goto done;
        mi[ORC_MI_FLAGS] |= ORC_F_FITTED;
        /* least-squares refit on the winner's inliers */
        score_h(Hb, &M, t2, NULL, fl);
        double* ip = (double*)malloc(sizeof(double) * 4 * bscore);
        double* iq = ip + 2 * bscore;
        int n = 0;
        for (int j = 0; j < N; ++j)
            if (fl[j]) {
                ip[2 * n] = M.p[2 * j]; ip[2 * n + 1] = M.p[2 * j + 1];
                iq[2 * n] = M.q[2 * j]; iq[2 * n + 1] = M.q[2 * j + 1];
                ++n;
            }
        double Hr[9];
        int famb = bamb, count = bscore;
        double gap = 0;
        if (h_dlt_gap(n, ip, iq, Hr, &gap)) {
            mi[ORC_MI_GAP10] = gap > 0 ? (int)floor(-log10(gap)) : 99;
            /* the eigenvector moves by about 1e-16 / gap under rounding of the normal matrix: below
               ORC_REFIT_GAP the refit is not determined to the 1e-6 a model is compared at */
            if (!(gap >= ORC_REFIT_GAP)) ambig = 1;
            normalise_sign(Hr, cxw, cyw);
            int ramb;
            int rscore = score_h(Hr, &M, t2, &ramb, NULL);
            if (rscore >= bscore) {
                if (rscore - ramb < bscore + bamb) ambig = 1;
                memcpy(Hb, Hr, sizeof Hb);
                count = rscore;
                famb = ramb;
                mi[ORC_MI_FLAGS] |= ORC_F_REFIT;
            } else if (rscore + ramb >= bscore - bamb) {
                ambig = 1;
            }
        }
        free(ip);
        normalise_sign(Hb, cxw, cyw);
        memcpy(Hout, Hb, sizeof Hb);
        mi[ORC_MI_COUNT] = count;
        mi[ORC_MI_AMB] = famb;
        /* support, denominator and scale checks (plane validity) */
        int valid = count >= P->min_inliers && 5 * count >= N;
        if ((count - famb < P->min_inliers || 5 * (count - famb) < N) && (count + famb >= P->min_inliers && 5 * (count + famb) >= N))
            ambig = 1;
        const int r = P->r;
        double cxs[4] = {x0 - r, x0 + s - 1 + r, x0 - r, x0 + s - 1 + r};
        double cys[4] = {y0 - r, y0 - r, y0 + s - 1 + r, y0 + s - 1 + r};
        for (int c = 0; c < 4; ++c)
            if (!(Hb[6] * cxs[c] + Hb[7] * cys[c] + Hb[8] > 0)) valid = 0;
        {
            double w = Hb[6] * cxw + Hb[7] * cyw + Hb[8];
            double X = (Hb[0] * cxw + Hb[1] * cyw + Hb[2]) / w, Y = (Hb[3] * cxw + Hb[4] * cyw + Hb[5]) / w;
            double j00 = (Hb[0] - X * Hb[6]) / w, j01 = (Hb[1] - X * Hb[7]) / w;
            double j10 = (Hb[3] - Y * Hb[6]) / w, j11 = (Hb[4] - Y * Hb[7]) / w;
            double det = j00 * j11 - j01 * j10;
            if (!(det > 0)) valid = 0;
            else {
                double sc = sqrt(det);
                if (!(sc >= P->scale_min && sc <= P->scale_max)) valid = 0;
                if (rel_gap(sc, P->scale_min) < ORC_TIE_REL || rel_gap(sc, P->scale_max) < ORC_TIE_REL) ambig = 1;
            }
        }
        if (!valid) mi[ORC_MI_FLAGS] |= ORC_F_BAD_GEOM;
        mi[ORC_MI_VALID] = valid;
        /* S_R intersect S_C: RANSAC inliers of the final H that are also colour inliers */
        score_h(Hb, &M, t2, NULL, fl);
        int nrc = 0;
        for (int j = 0; j < N; ++j) {
            if (!fl[j]) continue;
            double X, Y;
            if (!map_h(Hb, M.p[2 * j], M.p[2 * j + 1], &X, &Y)) continue;
            if (near_frame_edge(P, X, Y)) ambig = 1;
            if (!in_frame(P, X, Y)) continue;
            double d = delta_at(P, src, tgt, ix[j], iy[j], X, Y);
            if (d < P->eps) ++nrc;
            if (rel_gap(d, P->eps) < ORC_TIE_REL) ambig = 1;
        }
        mi[ORC_MI_NRC] = nrc;
        if (ambig) mi[ORC_MI_FLAGS] |= ORC_F_AMBIG;
    }
done:
    free(M.p);
    free(ix);
    free(fl);
}

void orc_fit_level(const orc_params* P, const double* src, const double* tgt, int dir, int level, int stage,
                   const int32_t* vx, const int32_t* vy, const uint8_t* resid, double* mh, int32_t* mi) {
    grid_t* g = (grid_t*)malloc(sizeof(grid_t));
    make_grid(P, level, g);
    int ncell = g->ncx * g->ncy;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < ncell; ++c) {
        int cx = c % g->ncx, cy = c / g->ncx;
        int id = (g->base + c) * 2 + (stage - 1);
        fit_cell(P, src, tgt, dir, level, stage, c, g->xs[cx], g->ys[cy], g->s, vx, vy, resid,
                 mh + (size_t)id * 9, mi + (size_t)id * ORC_MI);
    }
    free(g);
}

/* The same fit for a listed subset of the level's windows (spot checks of
   single windows at full frame sizes); indices outside the level are skipped. */
void orc_fit_cells(const orc_params* P, const double* src, const double* tgt, int dir, int level, int stage,
                   const int32_t* vx, const int32_t* vy, const uint8_t* resid, const int32_t* cells, int ncells,
                   double* mh, int32_t* mi) {
    grid_t* g = (grid_t*)malloc(sizeof(grid_t));
    make_grid(P, level, g);
    const int ncell = g->ncx * g->ncy;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < ncells; ++k) {
        const int c = cells[k];
        if (c < 0 || c >= ncell) continue;
        int cx = c % g->ncx, cy = c / g->ncx;
        int id = (g->base + c) * 2 + (stage - 1);
        fit_cell(P, src, tgt, dir, level, stage, c, g->xs[cx], g->ys[cy], g->s, vx, vy, resid,
                 mh + (size_t)id * 9, mi + (size_t)id * ORC_MI);
    }
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Plane distortion compensation and assignment.  Sec. 3.1.3: warp the      */
/* target frame toward the source by the plane (I_H(p) = I~_tgt(H p)),       */
/* colour error delta (eq. 3), robust loss L = |delta| if |delta| < eps else */
/* eps (eq. 4); a pixel is an inlier iff |delta| < eps and is assigned the   */
/* inlier plane with the smallest L among the overlapping windows (lowest   */
/* window index on ties, L closer than ORC_L_TIE counting as a tie), with    */
/* the homography-induced flow H p - p.                                     */
/* ------------------------------------------------------------------------ */
void orc_assign(const orc_params* P, const double* src, const double* tgt, int level, int stage,
                const double* mh, const int32_t* mi, const uint8_t* mask,
                int32_t* lm, double* lL, double* lfx, double* lfy, uint8_t* amb) {
    const int W = P->W, H = P->H;
    grid_t* g = (grid_t*)malloc(sizeof(grid_t));
    make_grid(P, level, g);
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        int iy[8], nyw = covering(g->ys, g->ncy, g->s, y, iy);
        for (int x = 0; x < W; ++x) {
            int i = y * W + x;
            if (mask && !mask[i]) continue;
            int ix[8], nxw = covering(g->xs, g->ncx, g->s, x, ix);
            int bm = -1, a = 0;
            double bL = DBL_MAX, bfx = 0, bfy = 0;
            for (int u = 0; u < nyw; ++u)
                for (int v = 0; v < nxw; ++v) {
                    int cell = iy[u] * g->ncx + ix[v];
                    int id = (g->base + cell) * 2 + (stage - 1);
                    if (!mi[id * ORC_MI + ORC_MI_VALID]) continue;
                    const double* Hm = mh + (size_t)id * 9;
                    double X, Y;
                    if (!map_h(Hm, x, y, &X, &Y)) continue;
                    if (near_frame_edge(P, X, Y)) a = 1;
                    if (!in_frame(P, X, Y)) continue;
                    double d = delta_at(P, src, tgt, x, y, X, Y);
                    if (near_colour(d, P->eps)) a = 1;
                    if (!(d < P->eps)) continue;
                    if (bm >= 0 && near_colour(d, bL - ORC_L_TIE)) a = 1;
                    if (d < bL - ORC_L_TIE) {
                        bL = d;
                        bm = id;
                        bfx = X - x;
                        bfy = Y - y;
                    }
                }
            lm[i] = bm;
            lL[i] = bm >= 0 ? bL : P->eps;
            lfx[i] = bfx;
            lfy[i] = bfy;
            if (amb) amb[i] = (uint8_t)a;
        }
    }
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Occlusion cues, Sec. 3.4.                                                 */
/* (1) forward-backward plane projection symmetry with threshold eta: a      */
/*     pixel with plane flow f is symmetric iff q = round(p + f) holds an    */
/*     assigned pixel of the other direction whose flow g has |f + g| < t_fb; */
/*     a plane whose assigned pixels are symmetric in a fraction below eta   */
/*     is discarded;                                                        */
/* (3) overlap of the RANSAC inliers S_R and the colour-consistent region S_C:*/
/*     |S_R n S_C| / |S_R| below kappa discards the plane.                    */
/* ------------------------------------------------------------------------ */
void orc_cue_counts(const orc_params* P, int level, int stage,
                    const int32_t* lm, const double* lfx, const double* lfy,
                    const int32_t* om, const double* ofx, const double* ofy,
                    int32_t* mi, uint8_t* amb) {
    const int W = P->W, H = P->H;
    grid_t* g = (grid_t*)malloc(sizeof(grid_t));
    make_grid(P, level, g);
    int ncell = g->ncx * g->ncy;
    for (int c = 0; c < ncell; ++c) {
        int id = (g->base + c) * 2 + (stage - 1);
        mi[id * ORC_MI + ORC_MI_NASSIGN] = 0;
        mi[id * ORC_MI + ORC_MI_NSYM] = 0;
    }
    int lo = g->base * 2, hi = (g->base + ncell) * 2;
    const double t2 = P->fb_px * P->fb_px;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int i = y * W + x, m = lm[i];
            if (m < lo || m >= hi || (m & 1) != stage - 1) continue;
            mi[m * ORC_MI + ORC_MI_NASSIGN]++;
            double tx = x + lfx[i] + 0.5, ty = y + lfy[i] + 0.5;
            double gx = fmin(tx - floor(tx), floor(tx) + 1 - tx), gy = fmin(ty - floor(ty), floor(ty) + 1 - ty);
            if (amb && (gx < 1e-5 * fmax(1, fabs(tx)) || gy < 1e-5 * fmax(1, fabs(ty)))) amb[i] = 1;
            int qx = (int)floor(tx), qy = (int)floor(ty);
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
            int j = qy * W + qx;
            if (om[j] < 0) continue;
            double ex = lfx[i] + ofx[j], ey = lfy[i] + ofy[j];
            double e2 = ex * ex + ey * ey;
            if (amb && rel_gap(e2, t2) < ORC_TIE_REL) amb[i] = 1;
            if (e2 < t2) mi[m * ORC_MI + ORC_MI_NSYM]++;
        }
    free(g);
}

void orc_cue_invalidate(const orc_params* P, int level, int stage, int32_t* mi) {
    grid_t* g = (grid_t*)malloc(sizeof(grid_t));
    make_grid(P, level, g);
    int ncell = g->ncx * g->ncy;
    for (int c = 0; c < ncell; ++c) {
        int32_t* f = mi + (size_t)((g->base + c) * 2 + (stage - 1)) * ORC_MI;
        if (!f[ORC_MI_VALID]) continue;
        if (f[ORC_MI_NASSIGN] > 0 && f[ORC_MI_NSYM] < P->eta * f[ORC_MI_NASSIGN]) {
            f[ORC_MI_VALID] = 0;
            f[ORC_MI_FLAGS] |= ORC_F_BAD_FB;
        }
        if (f[ORC_MI_NRC] < P->kappa * f[ORC_MI_COUNT]) {
            f[ORC_MI_VALID] = 0;
            f[ORC_MI_FLAGS] |= ORC_F_BAD_KAPPA;
        }
    }
    free(g);
}

/* (2) Many-to-one: when several assigned pixels land on the same target
   pixel q = round(p + f), the one with the smallest colour error L (then the
   lowest index) keeps it.  A loser whose flow differs from the winner's by
   t_fb or more belongs to another moving region mapped onto an already
   matched one: it is treated as occluded and loses its assignment.  (Pixels
   of one plane that crowd onto a target under zoom, possibly carrying the
   models of two overlapping windows, have nearly equal flows and are kept.) */
void orc_many_to_one(const orc_params* P, int32_t* lm, const double* lL, const double* lfx,
                     const double* lfy, uint8_t* cue, uint8_t* amb) {
    const int W = P->W, H = P->H, n = W * H;
    double* bL = (double*)malloc(sizeof(double) * n);
    int* bi = (int*)malloc(sizeof(int) * n);
    int* tq = (int*)malloc(sizeof(int) * n);
    for (int q = 0; q < n; ++q) {
        bL[q] = DBL_MAX;
        bi[q] = -1;
    }
    for (int i = 0; i < n; ++i) {
        tq[i] = -1;
        if (lm[i] < 0) continue;
        int x = i % W, y = i / W;
        double tx = x + lfx[i] + 0.5, ty = y + lfy[i] + 0.5;
        double gx = fmin(tx - floor(tx), floor(tx) + 1 - tx), gy = fmin(ty - floor(ty), floor(ty) + 1 - ty);
        if (amb && (gx < 1e-5 * fmax(1, fabs(tx)) || gy < 1e-5 * fmax(1, fabs(ty)))) amb[i] = 1;
        int qx = (int)floor(tx), qy = (int)floor(ty);
        if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
        int q = qy * W + qx;
        tq[i] = q;
        if (bi[q] >= 0 && amb && near_colour(lL[i], bL[q])) {
            amb[i] = 1;
            amb[bi[q]] = 1;
        }
        if (lL[i] < bL[q]) { /* ties keep the lower index, which came first */
            bL[q] = lL[i];
            bi[q] = i;
        }
    }
    const double t2 = P->fb_px * P->fb_px;
    uint8_t* lose = (uint8_t*)calloc((size_t)n, 1);
    for (int i = 0; i < n; ++i) {
        int q = tq[i];
        if (q < 0) continue;
        int w = bi[q];
        if (w == i) continue;
        double ex = lfx[i] - lfx[w], ey = lfy[i] - lfy[w];
        double e2 = ex * ex + ey * ey;
        if (amb && rel_gap(e2, t2) < ORC_TIE_REL) amb[i] = 1;
        if (!(e2 < t2)) lose[i] = 1;
    }
    for (int i = 0; i < n; ++i)
        if (lose[i]) {
            lm[i] = -1;
            cue[i] |= ORC_CUE_M2O;
        }
    free(lose);
    free(bL);
    free(bi);
    free(tq);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3: flows of different levels are merged with the same min-L rule,  */
/* with priority to the coarser (earlier) level: a finer plane replaces the  */
/* accumulated one only when its L is lower by more than beta.               */
/* ------------------------------------------------------------------------ */
void orc_merge(const orc_params* P, const int32_t* lm, const double* lL, const double* lfx,
               const double* lfy, int32_t* am, double* aL, double* afx, double* afy, uint8_t* amb) {
    const int n = P->W * P->H;
    for (int i = 0; i < n; ++i) {
        if (lm[i] < 0) continue;
        if (am[i] >= 0 && amb && near_colour(lL[i], aL[i] - P->beta)) amb[i] = 1;
        if (am[i] < 0 || lL[i] < aL[i] - P->beta) {
            am[i] = lm[i];
            aL[i] = lL[i];
            afx[i] = lfx[i];
            afy[i] = lfy[i];
        }
    }
}

/* Sec. 3.3.1: plane-assigned (low colour error) correspondences overwrite the
   next level's initial NNF with the rounded plane flow and are frozen. */
void orc_nnf_update(const orc_params* P, const int32_t* am, const double* afx, const double* afy,
                    int32_t* vx, int32_t* vy, uint8_t* frozen) {
    const int n = P->W * P->H;
    for (int i = 0; i < n; ++i) {
        frozen[i] = am[i] >= 0;
        if (am[i] >= 0) {
            vx[i] = (int)floor(afx[i] + 0.5);
            vy[i] = (int)floor(afy[i] + 0.5);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4.1: homography model propagation spreads the best plane (by      */
/* colour cost) of the 4-neighbours into unfilled pixels, here as fill_iters */
/* Jacobi iterations; a neighbour's plane is taken only if it is a colour    */
/* inlier at the pixel (smallest L wins, lowest model id on ties, L closer  */
/* than ORC_L_TIE counting as a tie).                                        */
/* ------------------------------------------------------------------------ */
void orc_fill(const orc_params* P, const double* src, const double* tgt, const double* mh,
              const int32_t* mi, const uint8_t* cue, int32_t* am, double* aL, double* afx, double* afy,
              uint8_t* amb) {
    (void)mi;
    const int W = P->W, H = P->H, n = W * H;
    int32_t* nm = (int32_t*)malloc(sizeof(int32_t) * n);
    double* nL = (double*)malloc(sizeof(double) * 3 * n);
    double *nfx = nL + n, *nfy = nfx + n;
    uint8_t* namb = amb ? (uint8_t*)malloc((size_t)n) : NULL;
    for (int it = 0; it < P->fill_iters; ++it) {
        memcpy(nm, am, sizeof(int32_t) * n);
        memcpy(nL, aL, sizeof(double) * n);
        memcpy(nfx, afx, sizeof(double) * n);
        memcpy(nfy, afy, sizeof(double) * n);
        if (amb) memcpy(namb, amb, (size_t)n);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int i = y * W + x;
                if (am[i] >= 0 || (cue[i] & ORC_CUE_M2O)) continue;
                static const int NX[4] = {-1, 1, 0, 0}, NY[4] = {0, 0, -1, 1};
                int bm = -1, nd = 0, a = 0;
                double bL = DBL_MAX, bfx = 0, bfy = 0, dl[4];
                for (int k = 0; k < 4; ++k) {
                    int xx = x + NX[k], yy = y + NY[k];
                    if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                    /* a neighbour whose label rests on a near tie may hold another plane, or none */
                    if (amb && amb[yy * W + xx]) a = 1;
                    int m = am[yy * W + xx];
                    if (m < 0) continue;
                    double X, Y;
                    if (!map_h(mh + (size_t)m * 9, x, y, &X, &Y)) continue;
                    if (amb && near_frame_edge(P, X, Y)) a = 1;
                    if (!in_frame(P, X, Y)) continue;
                    double d = delta_at(P, src, tgt, x, y, X, Y);
                    if (amb && near_colour(d, P->eps)) a = 1;
                    if (!(d < P->eps)) continue;
                    dl[nd++] = d;
                    if (d < bL - ORC_L_TIE || (fabs(d - bL) <= ORC_L_TIE && m < bm)) {
                        bL = d;
                        bm = m;
                        bfx = X - x;
                        bfy = Y - y;
                    }
                }
                /* two inlier candidates whose losses differ by about the tie margin */
                for (int u = 0; amb && u < nd; ++u)
                    for (int v = u + 1; v < nd; ++v)
                        if (near_colour(fabs(dl[u] - dl[v]), ORC_L_TIE)) a = 1;
                if (amb && a) namb[i] = 1;
                if (bm >= 0) {
                    nm[i] = bm;
                    nL[i] = bL;
                    nfx[i] = bfx;
                    nfy[i] = bfy;
                }
            }
        memcpy(am, nm, sizeof(int32_t) * n);
        memcpy(aL, nL, sizeof(double) * n);
        memcpy(afx, nfx, sizeof(double) * n);
        memcpy(afy, nfy, sizeof(double) * n);
        if (amb) memcpy(amb, namb, (size_t)n);
    }
    free(nm);
    free(nL);
    free(namb);
}

/* Final flow and occlusion map (Sec. 3.4 and 3.4.1): a pixel keeps its plane
   flow if it has one, else its NNF offset.  It is occluded if no plane was
   assigned (no correct plane model), if a cue flagged it, or if the colour
   error after warping by the final flow reaches occ_thresh. */
void orc_final(const orc_params* P, const double* src, const double* tgt, const int32_t* am,
               const double* afx, const double* afy, const int32_t* vx, const int32_t* vy,
               const uint8_t* cue, float* flow, uint8_t* occ, uint8_t* amb) {
    const int W = P->W, H = P->H;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int i = y * W + x;
            double fx = am[i] >= 0 ? afx[i] : vx[i];
            double fy = am[i] >= 0 ? afy[i] : vy[i];
            flow[2 * i] = (float)fx;
            flow[2 * i + 1] = (float)fy;
            int o = am[i] < 0 || (cue[i] & ORC_CUE_M2O);
            double X = x + fx, Y = y + fy;
            if (amb && !o && near_frame_edge(P, X, Y)) amb[i] = 1;
            if (!in_frame(P, X, Y)) o = 1;
            else {
                double d = delta_at(P, src, tgt, x, y, X, Y);
                if (amb && !o && near_colour(d, P->occ_thresh)) amb[i] = 1;
                if (!(d < P->occ_thresh)) o = 1;
            }
            occ[i] = (uint8_t)o;
        }
}

/* Illumination: scale the target frame by mean(I1) / mean(I2). */
double orc_gain(const orc_params* P, const double* f1, const double* f2) {
    double s1 = 0, s2 = 0;
    size_t n = (size_t)P->W * P->H * 3;
    for (size_t i = 0; i < n; ++i) {
        s1 += f1[i];
        s2 += f2[i];
    }
    return s2 > 0 ? s1 / s2 : 1.0;
}

/* Edge-aware fill (reading in oracle_color.c): a pixel without a plane and
   with a seed takes the seed's plane at its own position (H p - p), or the
   seed's flow where that plane's denominator is not positive there. */
void orc_interp_flow(const orc_params* P, const double* mh, const int32_t* am, const double* afx, const double* afy,
                     const int32_t* seed, float* flow) {
    const int W = P->W, H = P->H;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int i = y * W + x;
            if (am[i] >= 0 || seed[i] < 0) continue;
            const int s = seed[i];
            double X, Y;
            if (map_h(mh + (size_t)am[s] * 9, x, y, &X, &Y)) {
                flow[2 * i] = (float)(X - x);
                flow[2 * i + 1] = (float)(Y - y);
            } else {
                flow[2 * i] = (float)afx[s];
                flow[2 * i + 1] = (float)afy[s];
            }
        }
}
