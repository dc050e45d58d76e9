/*
 * FP64 oracle, part 3: the whole method for one frame pair.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Order of the steps (Algorithm 1 for each level, Sec. 3.3-3.4 around it),
 * both directions d = 0 (I1 -> I2) and d = 1 (I2 -> I1) at every step:
 *   level 0   PatchMatch NNF (random init + pm_iters red-black iterations)
 *   level l   stage 1: fit every window, assign, symmetry + overlap cues on
 *             the tentative assignment of both directions, drop failing
 *             planes and assign again;
 *             stage 2: fit every window on its still-unassigned pixels,
 *             assign those pixels, cues, drop, assign again;
 *             many-to-one cue; merge into the accumulated map with coarse
 *             priority; NNF update with the reliable plane flows;
 *             PatchMatch restricted to the unassigned pixels, patches
 *             distorted by the pixel's home-window plane.
 *   end       model propagation fill, final flow and occlusion map.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t* m;
    double *L, *fx, *fy;
} labels_t;

static void labels_alloc(labels_t* l, int n) {
    l->m = (int32_t*)malloc(sizeof(int32_t) * n);
    l->L = (double*)malloc(sizeof(double) * 3 * n);
    l->fx = l->L + n;
    l->fy = l->fx + n;
}
static void labels_free(labels_t* l) {
    free(l->m);
    free(l->L);
}
static void labels_copy(labels_t* d, const labels_t* s, int n) {
    memcpy(d->m, s->m, sizeof(int32_t) * n);
    memcpy(d->L, s->L, sizeof(double) * 3 * n);
}

static void pm_run(const orc_params* P, const double* src, const double* tgt, int dir, int level,
                   const double* mh, const int32_t* mi, const uint8_t* frozen, int32_t* vx, int32_t* vy,
                   double* cost) {
    for (int it = 0; it < P->pm_iters; ++it)
        for (int ph = 0; ph < 2; ++ph) orc_pm_sweep(P, src, tgt, dir, level, it, ph, mh, mi, frozen, vx, vy, cost, NULL);
}

void orc_run(const orc_params* Pin, const double* f1in, const double* f2in, orc_state* S, int stop_after) {
    const int W = Pin->W, H = Pin->H, n = W * H;
    const size_t nf = (size_t)n * 3;
    /* census data term (Sec. 6): code frames of the frames as given, read by the level-0 PatchMatch only */
    const double* raw[2] = {f1in, f2in};  /* the frames as given (census codes, fill greys) */
    const orc_params P0 = *Pin;
    orc_params Pc = *Pin;
    Pc.census = 0;
    const orc_params* P = &Pc;
    double* code[2] = {NULL, NULL};
    if (P0.census) {
        code[0] = (double*)malloc(sizeof(double) * nf);
        code[1] = (double*)malloc(sizeof(double) * nf);
        orc_census(&P0, f1in, code[0]);
        orc_census(&P0, f2in, code[1]);
    }
    double* f1e = NULL;
    double* f2e = NULL;
    const double* f1 = f1in;
    if (P->equalize) { /* Sec. 4.2: both frames equalised in HSV, then the unchanged method */
        f1e = (double*)malloc(sizeof(double) * nf);
        f2e = (double*)malloc(sizeof(double) * nf);
        orc_hsv_equalize(P, f1in, f1e);
        orc_hsv_equalize(P, f2in, f2e);
        f1 = f1e;
        f2in = f2e;
    }
    double* f2 = (double*)malloc(sizeof(double) * nf);
    double g = P->gain_normalize ? orc_gain(P, f1, f2in) : 1.0;
    for (size_t i = 0; i < nf; ++i) f2[i] = f2in[i] * g;
    const double* src[2] = {f1, f2};
    const double* tgt[2] = {f2, f1};
    int total = orc_total_cells(P, NULL);
    uint8_t* frozen[2];
    for (int d = 0; d < 2; ++d) {
        memset(S->mh[d], 0, sizeof(double) * 9 * 2 * total);
        memset(S->mi[d], 0, sizeof(int32_t) * ORC_MI * 2 * total);
        memset(S->cue[d], 0, (size_t)n);
        for (int i = 0; i < n; ++i) {
            S->am[d][i] = -1;
            S->aL[d][i] = P->eps;
            S->afx[d][i] = 0;
            S->afy[d][i] = 0;
        }
        frozen[d] = (uint8_t*)calloc((size_t)n, 1);
    }
    /* level 0: plain PatchMatch (Sec. 3.1, 7x7 patches in Sec. 4) */
    for (int d = 0; d < 2; ++d) {
        const double* s0 = P0.census ? code[d] : src[d];
        const double* t0 = P0.census ? code[1 - d] : tgt[d];
        if (P->pm_init)
            orc_pm_init(&P0, s0, t0, d, S->vx[d], S->vy[d], S->cost[d]);
        else
            orc_pm_recost(&P0, s0, t0, 0, NULL, NULL, NULL, S->vx[d], S->vy[d], S->cost[d]);
        pm_run(&P0, s0, t0, d, 0, NULL, NULL, NULL, S->vx[d], S->vy[d], S->cost[d]);
    }
    if (stop_after == 0) goto out;
    {
        labels_t T[2], S1[2], C[2];
        uint8_t* resid[2];
        for (int d = 0; d < 2; ++d) {
            labels_alloc(&T[d], n);
            labels_alloc(&S1[d], n);
            labels_alloc(&C[d], n);
            resid[d] = (uint8_t*)malloc((size_t)n);
        }
        for (int l = 1; l <= P->num_scales; ++l) {
            /* first stage */
            for (int d = 0; d < 2; ++d)
                orc_fit_level(P, src[d], tgt[d], d, l, 1, S->vx[d], S->vy[d], NULL, S->mh[d], S->mi[d]);
            for (int d = 0; d < 2; ++d)
                orc_assign(P, src[d], tgt[d], l, 1, S->mh[d], S->mi[d], NULL, T[d].m, T[d].L, T[d].fx, T[d].fy, NULL);
            for (int d = 0; d < 2; ++d)
                orc_cue_counts(P, l, 1, T[d].m, T[d].fx, T[d].fy, T[1 - d].m, T[1 - d].fx, T[1 - d].fy, S->mi[d], NULL);
            for (int d = 0; d < 2; ++d) orc_cue_invalidate(P, l, 1, S->mi[d]);
            for (int d = 0; d < 2; ++d) {
                orc_assign(P, src[d], tgt[d], l, 1, S->mh[d], S->mi[d], NULL, S1[d].m, S1[d].L, S1[d].fx, S1[d].fy, NULL);
                for (int i = 0; i < n; ++i) resid[d][i] = S1[d].m[i] < 0;
                if (S->s1m[d]) memcpy(S->s1m[d], S1[d].m, sizeof(int32_t) * (size_t)n);
            }
            /* second stage on the residual region (Sec. 3.2) */
            for (int d = 0; d < 2; ++d)
                orc_fit_level(P, src[d], tgt[d], d, l, 2, S->vx[d], S->vy[d], resid[d], S->mh[d], S->mi[d]);
            for (int d = 0; d < 2; ++d) {
                labels_copy(&C[d], &S1[d], n);
                orc_assign(P, src[d], tgt[d], l, 2, S->mh[d], S->mi[d], resid[d], C[d].m, C[d].L, C[d].fx, C[d].fy, NULL);
            }
            for (int d = 0; d < 2; ++d)
                orc_cue_counts(P, l, 2, C[d].m, C[d].fx, C[d].fy, C[1 - d].m, C[1 - d].fx, C[1 - d].fy, S->mi[d], NULL);
            for (int d = 0; d < 2; ++d) orc_cue_invalidate(P, l, 2, S->mi[d]);
            for (int d = 0; d < 2; ++d) {
                labels_copy(&C[d], &S1[d], n);
                orc_assign(P, src[d], tgt[d], l, 2, S->mh[d], S->mi[d], resid[d], C[d].m, C[d].L, C[d].fx, C[d].fy, NULL);
            }
            /* many-to-one cue, merge, NNF update */
            for (int d = 0; d < 2; ++d) {
                orc_many_to_one(P, C[d].m, C[d].L, C[d].fx, C[d].fy, S->cue[d], NULL);
                orc_merge(P, C[d].m, C[d].L, C[d].fx, C[d].fy, S->am[d], S->aL[d], S->afx[d], S->afy[d], NULL);
                orc_nnf_update(P, S->am[d], S->afx[d], S->afy[d], S->vx[d], S->vy[d], frozen[d]);
            }
            /* PatchMatch restricted to the unassigned pixels (Sec. 3.3.2) */
            for (int d = 0; d < 2; ++d) {
                orc_pm_recost(P, src[d], tgt[d], l, S->mh[d], S->mi[d], frozen[d], S->vx[d], S->vy[d], S->cost[d]);
                pm_run(P, src[d], tgt[d], d, l, S->mh[d], S->mi[d], frozen[d], S->vx[d], S->vy[d], S->cost[d]);
            }
            if (stop_after == l) break;
        }
        for (int d = 0; d < 2; ++d) {
            labels_free(&T[d]);
            labels_free(&S1[d]);
            labels_free(&C[d]);
            free(resid[d]);
        }
        if (stop_after >= 1 && stop_after <= P->num_scales) goto out;
    }
    /* fill and final flow / occlusion (Sec. 3.4.1) */
    for (int d = 0; d < 2; ++d) {
        orc_fill(P, src[d], tgt[d], S->mh[d], S->mi[d], S->cue[d], S->am[d], S->aL[d], S->afx[d], S->afy[d], NULL);
        orc_final(P, src[d], tgt[d], S->am[d], S->afx[d], S->afy[d], S->vx[d], S->vy[d], S->cue[d], S->flow[d], S->occ[d],
                  NULL);
        if (P->interp) { /* edge-aware fill of the pixels left without a plane */
            int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
            int32_t* seed = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
            orc_grey_q(P, raw[d], q);
            orc_interp_seeds(P, q, S->am[d], seed);
            orc_interp_flow(P, S->mh[d], S->am[d], S->afx[d], S->afy[d], seed, S->flow[d]);
            free(q);
            free(seed);
        }
    }
out:
    for (int d = 0; d < 2; ++d) free(frozen[d]);
    free(f2);
    free(f1e);
    free(f2e);
    free(code[0]);
    free(code[1]);
}
