/*
 * FP64 CPU oracle for Multi-Scale Generalized Plane Match (arXiv 1804.03787).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, step-by-step restatement
 * of the method in double precision.  It exists to check the CUDA library
 * against the paper; only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header or table with the CUDA
 * path, and the CUDA path never calls it.
 *
 * Conventions (the readings of the paper that both sides follow are stated
 * where they are used):
 *   frames      double, H x W x 3 (HWC), values in [0,1]
 *   NNF         int32 vx[H*W], vy[H*W]; target p + v is inside the frame
 *   labels      int32 model[H*W] (-1 = none), double L, fx, fy per pixel
 *   models      per direction, indexed by a global model id
 *               id = (cell_base[level] + cell) * 2 + (stage - 1);
 *               mh[id*9] = H (row major, maps source -> target pixels,
 *               normalised to unit Frobenius norm and positive denominator
 *               at the window centre), mi[id*ORC_MI] = integer fields below.
 */
#ifndef GPM_ORACLE_H
#define GPM_ORACLE_H
#include <stdint.h>

#define ORC_MAX_SCALES 8

typedef struct {
    int32_t W, H, r;                 /* frame size, patch radius */
    int32_t num_scales;
    int32_t cell[ORC_MAX_SCALES];    /* window side per level, coarse to fine */
    int32_t pm_iters, num_hyp, min_inliers, fill_iters;
    int32_t gain_normalize, pm_init;
    int32_t equalize;                /* HSV V-channel histogram equalisation of both frames (Sec. 4.2) */
    int32_t census;                  /* census data term for the level-0 NNF (Sec. 6); inside the PatchMatch
                                        routines: the frames given are census code frames */
    int32_t interp, pad1;            /* interp: edge-aware fill of the pixels left without a plane */
    double eps, ransac_px, fb_px, eta, kappa, beta, occ_thresh, scale_min, scale_max;
    uint64_t seed;
    uint32_t pair_id, pad;
} orc_params;

/* integer model fields */
enum {
    ORC_MI_VALID = 0,   /* 1 if the model survives every check */
    ORC_MI_COUNT,       /* inliers of the final H among the RANSAC input */
    ORC_MI_NIN,         /* number of matches given to RANSAC */
    ORC_MI_BESTK,       /* winning hypothesis index (-1 if none) */
    ORC_MI_BESTSCORE,   /* its inlier count */
    ORC_MI_FLAGS,       /* ORC_F_* bits */
    ORC_MI_NRC,         /* |S_R intersect S_C| (RANSAC inliers that are colour inliers) */
    ORC_MI_NASSIGN,     /* pixels assigned to the model (tentative labels) */
    ORC_MI_NSYM,        /* of those, forward-backward symmetric */
    ORC_MI_AMB,         /* ambiguous residual comparisons of the winner */
    ORC_MI_GAP10,       /* refit: floor(-log10) of the relative eigen-gap of its normal matrix (0: none) */
    ORC_MI_RESERVED1,
    ORC_MI
};
enum {
    ORC_F_FITTED = 1,      /* RANSAC produced a model */
    ORC_F_REFIT = 2,       /* the least-squares refit replaced the minimal H */
    ORC_F_AMBIG = 4,       /* the winner or the refit choice rests on a near tie */
    ORC_F_BAD_FB = 8,      /* invalidated by the symmetry cue (eta) */
    ORC_F_BAD_KAPPA = 16,  /* invalidated by the RANSAC/colour overlap cue (kappa) */
    ORC_F_BAD_GEOM = 32    /* failed support, denominator or scale checks */
};

/* per-pixel cue bits */
enum { ORC_CUE_M2O = 1 };

/* near-tie band (relative) used for the ambiguity logs */
#define ORC_TIE_REL 1e-5
/* a warped sample point counts as inside the frame up to this far beyond the
   border (clamped bilinear sampling is continuous there) */
#define ORC_FRAME_TOL 1e-3
/* a later plane displaces the current best one only if its robust loss L is
   lower by more than this (planes of one surface fitted in overlapping windows
   give equal L up to rounding; the first window keeps the pixel) */
#define ORC_L_TIE 1e-6
/* absolute floor of the near-tie band for decisions on a colour error (eq. 3):
   an FP32 evaluation of one carries up to ~1e-6 of rounding, and a decision
   compares two of them */
#define ORC_L_ATOL 2e-6

/* ---- counter-based RNG: Philox4x32-10 (Salmon et al., SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- window grid (Sec. 3.1.2: windows overlap their predecessor by half) ---- */
int orc_grid_axis(int n, int s, int32_t* pos);      /* returns count, fills pos (may be NULL) */
int orc_total_cells(const orc_params* P, int32_t* cell_base /* [num_scales+1] or NULL */);

/* ---- sampling and patch cost (eq. 2-3, patches warped by a plane) ---- */
void orc_sample_bilinear(const double* img, int W, int H, double X, double Y, double out[3]);
/* patch costs evaluated since the last reset (timing instrumentation) */
long long orc_eval_count(int reset);
double orc_patch_cost(const orc_params* P, const double* src, const double* tgt,
                      int px, int py, int vx, int vy, const double* G /* NULL = identity */);

/* ---- PatchMatch (Sec. 3.1, 3.3.2) ---- */
void orc_pm_init(const orc_params* P, const double* src, const double* tgt, int dir,
                 int32_t* vx, int32_t* vy, double* cost);
void orc_pm_recost(const orc_params* P, const double* src, const double* tgt, int level,
                   const double* mh, const int32_t* mi, const uint8_t* frozen,
                   const int32_t* vx, const int32_t* vy, double* cost);
void orc_pm_sweep(const orc_params* P, const double* src, const double* tgt, int dir, int level,
                  int it, int phase, const double* mh, const int32_t* mi, const uint8_t* frozen,
                  int32_t* vx, int32_t* vy, double* cost, double* amb /* per pixel, may be NULL */);

/* ---- homography solvers (Sec. 3.1.1) ---- */
int orc_h_minimal(const double* src /*4x2*/, const double* dst /*4x2*/, double H[9]);
int orc_h_dlt(int n, const double* src /*nx2*/, const double* dst /*nx2*/, double H[9]);

/* ---- robust plane fit per window (Sec. 3.1.2, 3.2) ---- */
void orc_fit_level(const orc_params* P, const double* src, const double* tgt, int dir, int level,
                   int stage, const int32_t* vx, const int32_t* vy, const uint8_t* resid,
                   double* mh, int32_t* mi);

/* exact: the 4-point homography of sample (s -> t) has a zero denominator at the centre of the window of
   side s at (x0, y0); such a hypothesis cannot be oriented and is rejected */
int orc_den_zero_at_centre(const int32_t* sx, const int32_t* sy, const int32_t* tx, const int32_t* ty, int x0, int y0,
                           int s);
void orc_fit_cells(const orc_params* P, const double* src, const double* tgt, int dir, int level, int stage,
                   const int32_t* vx, const int32_t* vy, const uint8_t* resid, const int32_t* cells, int ncells,
                   double* mh, int32_t* mi);

/* ---- plane distortion compensation and assignment (eq. 3-4) ---- */
void orc_assign(const orc_params* P, const double* src, const double* tgt, int level, int stage,
                const double* mh, const int32_t* mi, const uint8_t* mask,
                int32_t* lm, double* lL, double* lfx, double* lfy, uint8_t* amb);

/* ---- occlusion cues (Sec. 3.4) ---- */
void orc_cue_counts(const orc_params* P, int level, int stage,
                    const int32_t* lm, const double* lfx, const double* lfy,
                    const int32_t* om, const double* ofx, const double* ofy,
                    int32_t* mi, uint8_t* amb);
void orc_cue_invalidate(const orc_params* P, int level, int stage, int32_t* mi);
void orc_many_to_one(const orc_params* P, int32_t* lm, const double* lL, const double* lfx,
                     const double* lfy, uint8_t* cue, uint8_t* amb);

/* ---- cross-level merge and NNF update (Sec. 3.3, 3.3.1) ---- */
void orc_merge(const orc_params* P, const int32_t* lm, const double* lL, const double* lfx,
               const double* lfy, int32_t* am, double* aL, double* afx, double* afy, uint8_t* amb);
void orc_nnf_update(const orc_params* P, const int32_t* am, const double* afx, const double* afy,
                    int32_t* vx, int32_t* vy, uint8_t* frozen);

/* ---- filling and final occlusion map (Sec. 3.4.1) ---- */
/* amb (per pixel, may be NULL): in, the pixels whose label may differ on another evaluation of the same state;
   out, also those whose fill choice or occlusion decision rests on a near tie (colour error within the band of
   eps, occ_thresh or of the tie margin between two candidates; target within the band of the frame edge), or
   that looked at a neighbour marked in the previous iteration */
void orc_fill(const orc_params* P, const double* src, const double* tgt, const double* mh,
              const int32_t* mi, const uint8_t* cue, int32_t* am, double* aL, double* afx, double* afy,
              uint8_t* amb);
void orc_final(const orc_params* P, const double* src, const double* tgt, const int32_t* am,
               const double* afx, const double* afy, const int32_t* vx, const int32_t* vy,
               const uint8_t* cue, float* flow /*HxWx2*/, uint8_t* occ, uint8_t* amb);

/* ---- gain normalisation of the target frame ---- */
double orc_gain(const orc_params* P, const double* f1, const double* f2);

/* ---- HSV histogram equalisation (Sec. 4.2), oracle_color.c ---- */
void orc_rgb_to_hsv(double r, double g, double b, double* h, double* s, double* v);
void orc_hsv_to_rgb(double h, double s, double v, double* r, double* g, double* b);
int orc_v_lut(const orc_params* P, const double* rgb, double* lut);      /* 0: frame left unchanged */
void orc_hsv_equalize(const orc_params* P, const double* in, double* out);
/* ---- census data term (Sec. 6), oracle_color.c ---- */
void orc_census(const orc_params* P, const double* rgb, double* codes);   /* code frame: (code, 0, 0) per pixel */
int orc_popcount32(uint32_t v);
/* ---- edge-aware fill of unassigned pixels, oracle_color.c ---- */
void orc_grey_q(const orc_params* P, const double* rgb, int32_t* q);              /* floor(1024 (R+G+B)) */
void orc_interp_seeds(const orc_params* P, const int32_t* q, const int32_t* am, int32_t* seed);
void orc_interp_flow(const orc_params* P, const double* mh, const int32_t* am, const double* afx, const double* afy,
                     const int32_t* seed, float* flow);

/* ---- whole method (Algorithm 1 for every level, then Sec. 3.4) ---- */
typedef struct {
    /* per direction d in {0: I1->I2, 1: I2->I1}; caller-allocated */
    int32_t* vx[2]; int32_t* vy[2]; double* cost[2];
    double* mh[2]; int32_t* mi[2];
    int32_t* am[2]; double* aL[2]; double* afx[2]; double* afy[2];
    uint8_t* cue[2];
    float* flow[2]; uint8_t* occ[2];
    int32_t* s1m[2];   /* optional (NULL = not wanted): the first-stage labels of the last level run */
} orc_state;

/* stop_after: -1 = run everything; 0 = after level-0 PatchMatch;
   l >= 1 = after level l's restricted PatchMatch. */
void orc_run(const orc_params* P, const double* f1, const double* f2, orc_state* S, int stop_after);

#endif
