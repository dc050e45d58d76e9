/*
 * gpm.h -- C ABI of the GB300 (sm_103a) implementation of the data-parallel
 * hot path of Multi-Scale Generalized Plane Match for optical flow
 * (Choi and Banerjee, arXiv 1804.03787).
 *
 * One call per stage of the paper's problem statement:
 *   gpm_match(level 0)       the initial PatchMatch NNF (Sec. 3.1; 7x7 patches
 *                            in Sec. 4);
 *   gpm_fit_planes(level l)  Algorithm 1 for one level: robust plane
 *                            detection per overlapping window (Sec. 3.1.2),
 *                            plane distortion compensation and assignment
 *                            (Sec. 3.1.3, eq. 3-4), the residual second stage
 *                            (Sec. 3.2), occlusion cues (Sec. 3.4), the
 *                            cross-level merge and the NNF update (Sec. 3.3,
 *                            3.3.1);
 *   gpm_match(level l >= 1)  PatchMatch restricted to unassigned pixels, with
 *                            plane-distorted patches (Sec. 3.3.2);
 *   gpm_flow_and_occlusion   model propagation fill and the final flow and
 *                            occlusion map (Sec. 3.4.1).
 *
 * Conventions
 *   - All pointers to frames, flows and maps are DEVICE pointers unless a
 *     parameter says "host".  Sizes are in elements unless they say bytes.
 *   - Every call enqueues work on the context's CUDA stream and returns
 *     without synchronising.  Results are valid once that stream has
 *     reached them.  Argument errors are reported synchronously
 *     (GPM_EINVAL) before anything is enqueued.  A failed CUDA launch is
 *     reported by the call that enqueued it (GPM_ECUDA).  A consistency
 *     check on the device (imported labels that name a model outside the
 *     model table) is reported by gpm_sync (GPM_EINTERNAL).
 *   - No exception or C++ type crosses this boundary.  A context is used by
 *     one host thread at a time.
 *   - Ownership: the caller owns frames and outputs; the context owns every
 *     intermediate buffer, allocated at gpm_create through the caller's
 *     allocator callbacks (or cudaMallocAsync when they are NULL) and released
 *     by gpm_destroy.
 *   - Stage order per pair: match(0), then fit_planes(l) and match(l) for
 *     l = 1..num_scales, then flow_and_occlusion.  Out-of-order calls return
 *     GPM_EINVAL.
 */
#ifndef GPM_H
#define GPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPM_OK = 0,
    GPM_EINVAL = 1,     /* bad argument, shape, parameter or call order */
    GPM_ENOMEM = 2,     /* the allocator callback returned NULL */
    GPM_ECUDA = 3,      /* a CUDA runtime call failed (or no CUDA device) */
                        /* 4 is not used */
    GPM_EBUSY = 5,      /* the context would exceed its HBM budget */
    GPM_EINTERNAL = 6   /* a device-side consistency check failed (reported by gpm_sync) */
} gpm_status;

/* storage type of the frames inside the context (arithmetic is FP32) */
typedef enum { GPM_F32 = 0, GPM_F16 = 1, GPM_BF16 = 2 } gpm_dtype;

#define GPM_MAX_SCALES 8

/* Method parameters.  Names follow the paper where it names them. */
typedef struct {
    int32_t patch_radius;                 /* r: 3 -> 7x7 (Sec. 4), 4 -> 9x9 */
    int32_t num_scales;                   /* levels k of Sec. 3.3 */
    int32_t cell_size[GPM_MAX_SCALES];    /* window side per level, coarse to fine; even, 4..96 */
    int32_t pm_iters;                     /* PatchMatch red-black iterations per run */
    int32_t num_hyp;                      /* RANSAC hypotheses per window, 1..4096 */
    int32_t min_inliers;                  /* minimum RANSAC support (>= 4) */
    int32_t fill_iters;                   /* model propagation iterations */
    int32_t gain_normalize;               /* 1: scale I2 by mean(I1)/mean(I2) */
    int32_t pm_init;                      /* 1: random initial NNF; 0: keep the current one */
    int32_t storage;                      /* gpm_dtype of the ingested frames */
    int32_t equalize;                     /* 1: equalise each frame's HSV value histogram first (Sec. 4.2) */
    float eps;                            /* epsilon of eq. 4 (mean |RGB| error, frames in [0,1]) */
    float ransac_px;                      /* RANSAC inlier radius in pixels */
    float fb_px;                          /* forward-backward / many-to-one flow tolerance */
    float eta;                            /* symmetric-overlap threshold of Sec. 3.4 */
    float kappa;                          /* RANSAC / colour inlier overlap threshold */
    float beta;                           /* coarse-level priority margin in the merge */
    float occ_thresh;                     /* final warp-error occlusion threshold */
    float scale_min, scale_max;           /* plane validity: local area scale range */
    int32_t census;                       /* 1: level-0 PatchMatch on 5x5 census codes, Hamming cost (Sec. 6) */
    uint64_t seed;                        /* Philox4x32-10 key */
    int32_t interp;                       /* 1: pixels left without a plane take the geodesically nearest
                                             assigned pixel's plane (edge-aware fill; EpicFlow stand-in) */
    int32_t sweep_blocks_per_sm;          /* launch shape of the PatchMatch launches: blocks per SM of the grid
                                             (0 = 4; 1..32) of the initial field, the recosts and the sweeps
                                             other than level 0 with colour patches (one block per tile);
                                             results do not depend on it */
} gpm_params;

/* Capacity of a context, fixed at creation. */
typedef struct {
    int32_t max_width, max_height;        /* largest frame */
    int32_t max_pairs;                    /* pairs processed per call */
    int32_t reserved;
    size_t hbm_budget_bytes;              /* 0 = no limit; else gpm_create fails with GPM_EBUSY above it */
} gpm_limits;

/* One frame pair.  Frames are caller-owned DEVICE buffers, H x W x 3 (HWC), values in [0,1] stored as
   `dtype` (a gpm_dtype: GPM_F32, GPM_F16 or GPM_BF16; both frames alike), row stride in elements
   (>= 3 * width).  FP16/BF16 elements are converted to FP32 exactly on ingest, so a pair gives the same
   results as the FP32 frames holding the same values.  Any other dtype: GPM_EINVAL. */
typedef struct {
    int32_t width, height;
    int64_t row_stride;
    const void* frame1;
    const void* frame2;
    uint32_t pair_id;                     /* Philox counter word: results depend on it */
    int32_t dtype;                        /* gpm_dtype of the frames (0 = GPM_F32) */
} gpm_pair;

/* Optional allocator (e.g. PyTorch's caching allocator).  alloc returns a
   device pointer aligned to 256 bytes, or NULL. */
typedef void* (*gpm_alloc_fn)(void* user, size_t bytes, void* stream);
typedef void (*gpm_free_fn)(void* user, void* ptr, void* stream);

typedef struct gpm_ctx gpm_ctx;

/* Fills *p with the default parameters (7x7 patches, cells 32/16/8, ...). */
void gpm_default_params(gpm_params* p);

/* Creates a context for up to limits->max_pairs pairs of at most
   max_width x max_height.  stream: a cudaStream_t (NULL = legacy default).
   Order of the checks: GPM_EINVAL (bad params or limits); GPM_EBUSY when
   gpm_required_bytes exceeds a non-zero hbm_budget_bytes (nothing is
   allocated and no CUDA call is made); GPM_ENOMEM when the allocator
   callback (or cudaMallocAsync) returns NULL -- what was allocated is freed
   through free_fn; GPM_ECUDA when no CUDA device answers.  *out is NULL on
   error. */
gpm_status gpm_create(const gpm_params* params, const gpm_limits* limits, gpm_alloc_fn alloc,
                      gpm_free_fn free_fn, void* user, void* stream, gpm_ctx** out);

/* Releases everything the context allocated (synchronises its stream). */
gpm_status gpm_destroy(gpm_ctx* ctx);

/* Bytes of device memory a context with these parameters and limits holds. */
size_t gpm_required_bytes(const gpm_params* params, const gpm_limits* limits);

/* Batches: each stage of gpm_match / gpm_fit_planes / gpm_flow_and_occlusion
   is one kernel launch per 8 pairs of the call, whatever their sizes: the
   pairs' views and level geometries travel in the launch's parameters and
   the pair index is on the device (blockIdx.z).  Each pair's result is
   bitwise what it gets alone.  No call copies from the host in the stream,
   so a whole multi-pair pipeline can be captured in a CUDA graph. */

/* level 0: ingest the pairs' frames (RGB -> RGBX storage, gain
   normalisation), initial NNF for both directions (random offsets from
   Philox, Sec. 3.1) and pm_iters red-black PatchMatch iterations.
   level l >= 1: PatchMatch restricted to the pixels without an assigned
   plane after gpm_fit_planes(l), patches distorted by the pixel's home
   window plane (Sec. 3.3.2).  pairs is a HOST array of n_pairs descriptors;
   at level >= 1 it may be NULL (the pairs of the last level-0 call are
   used).  n_pairs outside 1..max_pairs (an empty batch included), frames
   smaller than the largest window or beyond the limits, and a level out of
   the stage order return GPM_EINVAL before anything is enqueued. */
gpm_status gpm_match(gpm_ctx* ctx, const gpm_pair* pairs, int32_t n_pairs, int32_t level);

/* Algorithm 1 for level l (1 <= l <= num_scales) on every pair of the last
   gpm_match(0): both RANSAC stages per window, assignment by eq. 3-4, the
   symmetry, overlap and many-to-one cues of Sec. 3.4, the coarse-priority
   merge of Sec. 3.3 and the NNF update of Sec. 3.3.1.  GPM_EINVAL for n_pairs
   outside 1..max_pairs or a level out of the stage order. */
gpm_status gpm_fit_planes(gpm_ctx* ctx, int32_t n_pairs, int32_t level);

/* Model propagation fill, final flow and occlusion map (Sec. 3.4.1) for the
   forward direction I1 -> I2.  flow_out[i]: DEVICE buffer H x W x 2 float
   (x, y); occ_out[i]: DEVICE buffer H x W uint8 (1 = occluded).  Both are
   HOST arrays of n_pairs device pointers. */
gpm_status gpm_flow_and_occlusion(gpm_ctx* ctx, int32_t n_pairs, float* const* flow_out,
                                  uint8_t* const* occ_out);

/* Waits for the context's stream and reports any pending device error:
   GPM_ECUDA for a CUDA error, GPM_EINTERNAL when a device consistency check
   failed since the last gpm_sync (an imported label named a model id outside
   [-1, m) or carried a non-finite flow: that pixel was set to no plane, so
   nothing read outside the model table).  The flag is cleared when reported,
   and the context stays usable. */
gpm_status gpm_sync(gpm_ctx* ctx);

/* ---- state export / import (parity checks, resume at a level boundary) ----
   All buffers are DEVICE pointers; n = width * height of the pair,
   m = number of models of one direction = 2 * (total windows over all
   levels), model id = (first window of the level + window) * 2 + stage - 1.
   Layouts (direction-major: [direction 0 = I1->I2, direction 1 = I2->I1]):
     GPM_NNF        int32  [2][n][2]   offsets (dx, dy) to the match p + v
     GPM_COST       float  [2][n]      patch cost of the current offset
     GPM_MODELS     double [2][m][9]   homographies (row major, source ->
                                       target pixels, unit Frobenius norm,
                                       positive denominator at the window centre)
     GPM_MODEL_INFO int32  [2][m][12]  valid, inliers, RANSAC input size,
                                       winning hypothesis, its inliers, flags,
                                       |S_R n S_C|, assigned, symmetric, 3 x 0;
                                       fewer than max(4, min_inliers) matches:
                                       winner -1, its inliers 0; enough matches
                                       but every sample degenerate: winner -1,
                                       its inliers -1
     GPM_LABELS     int32  [2][n] model id (-1 none), then float [2][n] L,
                    then double [2][n][2] plane flow (8-byte aligned: the
                    float block is padded to a multiple of 8 bytes)
                                                              (accumulated map)
     GPM_LEVEL_LABELS same layout: this level's labels after the cues
     GPM_STAGE1_LABELS same layout: this level's first-stage labels
     GPM_CUES       uint8  [2][n]      bit 0 = many-to-one occlusion cue
     GPM_FRAMES     float  [2][n][4]   ingested frames as FP32 RGBX (export only)
     GPM_TENT_LABELS same layout as GPM_LABELS: this level's first-stage
                    tentative labels, before the cues dropped any plane (the
                    labels the symmetry cue counts; export only)
   Import accepts GPM_NNF, GPM_MODELS (+ valid bits from GPM_MODEL_INFO when
   imported right after), GPM_LABELS (also sets the frozen pixels: those with
   a plane) and GPM_CUES; it sets the stage order so that the next call may
   follow the imported state. */
enum {
    GPM_NNF = 0,
    GPM_COST = 1,
    GPM_MODELS = 2,
    GPM_MODEL_INFO = 3,
    GPM_LABELS = 4,
    GPM_LEVEL_LABELS = 5,
    GPM_STAGE1_LABELS = 6,
    GPM_CUES = 7,
    GPM_FRAMES = 8,
    GPM_TENT_LABELS = 9
};
/* Bytes of one export of `what` for pair `pair` (0 if unknown). */
size_t gpm_state_bytes(const gpm_ctx* ctx, int32_t pair, int32_t what);
gpm_status gpm_export(gpm_ctx* ctx, int32_t pair, int32_t what, void* dst_device);
/* stage: where in the stage order the imported state belongs: 2l = after
   gpm_match(l) (0 = after the level-0 PatchMatch), 2l - 1 = after
   gpm_fit_planes(l). */
gpm_status gpm_import(gpm_ctx* ctx, int32_t pair, int32_t what, const void* src_device, int32_t stage);

/* ---- measurement ----
   With profiling on, every kernel launch of the context is bracketed by CUDA
   events on the context's stream, and the kernels count their work (counts
   on request only, see gpm_profile_select):
     GPM_COUNT_SWEEP0         candidate offsets evaluated by the level-0
                              sweeps (one evaluation = one (2r+1)^2-tap,
                              3-channel patch cost, possibly abandoned);
     GPM_COUNT_SWEEP_PLANE    the same for the restricted, plane-distorted
                              sweeps of levels >= 1;
     GPM_COUNT_RANSAC         RANSAC residual tests (scored hypotheses x
                              window matches);
     GPM_COUNT_INIT           evaluations of the initial field and recosts;
     GPM_COUNT_SWEEP0_TAPS    taps the level-0 sweep evaluations actually
                              summed (an abandoned evaluation stops early);
     GPM_COUNT_SWEEP_PLANE_TAPS  the same for the plane-level sweeps;
     GPM_COUNT_SWEEP0_PRUNED  level-0 sweep candidates rejected without any
                              tap by the patch-sum lower bound (not counted
                              as evaluations);
     GPM_COUNT_RANSAC_FP64    RANSAC residual tests whose FP32 decision was
                              within its rounding bound, decided again in FP64;
     GPM_COUNT_RANSAC_LOOSE   hypotheses whose window-wide rounding bound was
                              too loose, tested with a bound per match.
   gpm_profile_read synchronises the stream, returns per kernel class the
   summed device milliseconds and the launch count, and the GPM_COUNTERS
   counts, then clears them.  Host arrays: ms[GPM_PROF_CLASSES],
   launches[GPM_PROF_CLASSES], counts[GPM_COUNTERS]. */
enum {
    GPM_COUNT_SWEEP0 = 0,
    GPM_COUNT_SWEEP_PLANE = 1,
    GPM_COUNT_RANSAC = 2,
    GPM_COUNT_INIT = 3,
    GPM_COUNT_SWEEP0_TAPS = 4,
    GPM_COUNT_SWEEP_PLANE_TAPS = 5,
    GPM_COUNT_SWEEP0_PRUNED = 6,
    GPM_COUNT_RANSAC_FP64 = 7,
    GPM_COUNT_RANSAC_LOOSE = 8,
    GPM_COUNTERS = 9
};
enum {
    GPM_PROF_INGEST = 0,
    GPM_PROF_PM_INIT = 1,
    GPM_PROF_PM_SWEEP = 2,        /* level-0 square-patch sweeps */
    GPM_PROF_PM_SWEEP_PLANE = 3,  /* restricted, plane-distorted sweeps */
    GPM_PROF_PM_RECOST = 4,
    GPM_PROF_RANSAC = 5,
    GPM_PROF_ASSIGN = 6,
    GPM_PROF_CUES = 7,
    GPM_PROF_MANY_TO_ONE = 8,
    GPM_PROF_MERGE = 9,
    GPM_PROF_LISTS = 10,
    GPM_PROF_FILL = 11,
    GPM_PROF_FINAL = 12,
    GPM_PROF_CLASSES = 13
};
gpm_status gpm_profile_enable(gpm_ctx* ctx, int32_t enable);
/* Finer control: bracket only the launches of the kernel classes whose bit
   (1 << GPM_PROF_*) is set in class_mask, and count evaluations only if
   count_evals != 0 (the counters add atomics and reductions to the kernels).
   gpm_profile_enable(ctx, e) is gpm_profile_select(ctx, e ? all : 0, e).
   GPM_EINVAL for a bit beyond the last class. */
gpm_status gpm_profile_select(gpm_ctx* ctx, uint32_t class_mask, int32_t count_evals);
gpm_status gpm_profile_read(gpm_ctx* ctx, double* ms, uint64_t* launches, uint64_t* evals);

/* ---- measurement aid ----
   The paper has no counterpart to this call.  It launches, on `stream`,
   `blocks` blocks of 256 threads, each thread running 8 independent chains
   of iters x 64 FP32 fused multiply-adds, and writes one float per thread to
   sink (a DEVICE buffer of blocks x 256 floats).  One launch executes
   blocks x 256 x iters x 512 FP32 lane operations; timed with CUDA events
   on the same stream it measures the FP32 lane-operation peak that the
   PatchMatch kernels' ALU roofline is quoted against.  GPM_EINVAL for
   blocks or iters outside 1..2^20 or a NULL sink, GPM_ECUDA if the launch
   fails (an error earlier work left pending is reported too). */
gpm_status gpm_fp32_peak_probe(int32_t blocks, int32_t iters, float* sink, void* stream);

/* ---- ingest without allocation ----
   The paper has no counterpart to this call.  It serves callers that must
   not allocate device memory when they ingest a pair: real-time and embedded
   hosts whose device memory is reserved once at start-up, plugins of
   frameworks that own the device memory pool and forbid allocations behind
   their back, and latency-critical loops where cudaMalloc (and the
   synchronisation it can bring) is not allowed.
   It runs the ingest of gpm_match(level 0) -- the same kernels on the same
   grid, so the output is bitwise the same: frame1/frame2 are DEVICE
   buffers, height x width x 3 FP32 (HWC, row stride in elements); out1/out2
   are caller-owned DEVICE buffers of width x height RGBX texels in `storage`
   (GPM_F32: 16 bytes each, GPM_F16 / GPM_BF16: 8 bytes); with equalize, each
   frame's HSV value histogram is equalised first (Sec. 4.2); with
   gain_normalize, frame 2 is then scaled by mean(I1) / mean(I2).
   It allocates nothing: its scratch is one static device array of 6.25 KiB
   (partial sums, the gain, the histograms and tables), held on every GPU that
   loads the library until the process exits.  Frames up to 32767 x 32767
   and 2^26 pixels (the largest frame a context takes); larger ones, NULL
   pointers, a row stride below 3 * width or a bad storage / equalize value
   return GPM_EINVAL before anything is enqueued.  GPM_ECUDA if a CUDA call
   fails; an error that earlier work left pending in the CUDA runtime is
   reported and cleared by this call too.  The first call on a device looks
   up the array's device address (once per device, with that device
   current); make that first call before any stream capture.  All calls share
   the array: calls that overlap on the GPU (unordered streams) race, so
   order them.  stream: a cudaStream_t (NULL = legacy default). */
gpm_status gpm_ingest_noalloc(const float* frame1, const float* frame2, int32_t width, int32_t height,
                              int64_t row_stride, int32_t gain_normalize, int32_t equalize, int32_t storage,
                              void* out1, void* out2, void* stream);

/* Human-readable status name and the context's last error message. */
const char* gpm_status_string(gpm_status s);
const char* gpm_last_error(const gpm_ctx* ctx);

/* Kernel launches the context has enqueued since creation (all calls). */
uint64_t gpm_launch_count(const gpm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GPM_H */
