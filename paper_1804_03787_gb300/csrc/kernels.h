// Host-side launch descriptors of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gpm {

struct PmLaunch {
    enum Op { INIT, RECOST, SWEEP } op;
    const PairView* pv;
    LevelGeom geom;
    int radius, storage, level, it, phase, nrad, grid_blocks;
    int census;  // level 0: census data term (codes in pv.code)
    uint32_t k0, k1;
};
void launch_pm(const PmLaunch& L, cudaStream_t st);
// Blocks of the FP64 frame sums behind the gain (a fixed grid, so a fixed summation order): partial holds
// 2 * kIngestPartialBlocks doubles.
constexpr int kIngestPartialBlocks = 128;
// eq_hist / eq_lut (2 x 256 each, device) non-null: HSV histogram equalisation of both frames first (Sec. 4.2).
void launch_ingest(const float* f1, const float* f2, int W, int H, int64_t stride, int gain_enable, int storage,
                   double* partial, int nblk, double* gain, void* o1, void* o2, int* eq_hist, float* eq_lut,
                   cudaStream_t st);
// Padded copies of both ingested frames (imgp), borders replicating the edges.
void launch_pad_frames(const PairView& pv, int storage, int grid_blocks, cudaStream_t st);
// Patch sums of both ingested frames (pv.box), after launch_pad_frames: the level-0 sweep's lower bound.
void launch_box_sums(const PairView& pv, int radius, int storage, int grid_blocks, cudaStream_t st);
void launch_build_lists(const PairView& pv, int grid_blocks, cudaStream_t st);
// Census codes of both input frames (k1, k2: n int64 of scratch each).
void launch_census(const float* f1, const float* f2, int W, int H, int64_t stride, long long* k1, long long* k2,
                   uint32_t* c1, uint32_t* c2, cudaStream_t st);
// dst[i] = src[i] / (3 (2 radius + 1)^2), or / 24 (2 radius + 1)^2 for census costs: the NNF cost buffer holds
// raw tap sums, the export means.
void launch_cost_export(const float* src, float* dst, int n, int radius, int census, cudaStream_t st);
// Writes the level geometries (host array, copied by value into the launch) to dst: no host copy in the
// stream, so a pipeline that changes frame size can be captured into a CUDA graph.
void launch_set_geoms(const LevelGeom* host_geoms, LevelGeom* dst, cudaStream_t st);
// RGB -> RGBX storage of both frames, frame 2 scaled by *gain (a device scalar)
void launch_pack(const float* f1, const float* f2, int W, int H, int64_t stride, int storage, const double* gain,
                 void* o1, void* o2, cudaStream_t st);

struct PlaneParams {
    int num_hyp, min_inliers, radius, storage;
    float t2, eps, fb2, eta, kappa, beta, occ_thresh, scale_min, scale_max;
    uint32_t k0, k1;
};

// RANSAC per window for both directions (blockIdx.y = direction).
void launch_ransac(const PairView& pv, const LevelGeom& g, int level, int stage, const PlaneParams& pp,
                   cudaStream_t st);
// Assignment by eq. 3-4 into `out` (which = 0 tent, 1 st1, 2 lvl); stage 1 or 2; masked by resid for stage 2.
void launch_assign(const PairView& pv, const LevelGeom& g, int stage, int which, int write_resid,
                   const PlaneParams& pp, int grid_blocks, cudaStream_t st);
void launch_cues(const PairView& pv, const LevelGeom& g, int stage, int which, const PlaneParams& pp,
                 int grid_blocks, cudaStream_t st);
void launch_many_to_one(const PairView& pv, const PlaneParams& pp, int grid_blocks, cudaStream_t st);
void launch_merge_update(const PairView& pv, const PlaneParams& pp, int grid_blocks, cudaStream_t st);
void launch_fill(const PairView& pv, const PlaneParams& pp, int iters, int grid_blocks, Labels tmp, cudaStream_t st);
void launch_reset_labels(const PairView& pv, float eps, int grid_blocks, cudaStream_t st);
void launch_frozen_from_labels(const PairView& pv, int grid_blocks, cudaStream_t st);
void launch_frames_export(const PairView& pv, int storage, float* dst, cudaStream_t st);
// seed: nearest assigned pixel of each pixel (edge-aware fill), or nullptr for the plain rule (NNF offset)
void launch_final(const PairView& pv, const PlaneParams& pp, const int* seed, float* flow, uint8_t* occ,
                  int grid_blocks, cudaStream_t st);
// q = floor(1024 (R + G + B)) of a frame as given, for the geodesic steps of the fill
void launch_grey_q(const float* f, int W, int H, int64_t stride, int* q, cudaStream_t st);
// Seeds of the edge-aware fill (direction 0): dist (n int64) and seed (n int) are scratch / output
void launch_fill_seeds(const PairView& pv, const int* q, long long* dist, int* seed, int rounds, int grid_blocks,
                       cudaStream_t st);
// geoms: DEVICE array of nlev level geometries
void launch_import_models(const PairView& pv, const LevelGeom* geoms, int nlev, int m, cudaStream_t st);
void launch_labels_export(const Labels& l, int n, int* om, float* oL, double* of, cudaStream_t st);
// Imported labels are checked: a model id outside [-1, m) or a non-finite or huge flow sets *flag and the pixel
// gets no plane (so no later kernel reads outside the model table).
void launch_labels_import(const Labels& l, int n, int m, const int* im, const float* iL, const double* iF, int* flag,
                          cudaStream_t st);

}  // namespace gpm
