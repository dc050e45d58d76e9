// Host-side launch descriptors of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gpm {

// Every launch covers np <= kBatch pairs (blockIdx.z = pair; Batch: their views and level geometries, a kernel
// parameter); grid sizes come from the largest pair.
struct PmLaunch {
    enum Op { INIT, RECOST, SWEEP } op;
    Batch bt;
    int np;
    int radius, storage, level, it, phase, grid_blocks;
    int tiles0;  // level-0 sweep: its tiles for the largest pair (sweep0_tiles)
    int census;  // level 0: census data term (codes in pv.code)
    uint32_t k0, k1;
};
void launch_pm(const PmLaunch& L, cudaStream_t st);
// Tiles (blocks per direction and pair) of the level-0 sweep of a W x H frame.
int sweep0_tiles(int W, int H);
// Blocks of the FP64 frame sums behind the gain (a fixed grid, so a fixed summation order): partial holds
// 2 * kIngestPartialBlocks doubles.
constexpr int kIngestPartialBlocks = 128;
// One pair's ingest: its frames as given and the buffers the ingest fills.
struct IngestJob {
    const void* f1;  // frames as given, elements of type `dtype` (gpm_dtype)
    const void* f2;
    int dtype;
    int W, H;
    int64_t stride;
    double* partial;  // 2 * kIngestPartialBlocks doubles
    double* gain;     // one double
    void* o1;         // ingested frames (RGBX in the storage type)
    void* o2;
    int* hist;        // HSV equalisation (Sec. 4.2): 2 x 256 counts and tables, or nullptr
    float* lut;
    long long* k1;    // census codes (Sec. 6): grey-key scratch (n each) and the codes, or nullptr
    long long* k2;
    uint32_t* c1;
    uint32_t* c2;
    int* gq;          // greys of frame 1 for the edge-aware fill, or nullptr
};
// The jobs of one ingest launch (kernel parameters, blockIdx.z = job).
struct IngestJobs {
    IngestJob j[kBatch];
};
// Ingest of nj pairs (every optional part where the job asks for it); max_n, max_h: the largest frame's pixels
// and rows among them.
void launch_ingest_jobs(const IngestJobs& J, int nj, int max_n, int max_h, int gain_enable, int storage,
                        cudaStream_t st);
// One pair: eq_hist / eq_lut (2 x 256 each, device) non-null: HSV histogram equalisation of both frames first.
void launch_ingest(const float* f1, const float* f2, int W, int H, int64_t stride, int gain_enable, int storage,
                   double* partial, int nblk, double* gain, void* o1, void* o2, int* eq_hist, float* eq_lut,
                   cudaStream_t st);
// Padded copies of both ingested frames (imgp), borders replicating the edges.
void launch_pad_frames(const Batch& bt, int np, int storage, int grid_blocks, cudaStream_t st);
// Patch sums of both ingested frames (pv.box), after launch_pad_frames: the level-0 sweep's lower bound.
void launch_box_sums(const Batch& bt, int np, int max_w, int max_h, int radius, int storage, cudaStream_t st);
// The unfrozen pixels of each colour (the restricted sweeps' lists), counts cleared first.
void launch_build_lists(const Batch& bt, int np, int grid_blocks, cudaStream_t st);
// dst[i] = src[i] / (3 (2 radius + 1)^2), or / 24 (2 radius + 1)^2 for census costs: the NNF cost buffer holds
// raw tap sums, the export means.
void launch_cost_export(const float* src, float* dst, int n, int radius, int census, cudaStream_t st);

struct PlaneParams {
    int num_hyp, min_inliers, radius, storage;
    float t2, eps, fb2, eta, kappa, beta, occ_thresh, scale_min, scale_max;
    uint32_t k0, k1;
};

// Every launch below covers np <= kBatch pairs (blockIdx.z) whose views and level geometries are in bt; grid
// sizes come from the largest pair (max_cells: the most windows a pair has at the level).
// RANSAC per window for both directions (blockIdx.y = direction); s: the level's window side.
void launch_ransac(const Batch& bt, int np, int level, int s, int max_cells, int stage, const PlaneParams& pp,
                   cudaStream_t st);
// Assignment by eq. 3-4 into `which` (0 tent, 1 st1, 2 lvl); stage 1 or 2; masked by resid for stage 2.
void launch_assign(const Batch& bt, int np, int level, int stage, int which, int write_resid, const PlaneParams& pp,
                   int grid_blocks, cudaStream_t st);
void launch_cues(const Batch& bt, int np, int level, int max_cells, int stage, int which, const PlaneParams& pp,
                 int grid_blocks, cudaStream_t st);
void launch_many_to_one(const Batch& bt, int np, const PlaneParams& pp, int grid_blocks, cudaStream_t st);
void launch_merge_update(const Batch& bt, int np, const PlaneParams& pp, int grid_blocks, cudaStream_t st);
// Copies label set `from` into `to` (0 acc, 1 tent, 2 st1, 3 lvl), both directions.
void launch_copy_labels(const Batch& bt, int np, int from, int to, int grid_blocks, cudaStream_t st);
void launch_fill(const Batch& bt, int np, const PlaneParams& pp, int iters, int grid_blocks, cudaStream_t st);
void launch_reset_labels(const Batch& bt, int np, float eps, int grid_blocks, cudaStream_t st);
// Clears every model of each pair (ids below its m_models); max_models: the most a pair has.
void launch_reset_models(const Batch& bt, int np, int max_models, cudaStream_t st);
void launch_frozen_from_labels(const Batch& bt, int np, int grid_blocks, cudaStream_t st);
// One pair (entry 0 of bt): both ingested frames as FP32 RGBX (n pixels each).
void launch_frames_export(const Batch& bt, int n, int storage, float* dst, cudaStream_t st);
// Seeds of the edge-aware fill (direction 0), into the pairs' scratch (many-to-one keys, pixel lists).
void launch_fill_seeds(const Batch& bt, int np, int max_w, int max_h, int rounds, int grid_blocks, cudaStream_t st);
// Final flow and occlusion into out (pair z of the launch: out.flow[z], out.occ[z]); interp: the edge-aware fill.
void launch_final(const Batch& bt, int np, const PlaneParams& pp, int interp, const FinalOut& out, int grid_blocks,
                  cudaStream_t st);
// One pair (entry 0 of bt): evaluation forms of imported models.
void launch_import_models(const Batch& bt, int nlev, int m, cudaStream_t st);
void launch_labels_export(const Labels& l, int n, int* om, float* oL, double* of, cudaStream_t st);
// Imported labels are checked: a model id outside [-1, m) or a non-finite or huge flow sets *flag and the pixel
// gets no plane (so no later kernel reads outside the model table).
void launch_labels_import(const Labels& l, int n, int m, const int* im, const float* iL, const double* iF, int* flag,
                          cudaStream_t st);

}  // namespace gpm
