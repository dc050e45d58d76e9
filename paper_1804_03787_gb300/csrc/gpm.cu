// Host runtime of the C ABI declared in include/gpm.h: context and memory
// layout, stage ordering, the level loop of Algorithm 1 and state
// import/export.  All device work goes to the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gpm.h"
#include "common.cuh"
#include "kernels.h"

using namespace gpm;

namespace {

constexpr size_t kAlign = 256;

struct Slot {
    int W = 0, H = 0, n = 0;
    uint32_t pair_id = 0;
    int stage = -1;  // -1 nothing; 2l = after match(l); 2l-1 = after fit_planes(l)
    void* block = nullptr;
    PairView pv{};  // the pair's views (passed to the kernels by value)
    LevelGeom geoms[GPM_MAX_SCALES];
    int total_cells = 0, m = 0;
    double* partial = nullptr;
    double* gain = nullptr;
    bool census_costs = false;  // the NNF costs are census Hamming sums (level 0 with the census data term)
    int* eq_hist = nullptr;    // 2 x 256 V-histogram counts (HSV equalisation)
    float* eq_lut = nullptr;   // 2 x 256 equalised V per bin
    unsigned long long* d_evals = nullptr;
};

}  // namespace

struct gpm_ctx {
    gpm_params P{};
    gpm_limits lim{};
    gpm_alloc_fn alloc = nullptr;
    gpm_free_fn free_fn = nullptr;
    void* user = nullptr;
    cudaStream_t stream = nullptr;
    int nsm = 152;
    int max_n = 0, max_models = 0, max_cells = 1;
    int max_np = 0;  // texels of a padded frame copy at the largest frame size
    size_t slot_bytes = 0;
    std::vector<Slot> slots;
    std::string err;
    uint64_t launches = 0;
    // measurement: CUDA events around every launch, per kernel class
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
    };
    uint32_t prof_mask = 0;  // kernel classes whose launches are bracketed by events
    bool prof_open = false;  // the last pbeg opened a bracket
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    uint64_t prof_launches[GPM_PROF_CLASSES] = {};
};

namespace {

const int kPartialBlocks = kIngestPartialBlocks;

cudaEvent_t take_event(gpm_ctx* c) {
    if (c->pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
}

// Counts `n` kernel launches of class `cls` and, with profiling on for that
// class, opens an event bracket on the context's stream (closed by pend).
void pbeg(gpm_ctx* c, int cls, int n) {
    c->launches += n;
    c->prof_open = (c->prof_mask >> cls) & 1u;
    if (!c->prof_open) return;
    c->prof_launches[cls] += n;
    gpm_ctx::ProfRec r{cls, take_event(c), take_event(c)};
    cudaEventRecord(r.a, c->stream);
    c->recs.push_back(r);
}
void pend(gpm_ctx* c) {
    if (!c->prof_open) return;
    cudaEventRecord(c->recs.back().b, c->stream);
    c->prof_open = false;
}

gpm_status fail(gpm_ctx* c, gpm_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

gpm_status cuda_check(gpm_ctx* c, const char* where) {
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GPM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    }
    return GPM_OK;
}

constexpr int kFillRounds = 4;  // fast-sweeping rounds of the edge-aware fill

// Windows of the level with the most (refit records are per window of one level).
int max_level_cells_for(const gpm_params& P, int W, int H) {
    int mx = 1;
    for (int l = 0; l < P.num_scales; ++l) {
        LevelGeom g{};
        g.s = P.cell_size[l];
        g.h = g.s / 2;
        g.gx = make_axis(W, g.s);
        g.gy = make_axis(H, g.s);
        mx = std::max(mx, g.ncells());
    }
    return mx;
}

int total_cells_for(const gpm_params& P, int W, int H, LevelGeom* geoms) {
    int total = 0;
    for (int l = 0; l < P.num_scales; ++l) {
        LevelGeom g{};
        g.s = P.cell_size[l];
        g.h = g.s / 2;
        g.gx = make_axis(W, g.s);
        g.gy = make_axis(H, g.s);
        g.base = total;
        if (geoms) geoms[l] = g;
        total += g.ncells();
    }
    return total;
}

gpm_status validate_params(const gpm_params& P, std::string& why) {
    if (P.patch_radius < 1 || P.patch_radius > 4) return why = "patch_radius must be 1..4", GPM_EINVAL;
    if (P.num_scales < 0 || P.num_scales > GPM_MAX_SCALES) return why = "num_scales must be 0..8", GPM_EINVAL;
    for (int l = 0; l < P.num_scales; ++l) {
        const int s = P.cell_size[l];
        if (s < 4 || s > kMaxCell || (s & 1)) return why = "cell sizes must be even, 4..96", GPM_EINVAL;
    }
    if (P.pm_iters < 0 || P.pm_iters > 64) return why = "pm_iters must be 0..64", GPM_EINVAL;
    if (P.num_hyp < 1 || P.num_hyp > 4096) return why = "num_hyp must be 1..4096", GPM_EINVAL;
    if (P.min_inliers < 4) return why = "min_inliers must be >= 4", GPM_EINVAL;
    if (P.fill_iters < 0 || P.fill_iters > 1024) return why = "fill_iters must be 0..1024", GPM_EINVAL;
    if (P.storage < 0 || P.storage > 2) return why = "storage must be GPM_F32, GPM_F16 or GPM_BF16", GPM_EINVAL;
    if (P.equalize != 0 && P.equalize != 1) return why = "equalize must be 0 or 1", GPM_EINVAL;
    if (P.census != 0 && P.census != 1) return why = "census must be 0 or 1", GPM_EINVAL;
    if (P.census && !P.pm_init) return why = "census needs pm_init = 1 (a random initial NNF)", GPM_EINVAL;
    if (P.interp != 0 && P.interp != 1) return why = "interp must be 0 or 1", GPM_EINVAL;
    if (P.sweep_blocks_per_sm < 0 || P.sweep_blocks_per_sm > 32)
        return why = "sweep_blocks_per_sm must be 0..32", GPM_EINVAL;
    if (!(P.eps > 0) || !(P.ransac_px > 0) || !(P.fb_px > 0)) return why = "eps, ransac_px, fb_px must be > 0", GPM_EINVAL;
    if (!(P.scale_min > 0) || !(P.scale_max >= P.scale_min)) return why = "bad scale range", GPM_EINVAL;
    return GPM_OK;
}

// Carves one slot's buffers out of a single block; returns bytes needed.
size_t layout_slot(const gpm_params& P, int max_n, int max_np, int max_models, int max_cells, char* base, Slot* s) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = (off + kAlign - 1) / kAlign * kAlign;
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t n = (size_t)max_n, m = (size_t)max_models;
    const size_t texel = P.storage == 0 ? 16 : 8;
    PairView pv{};
    for (int d = 0; d < 2; ++d) pv.img[d] = take(n * texel);
    for (int d = 0; d < 2; ++d) pv.imgp[d] = take((size_t)max_np * texel);
    for (int d = 0; d < 2; ++d) pv.box[d] = (float4*)take(n * sizeof(float4));
    for (int d = 0; d < 2; ++d) {
        pv.nnf[d] = (int2*)take(n * sizeof(int2));
        pv.cost[d] = (float*)take(n * sizeof(float));
        pv.frozen[d] = (uint8_t*)take(n);
        pv.cue[d] = (uint8_t*)take(n);
        pv.resid[d] = (uint8_t*)take(n);
        Labels* sets[4] = {&pv.acc[d], &pv.tent[d], &pv.st1[d], &pv.lvl[d]};
        for (Labels* l : sets) {
            l->m = (int*)take(n * sizeof(int));
            l->L = (float*)take(n * sizeof(float));
            l->v = (int2*)take(n * sizeof(int2));
            l->r = (float2*)take(n * sizeof(float2));
        }
        pv.mh[d] = (double*)take(m * 9 * sizeof(double));
        pv.mef[d] = (Mef*)take(m * sizeof(Mef));
        pv.mi[d] = (int*)take(m * kMI * sizeof(int));
        pv.list[d] = (int*)take(2 * n * sizeof(int));
        pv.m2o_key[d] = (unsigned long long*)take(n * sizeof(unsigned long long));
        pv.rw[d] = (RefitWork*)take((size_t)max_cells * sizeof(RefitWork));
        pv.code[d] = (uint32_t*)take(n * sizeof(uint32_t));
    }
    pv.list_count = (int*)take(4 * sizeof(int));
    pv.flag = (int*)take(sizeof(int));
    pv.gq = (int*)take(n * sizeof(int));
    double* partial = (double*)take(sizeof(double) * 2 * kPartialBlocks);
    double* gain = (double*)take(sizeof(double));
    int* eq_hist = (int*)take(2 * 256 * sizeof(int));
    float* eq_lut = (float*)take(2 * 256 * sizeof(float));
    unsigned long long* evals = (unsigned long long*)take(GPM_COUNTERS * sizeof(unsigned long long));
    if (s) {
        s->d_evals = evals;
        s->pv = pv;
        s->partial = partial;
        s->gain = gain;
        s->eq_hist = eq_hist;
        s->eq_lut = eq_lut;
    }
    return off;
}

PlaneParams plane_params(const gpm_params& P) {
    PlaneParams pp{};
    pp.num_hyp = P.num_hyp;
    pp.min_inliers = P.min_inliers;
    pp.radius = P.patch_radius;
    pp.storage = P.storage;
    pp.t2 = P.ransac_px * P.ransac_px;
    pp.eps = P.eps;
    pp.fb2 = P.fb_px * P.fb_px;
    pp.eta = P.eta;
    pp.kappa = P.kappa;
    pp.beta = P.beta;
    pp.occ_thresh = P.occ_thresh;
    pp.scale_min = P.scale_min;
    pp.scale_max = P.scale_max;
    pp.k0 = (uint32_t)(P.seed & 0xFFFFFFFFull);
    pp.k1 = (uint32_t)(P.seed >> 32);
    return pp;
}

// Grid of the PatchMatch launches (init, recost, sweeps): the launch shape chosen by the parameters.
int pm_grid(const gpm_ctx* c) { return c->nsm * (c->P.sweep_blocks_per_sm > 0 ? c->P.sweep_blocks_per_sm : 4); }

int grid_for(const gpm_ctx* c, int n) {
    const int want = (n + 255) / 256;
    return std::max(1, std::min(want, c->nsm * 8));
}

// The kernel-parameter table of pairs [first, first + nb), nb <= kBatch (blockIdx.z = pair - first).
Batch batch(const gpm_ctx* c, int first, int nb) {
    static_assert(kMaxScales == GPM_MAX_SCALES, "level tables");
    Batch b;
    std::memset(&b, 0, sizeof b);
    for (int k = 0; k < nb; ++k) {
        const Slot& s = c->slots[first + k];
        b.pv[k] = s.pv;
        for (int l = 0; l < kMaxScales; ++l) b.geo[k][l] = s.geoms[l];
    }
    return b;
}
// Calls f(batch, nb) for pairs [first, first + np) in launches of up to kBatch pairs.
template <class F>
void each_batch(const gpm_ctx* c, int first, int np, F&& f) {
    for (int i0 = 0; i0 < np; i0 += kBatch) {
        const int nb = std::min(kBatch, np - i0);
        f(batch(c, first + i0, nb), nb);
    }
}
int batches(int np) { return (np + kBatch - 1) / kBatch; }

// Host-side sizes of the pairs 0..np-1 of a call: grids are sized for the largest.
struct Dims {
    int np = 0, max_n = 0, max_w = 0, max_h = 0, max_m = 0;
    int max_cells[GPM_MAX_SCALES] = {};
};
Dims dims_of(const gpm_ctx* c, int np) {
    Dims d;
    d.np = np;
    for (int i = 0; i < np; ++i) {
        const Slot& s = c->slots[i];
        d.max_n = std::max(d.max_n, s.n);
        d.max_w = std::max(d.max_w, s.W);
        d.max_h = std::max(d.max_h, s.H);
        d.max_m = std::max(d.max_m, s.m);
        for (int l = 0; l < c->P.num_scales; ++l) d.max_cells[l] = std::max(d.max_cells[l], s.geoms[l].ncells());
    }
    return d;
}

// Sets the slot's frame size and level geometry (its table entry is written by the caller).
gpm_status set_dims(gpm_ctx* c, Slot& s, int W, int H) {
    if (s.W == W && s.H == H) return GPM_OK;
    s.W = W;
    s.H = H;
    s.n = W * H;
    s.total_cells = total_cells_for(c->P, W, H, s.geoms);
    s.m = 2 * s.total_cells;
    s.pv.W = W;
    s.pv.H = H;
    s.pv.n = s.n;
    s.pv.Wp = W + 2 * kPad;
    s.pv.m_models = s.m;
    // a defined NNF (zero offsets) before anything reads it
    for (int d = 0; d < 2; ++d) cudaMemsetAsync(s.pv.nnf[d], 0, sizeof(int2) * s.n, c->stream);
    return cuda_check(c, "set_dims");
}

// Restricted-sweep lists of pairs [first, first + np).
void build_lists(gpm_ctx* c, int first, int np, int max_n) {
    pbeg(c, GPM_PROF_LISTS, 2 * batches(np));
    each_batch(c, first, np, [&](const Batch& b, int nb) { launch_build_lists(b, nb, grid_for(c, max_n), c->stream); });
    pend(c);
}

// One PatchMatch launch per batch of pairs.
void launch_pm_all(gpm_ctx* c, PmLaunch& L, int np) {
    each_batch(c, 0, np, [&](const Batch& b, int nb) {
        L.bt = b;
        L.np = nb;
        launch_pm(L, c->stream);
    });
}

void pm_sweeps(gpm_ctx* c, const Dims& D, int level) {
    PmLaunch L{};
    L.radius = c->P.patch_radius;
    L.storage = c->P.storage;
    L.level = level;
    L.grid_blocks = pm_grid(c);
    L.tiles0 = sweep0_tiles(D.max_w, D.max_h);
    L.k0 = (uint32_t)(c->P.seed & 0xFFFFFFFFull);
    L.k1 = (uint32_t)(c->P.seed >> 32);
    L.census = level == 0 ? c->P.census : 0;
    for (int i = 0; i < D.np; ++i) c->slots[i].census_costs = L.census != 0;
    const int nb = batches(D.np);
    if (level > 0 || !c->P.pm_init) {
        L.op = PmLaunch::RECOST;
        pbeg(c, GPM_PROF_PM_RECOST, nb);
        launch_pm_all(c, L, D.np);
        pend(c);
    }
    L.op = PmLaunch::SWEEP;
    for (int it = 0; it < c->P.pm_iters; ++it)
        for (int ph = 0; ph < 2; ++ph) {
            L.it = it;
            L.phase = ph;
            pbeg(c, level == 0 ? GPM_PROF_PM_SWEEP : GPM_PROF_PM_SWEEP_PLANE, nb);
            launch_pm_all(c, L, D.np);
            pend(c);
        }
}

// Algorithm 1 for one level on pairs 0..np-1 (both directions and every pair in each launch).
void fit_level(gpm_ctx* c, const Dims& D, int level) {
    const int s = c->P.cell_size[level - 1], mc = D.max_cells[level - 1], np = D.np, nb = batches(np);
    const PlaneParams pp = plane_params(c->P);
    const int gb = grid_for(c, D.max_n);
    cudaStream_t st = c->stream;
    auto each = [&](auto&& f) { each_batch(c, 0, np, f); };
    // first stage: fit, tentative assignment, cues on both directions, final assignment
    pbeg(c, GPM_PROF_RANSAC, 3 * nb);
    each([&](const Batch& b, int n) { launch_ransac(b, n, level, s, mc, 1, pp, st); });
    pend(c);
    pbeg(c, GPM_PROF_ASSIGN, nb);
    each([&](const Batch& b, int n) { launch_assign(b, n, level, 1, 0, 0, pp, gb, st); });
    pend(c);
    pbeg(c, GPM_PROF_CUES, 3 * nb);
    each([&](const Batch& b, int n) { launch_cues(b, n, level, mc, 1, 0, pp, gb, st); });
    pend(c);
    pbeg(c, GPM_PROF_ASSIGN, nb);
    each([&](const Batch& b, int n) { launch_assign(b, n, level, 1, 1, 1, pp, gb, st); });
    pend(c);
    // second stage on the residual pixels
    pbeg(c, GPM_PROF_RANSAC, 3 * nb);
    each([&](const Batch& b, int n) { launch_ransac(b, n, level, s, mc, 2, pp, st); });
    pend(c);
    for (int pass = 0; pass < 2; ++pass) {  // assignment, cues, then the assignment after the cues
        pbeg(c, GPM_PROF_ASSIGN, 2 * nb);
        each([&](const Batch& b, int n) {
            launch_copy_labels(b, n, 2, 3, gb, st);
            launch_assign(b, n, level, 2, 2, 0, pp, gb, st);
        });
        pend(c);
        if (pass == 0) {
            pbeg(c, GPM_PROF_CUES, 3 * nb);
            each([&](const Batch& b, int n) { launch_cues(b, n, level, mc, 2, 2, pp, gb, st); });
            pend(c);
        }
    }
    // many-to-one, merge, NNF update, lists for the restricted sweeps
    pbeg(c, GPM_PROF_MANY_TO_ONE, 3 * nb);
    each([&](const Batch& b, int n) { launch_many_to_one(b, n, pp, gb, st); });
    pend(c);
    pbeg(c, GPM_PROF_MERGE, nb);
    each([&](const Batch& b, int n) { launch_merge_update(b, n, pp, gb, st); });
    pend(c);
    build_lists(c, 0, np, D.max_n);
}

}  // namespace

extern "C" {

void gpm_default_params(gpm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->patch_radius = 3;
    p->num_scales = 3;
    p->cell_size[0] = 32;
    p->cell_size[1] = 16;
    p->cell_size[2] = 8;
    p->pm_iters = 4;
    p->num_hyp = 256;
    p->min_inliers = 8;
    p->fill_iters = 8;
    p->gain_normalize = 1;
    p->pm_init = 1;
    p->storage = GPM_F32;
    p->eps = 0.06f;
    p->ransac_px = 1.5f;
    p->fb_px = 1.0f;
    p->eta = 0.5f;
    p->kappa = 0.5f;
    p->beta = 0.015f;
    p->occ_thresh = 0.06f;
    p->scale_min = 0.5f;
    p->scale_max = 2.0f;
    p->seed = 0;
}

size_t gpm_required_bytes(const gpm_params* params, const gpm_limits* limits) {
    if (!params || !limits || limits->max_width <= 0 || limits->max_height <= 0 || limits->max_pairs <= 0) return 0;
    const int max_n = limits->max_width * limits->max_height;
    const int max_models = 2 * total_cells_for(*params, limits->max_width, limits->max_height, nullptr);
    const int max_cells = max_level_cells_for(*params, limits->max_width, limits->max_height);
    const int max_np = (limits->max_width + 2 * kPad) * (limits->max_height + 2 * kPad);
    const size_t per = layout_slot(*params, max_n, max_np, std::max(max_models, 2), max_cells, nullptr, nullptr);
    return per * (size_t)limits->max_pairs;
}

gpm_status gpm_create(const gpm_params* params, const gpm_limits* limits, gpm_alloc_fn alloc, gpm_free_fn free_fn,
                      void* user, void* stream, gpm_ctx** out) {
    if (!out) return GPM_EINVAL;
    *out = nullptr;
    if (!params || !limits) return GPM_EINVAL;
    std::string why;
    if (validate_params(*params, why) != GPM_OK) return GPM_EINVAL;
    if (limits->max_width < 4 || limits->max_height < 4 || limits->max_pairs < 1 || limits->max_pairs > 4096 ||
        (int64_t)limits->max_width * limits->max_height > (1 << 26) || limits->max_width > 32767 ||
        limits->max_height > 32767)
        return GPM_EINVAL;
    if ((alloc == nullptr) != (free_fn == nullptr)) return GPM_EINVAL;
    gpm_ctx* c = new (std::nothrow) gpm_ctx();
    if (!c) return GPM_ENOMEM;
    c->P = *params;
    c->lim = *limits;
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = user;
    c->stream = (cudaStream_t)stream;
    c->max_n = limits->max_width * limits->max_height;
    c->max_models = std::max(2, 2 * total_cells_for(*params, limits->max_width, limits->max_height, nullptr));
    c->max_cells = max_level_cells_for(*params, limits->max_width, limits->max_height);
    c->max_np = (limits->max_width + 2 * kPad) * (limits->max_height + 2 * kPad);
    c->slot_bytes = layout_slot(*params, c->max_n, c->max_np, c->max_models, c->max_cells, nullptr, nullptr);
    // the budget is checked before anything is allocated or any CUDA call is made
    if (limits->hbm_budget_bytes && c->slot_bytes * (size_t)limits->max_pairs > limits->hbm_budget_bytes) {
        delete c;
        return GPM_EBUSY;
    }
    c->slots.resize(limits->max_pairs);
    for (auto& s : c->slots) {
        void* p = nullptr;
        if (alloc) {
            p = alloc(user, c->slot_bytes, stream);
        } else if (cudaMallocAsync(&p, c->slot_bytes, c->stream) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (!p) {
            gpm_destroy(c);
            return GPM_ENOMEM;
        }
        s.block = p;
        layout_slot(*params, c->max_n, c->max_np, c->max_models, c->max_cells, (char*)p, &s);
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        gpm_destroy(c);
        return GPM_ECUDA;
    }
    // the device consistency flags start clear
    for (auto& s : c->slots) cudaMemsetAsync(s.pv.flag, 0, sizeof(int), c->stream);
    if (cuda_check(c, "gpm_create") != GPM_OK) {
        gpm_destroy(c);
        return GPM_ECUDA;
    }
    *out = c;
    return GPM_OK;
}

gpm_status gpm_destroy(gpm_ctx* c) {
    if (!c) return GPM_EINVAL;
    cudaStreamSynchronize(c->stream);
    for (auto& r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    for (auto& s : c->slots) {
        if (!s.block) continue;
        if (c->free_fn)
            c->free_fn(c->user, s.block, c->stream);
        else
            cudaFreeAsync(s.block, c->stream);
        s.block = nullptr;
    }

    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    delete c;
    return GPM_OK;
}

gpm_status gpm_match(gpm_ctx* c, const gpm_pair* pairs, int32_t n_pairs, int32_t level) {
    if (!c) return GPM_EINVAL;
    if (n_pairs < 1 || n_pairs > (int)c->slots.size()) return fail(c, GPM_EINVAL, "n_pairs out of range");
    if (level < 0 || level > c->P.num_scales) return fail(c, GPM_EINVAL, "level out of range");
    if (level == 0) {
        if (!pairs) return fail(c, GPM_EINVAL, "pairs is NULL");
        int smax = 0;
        for (int l = 0; l < c->P.num_scales; ++l) smax = std::max(smax, c->P.cell_size[l]);
        for (int i = 0; i < n_pairs; ++i) {
            const gpm_pair& p = pairs[i];
            if (!p.frame1 || !p.frame2) return fail(c, GPM_EINVAL, "NULL frame");
            if (p.dtype != GPM_F32 && p.dtype != GPM_F16 && p.dtype != GPM_BF16)
                return fail(c, GPM_EINVAL, "frame dtype must be GPM_F32, GPM_F16 or GPM_BF16");
            if (p.width < std::max(4, smax) || p.height < std::max(4, smax) || p.width > c->lim.max_width ||
                p.height > c->lim.max_height)
                return fail(c, GPM_EINVAL, "frame size outside [largest cell, limits]");
            if (p.row_stride < 3 * (int64_t)p.width) return fail(c, GPM_EINVAL, "row_stride < 3 * width");
        }
        for (int i = 0; i < n_pairs; ++i) {
            const gpm_pair& p = pairs[i];
            Slot& s = c->slots[i];
            gpm_status e = set_dims(c, s, p.width, p.height);
            if (e) return e;
            s.pair_id = p.pair_id;
            s.pv.pair_id = p.pair_id;
        }
        const Dims D = dims_of(c, n_pairs);
        // ingest of every pair, in launches of up to kBatch pairs (census codes of the frames as given:
        // census ignores a global gain; greys of frame 1 for the edge-aware fill)
        for (int i0 = 0; i0 < n_pairs; i0 += kBatch) {
            const int nj = std::min(kBatch, n_pairs - i0);
            IngestJobs J{};
            int mn = 0, mh = 0;
            for (int k = 0; k < nj; ++k) {
                const gpm_pair& p = pairs[i0 + k];
                Slot& s = c->slots[i0 + k];
                IngestJob& j = J.j[k];
                j.f1 = p.frame1;
                j.f2 = p.frame2;
                j.dtype = p.dtype;
                j.W = p.width;
                j.H = p.height;
                j.stride = p.row_stride;
                j.partial = s.partial;
                j.gain = s.gain;
                j.o1 = const_cast<void*>(s.pv.img[0]);
                j.o2 = const_cast<void*>(s.pv.img[1]);
                j.hist = c->P.equalize ? s.eq_hist : nullptr;
                j.lut = c->P.equalize ? s.eq_lut : nullptr;
                if (c->P.census) {
                    j.k1 = reinterpret_cast<long long*>(s.pv.m2o_key[0]);
                    j.k2 = reinterpret_cast<long long*>(s.pv.m2o_key[1]);
                    j.c1 = s.pv.code[0];
                    j.c2 = s.pv.code[1];
                }
                if (c->P.interp) j.gq = s.pv.gq;
                mn = std::max(mn, s.n);
                mh = std::max(mh, s.H);
            }
            pbeg(c, GPM_PROF_INGEST, (c->P.equalize ? 6 : 3) + (c->P.census ? 2 : 0) + (c->P.interp ? 1 : 0));
            launch_ingest_jobs(J, nj, mn, mh, c->P.gain_normalize, c->P.storage, c->stream);
            pend(c);
        }
        const int gb = grid_for(c, D.max_n);
        pbeg(c, GPM_PROF_INGEST, (4 + (c->P.census ? 0 : 1)) * batches(n_pairs));
        each_batch(c, 0, n_pairs, [&](const Batch& b, int nb) {
            launch_pad_frames(b, nb, c->P.storage, grid_for(c, (D.max_w + 2 * kPad) * (D.max_h + 2 * kPad)),
                              c->stream);
            if (!c->P.census) launch_box_sums(b, nb, D.max_w, D.max_h, c->P.patch_radius, c->P.storage, c->stream);
            launch_reset_models(b, nb, D.max_m, c->stream);
            launch_reset_labels(b, nb, c->P.eps, gb, c->stream);
        });
        pend(c);
        if (c->P.pm_init) {
            PmLaunch L{};
            L.op = PmLaunch::INIT;
            L.radius = c->P.patch_radius;
            L.storage = c->P.storage;
            L.grid_blocks = pm_grid(c);
            L.k0 = (uint32_t)(c->P.seed & 0xFFFFFFFFull);
            L.k1 = (uint32_t)(c->P.seed >> 32);
            L.census = c->P.census;
            pbeg(c, GPM_PROF_PM_INIT, batches(n_pairs));
            launch_pm_all(c, L, n_pairs);
            pend(c);
        } else {
            build_lists(c, 0, n_pairs, D.max_n);  // every pixel (nothing frozen) for the recost
        }
        pm_sweeps(c, D, 0);
        for (int i = 0; i < n_pairs; ++i) c->slots[i].stage = 0;
    } else {
        for (int i = 0; i < n_pairs; ++i)
            if (c->slots[i].stage != 2 * level - 1) return fail(c, GPM_EINVAL, "gpm_match(l) must follow gpm_fit_planes(l)");
        pm_sweeps(c, dims_of(c, n_pairs), level);
        for (int i = 0; i < n_pairs; ++i) c->slots[i].stage = 2 * level;
    }
    return cuda_check(c, "gpm_match");
}

gpm_status gpm_fit_planes(gpm_ctx* c, int32_t n_pairs, int32_t level) {
    if (!c) return GPM_EINVAL;
    if (n_pairs < 1 || n_pairs > (int)c->slots.size()) return fail(c, GPM_EINVAL, "n_pairs out of range");
    if (level < 1 || level > c->P.num_scales) return fail(c, GPM_EINVAL, "level out of range");
    for (int i = 0; i < n_pairs; ++i)
        if (c->slots[i].stage != 2 * (level - 1))
            return fail(c, GPM_EINVAL, "gpm_fit_planes(l) must follow gpm_match(l-1)");
    fit_level(c, dims_of(c, n_pairs), level);
    for (int i = 0; i < n_pairs; ++i) c->slots[i].stage = 2 * level - 1;
    return cuda_check(c, "gpm_fit_planes");
}

gpm_status gpm_flow_and_occlusion(gpm_ctx* c, int32_t n_pairs, float* const* flow_out, uint8_t* const* occ_out) {
    if (!c) return GPM_EINVAL;
    if (n_pairs < 1 || n_pairs > (int)c->slots.size()) return fail(c, GPM_EINVAL, "n_pairs out of range");
    if (!flow_out || !occ_out) return fail(c, GPM_EINVAL, "NULL output array");
    for (int i = 0; i < n_pairs; ++i) {
        if (!flow_out[i] || !occ_out[i]) return fail(c, GPM_EINVAL, "NULL output buffer");
        if (c->slots[i].stage < 0 || (c->slots[i].stage & 1))
            return fail(c, GPM_EINVAL, "gpm_flow_and_occlusion must follow a gpm_match call");
    }
    const PlaneParams pp = plane_params(c->P);
    const Dims D = dims_of(c, n_pairs);
    const int gb = grid_for(c, D.max_n);
    const int nb = batches(n_pairs);
    pbeg(c, GPM_PROF_FILL, (c->P.fill_iters + (c->P.fill_iters & 1)) * nb);
    each_batch(c, 0, n_pairs, [&](const Batch& b, int n) { launch_fill(b, n, pp, c->P.fill_iters, gb, c->stream); });
    pend(c);
    if (c->P.interp) {  // seeds into scratch: the many-to-one keys and the pixel lists are idle by now
        pbeg(c, GPM_PROF_FILL, (1 + 2 * kFillRounds) * nb);
        each_batch(c, 0, n_pairs, [&](const Batch& b, int n) {
            launch_fill_seeds(b, n, D.max_w, D.max_h, kFillRounds, gb, c->stream);
        });
        pend(c);
    }
    pbeg(c, GPM_PROF_FINAL, nb);
    for (int i0 = 0; i0 < n_pairs; i0 += kBatch) {  // the caller's buffers travel as kernel parameters too
        const int nf = std::min(kBatch, n_pairs - i0);
        FinalOut out{};
        for (int k = 0; k < nf; ++k) {
            out.flow[k] = flow_out[i0 + k];
            out.occ[k] = occ_out[i0 + k];
        }
        launch_final(batch(c, i0, nf), nf, pp, c->P.interp, out, gb, c->stream);
    }
    pend(c);
    return cuda_check(c, "gpm_flow_and_occlusion");
}

gpm_status gpm_sync(gpm_ctx* c) {
    if (!c) return GPM_EINVAL;
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, GPM_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
    gpm_status st = cuda_check(c, "gpm_sync");
    if (st != GPM_OK) return st;
    // device consistency flags: read, then cleared so that the context stays usable
    int bad = 0;
    for (auto& s : c->slots) {
        if (!s.block) continue;
        int f = 0;
        if (cudaMemcpy(&f, s.pv.flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_check(c, "gpm_sync");
        if (f) {
            bad |= f;
            cudaMemset(s.pv.flag, 0, sizeof(int));
        }
    }
    if (bad)
        return fail(c, GPM_EINTERNAL,
                    "device consistency check: imported labels named a model outside the model table or a "
                    "non-finite flow (those pixels were set to no plane)");
    return cuda_check(c, "gpm_sync");
}

static size_t state_bytes(const Slot& s, int what) {
    const size_t n = (size_t)s.n, m = (size_t)s.m;
    switch (what) {
        case GPM_NNF: return 2 * n * 2 * sizeof(int32_t);
        case GPM_COST: return 2 * n * sizeof(float);
        case GPM_MODELS: return 2 * m * 9 * sizeof(double);
        case GPM_MODEL_INFO: return 2 * m * kMI * sizeof(int32_t);
        case GPM_LABELS:
        case GPM_LEVEL_LABELS:
        case GPM_STAGE1_LABELS:
        case GPM_TENT_LABELS: {
            size_t a = 2 * n * (sizeof(int32_t) + sizeof(float));
            a = (a + 7) / 8 * 8;
            return a + 2 * n * 2 * sizeof(double);
        }
        case GPM_CUES: return 2 * n;
        case GPM_FRAMES: return 2 * n * 4 * sizeof(float);
        default: return 0;
    }
}

size_t gpm_state_bytes(const gpm_ctx* c, int32_t pair, int32_t what) {
    if (!c || pair < 0 || pair >= (int)c->slots.size() || c->slots[pair].n == 0) return 0;
    return state_bytes(c->slots[pair], what);
}

gpm_status gpm_export(gpm_ctx* c, int32_t pair, int32_t what, void* dst) {
    if (!c) return GPM_EINVAL;
    if (pair < 0 || pair >= (int)c->slots.size() || !dst) return fail(c, GPM_EINVAL, "bad pair or NULL destination");
    Slot& s = c->slots[pair];
    if (s.n == 0) return fail(c, GPM_EINVAL, "pair has no state yet");
    const size_t n = (size_t)s.n, m = (size_t)s.m;
    cudaStream_t st = c->stream;
    char* d = (char*)dst;
    switch (what) {
        case GPM_NNF:
            for (int k = 0; k < 2; ++k)
                cudaMemcpyAsync(d + k * n * sizeof(int2), s.pv.nnf[k], n * sizeof(int2), cudaMemcpyDeviceToDevice, st);
            break;
        case GPM_COST:
            for (int k = 0; k < 2; ++k)
                launch_cost_export(s.pv.cost[k], (float*)(d + k * n * sizeof(float)), (int)n, c->P.patch_radius,
                                   s.census_costs ? 1 : 0, st);
            break;
        case GPM_MODELS:
            for (int k = 0; k < 2; ++k)
                cudaMemcpyAsync(d + k * m * 9 * sizeof(double), s.pv.mh[k], m * 9 * sizeof(double),
                                cudaMemcpyDeviceToDevice, st);
            break;
        case GPM_MODEL_INFO:
            for (int k = 0; k < 2; ++k)
                cudaMemcpyAsync(d + k * m * kMI * sizeof(int), s.pv.mi[k], m * kMI * sizeof(int),
                                cudaMemcpyDeviceToDevice, st);
            break;
        case GPM_LABELS:
        case GPM_LEVEL_LABELS:
        case GPM_STAGE1_LABELS:
        case GPM_TENT_LABELS: {
            int* om = (int*)d;
            float* oL = (float*)(d + 2 * n * sizeof(int));
            size_t a = 2 * n * (sizeof(int32_t) + sizeof(float));
            a = (a + 7) / 8 * 8;
            double* of = (double*)(d + a);
            for (int k = 0; k < 2; ++k) {
                const Labels& l = what == GPM_LABELS         ? s.pv.acc[k]
                                  : what == GPM_LEVEL_LABELS   ? s.pv.lvl[k]
                                  : what == GPM_STAGE1_LABELS ? s.pv.st1[k]
                                                               : s.pv.tent[k];
                launch_labels_export(l, s.n, om + k * n, oL + k * n, of + k * n * 2, st);
            }
            break;
        }
        case GPM_CUES:
            for (int k = 0; k < 2; ++k) cudaMemcpyAsync(d + k * n, s.pv.cue[k], n, cudaMemcpyDeviceToDevice, st);
            break;
        case GPM_FRAMES:
            launch_frames_export(batch(c, pair, 1), s.n, c->P.storage, (float*)d, st);
            c->launches += 1;
            break;
        default:
            return fail(c, GPM_EINVAL, "unknown export kind");
    }
    return cuda_check(c, "gpm_export");
}

gpm_status gpm_import(gpm_ctx* c, int32_t pair, int32_t what, const void* src, int32_t stage) {
    if (!c) return GPM_EINVAL;
    if (pair < 0 || pair >= (int)c->slots.size() || !src) return fail(c, GPM_EINVAL, "bad pair or NULL source");
    if (stage < 0 || stage > 2 * c->P.num_scales) return fail(c, GPM_EINVAL, "stage out of range");
    Slot& s = c->slots[pair];
    if (s.n == 0) return fail(c, GPM_EINVAL, "run gpm_match(level 0) on the pair first");
    const size_t n = (size_t)s.n, m = (size_t)s.m;
    cudaStream_t st = c->stream;
    const char* d = (const char*)src;
    switch (what) {
        case GPM_NNF:
            for (int k = 0; k < 2; ++k)
                cudaMemcpyAsync(s.pv.nnf[k], d + k * n * sizeof(int2), n * sizeof(int2), cudaMemcpyDeviceToDevice, st);
            break;
        case GPM_MODELS:
            for (int k = 0; k < 2; ++k)
                cudaMemcpyAsync(s.pv.mh[k], d + k * m * 9 * sizeof(double), m * 9 * sizeof(double),
                                cudaMemcpyDeviceToDevice, st);
            launch_import_models(batch(c, pair, 1), c->P.num_scales, s.m, st);
            c->launches += 1;
            break;
        case GPM_MODEL_INFO:
            for (int k = 0; k < 2; ++k)
                cudaMemcpyAsync(s.pv.mi[k], d + k * m * kMI * sizeof(int), m * kMI * sizeof(int),
                                cudaMemcpyDeviceToDevice, st);
            launch_import_models(batch(c, pair, 1), c->P.num_scales, s.m, st);
            c->launches += 1;
            break;
        case GPM_LABELS: {
            const int* im = (const int*)d;
            const float* iL = (const float*)(d + 2 * n * sizeof(int));
            size_t a = 2 * n * (sizeof(int32_t) + sizeof(float));
            a = (a + 7) / 8 * 8;
            const double* iF = (const double*)(d + a);
            for (int k = 0; k < 2; ++k) {
                launch_labels_import(s.pv.acc[k], s.n, s.m, im + k * n, iL + k * n, iF + k * n * 2, s.pv.flag, st);
                c->launches += 1;
            }
            // frozen pixels and the restricted PatchMatch lists follow the accumulated map
            launch_frozen_from_labels(batch(c, pair, 1), 1, grid_for(c, s.n), st);
            c->launches += 1;
            build_lists(c, pair, 1, s.n);
            break;
        }
        case GPM_CUES:
            for (int k = 0; k < 2; ++k) cudaMemcpyAsync(s.pv.cue[k], d + k * n, n, cudaMemcpyDeviceToDevice, st);
            break;
        default:
            return fail(c, GPM_EINVAL, "unknown or export-only import kind");
    }
    s.stage = stage;
    return cuda_check(c, "gpm_import");
}

gpm_status gpm_profile_select(gpm_ctx* c, uint32_t class_mask, int32_t count_evals) {
    if (!c) return GPM_EINVAL;
    if (class_mask >> GPM_PROF_CLASSES) return fail(c, GPM_EINVAL, "class_mask names no kernel class");
    c->prof_mask = class_mask;
    for (int i = 0; i < (int)c->slots.size(); ++i) {
        Slot& s = c->slots[i];
        s.pv.evals = count_evals ? s.d_evals : nullptr;
        if (count_evals) cudaMemsetAsync(s.d_evals, 0, GPM_COUNTERS * sizeof(unsigned long long), c->stream);
    }
    return cuda_check(c, "gpm_profile_select");
}

gpm_status gpm_profile_enable(gpm_ctx* c, int32_t enable) {
    return gpm_profile_select(c, enable ? (1u << GPM_PROF_CLASSES) - 1u : 0u, enable);
}

gpm_status gpm_profile_read(gpm_ctx* c, double* ms, uint64_t* launches, uint64_t* evals) {
    if (!c) return GPM_EINVAL;
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, GPM_ECUDA, std::string("profile sync: ") + cudaGetErrorString(e));
    double acc[GPM_PROF_CLASSES] = {};
    for (auto& r : c->recs) {
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        acc[r.cls] += t;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    for (int k = 0; k < GPM_PROF_CLASSES; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = c->prof_launches[k];
        c->prof_launches[k] = 0;
    }
    uint64_t ev[GPM_COUNTERS] = {};
    for (auto& s : c->slots) {
        if (!s.d_evals) continue;
        unsigned long long h[GPM_COUNTERS] = {};
        cudaMemcpy(h, s.d_evals, sizeof h, cudaMemcpyDeviceToHost);
        for (int k = 0; k < GPM_COUNTERS; ++k) ev[k] += h[k];
        cudaMemset(s.d_evals, 0, sizeof h);
    }
    if (evals)
        for (int k = 0; k < GPM_COUNTERS; ++k) evals[k] = ev[k];
    return cuda_check(c, "gpm_profile_read");
}

const char* gpm_status_string(gpm_status s) {
    switch (s) {
        case GPM_OK: return "GPM_OK";
        case GPM_EINVAL: return "GPM_EINVAL";
        case GPM_ENOMEM: return "GPM_ENOMEM";
        case GPM_ECUDA: return "GPM_ECUDA";
        case GPM_EBUSY: return "GPM_EBUSY";
        case GPM_EINTERNAL: return "GPM_EINTERNAL";
    }
    return "unknown";
}

const char* gpm_last_error(const gpm_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

uint64_t gpm_launch_count(const gpm_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
