// Batched MPPI iterations over many independent controllers.
//
// One iteration of every controller in the batch is ONE persistent rollout
// launch (one CTA per SM) whose CTAs take (controller, sample tile) items
// from an atomic work queue - FP32 CUDA-core tiles and FP16- or BF16-split
// tensor-core tiles alike, longest first - followed by one launch of the
// weights/update for all controllers.  The autotuner picks, per controller
// shape, the producer threads per sample of its tensor-core tiles (128, 64 or
// 32 samples per tile) from measured tile times, and orders the queue by
// them.  States, nominal controls, outputs and the Philox iteration counters
// live in device buffers owned by the batch, so the whole iteration (queue
// reset, rollout, update) can be captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "common.cuh"

// handle internals shared with abi.cu
#include "handles.cuh"

using namespace gpm;

namespace {

constexpr uint32_t kBatchMagic = 0x42415431u;   // "BAT1"

int check_ctrl_handle(gpmppi_ctrl c) {
    if (!c || c->magic != kCtrlMagicValue || !c->gp || c->gp->magic != kGpMagicValue)
        return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_create: invalid controller handle");
    if (c->ens && c->fmt < 0)
        return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_batch_create: FP32 terrain ensembles are not batched");
    return GPMPPI_OK;
}

}  // namespace

struct gpmppi_batch_s {
    uint32_t magic = kBatchMagic;
    int B = 0;
    int device = 0;
    std::vector<gpmppi_ctrl> ctrls;
    std::vector<size_t> uoff, woff;     // offsets (floats) of each controller's U and weights
    size_t utotal = 0, wtotal = 0;
    float* states = nullptr;            // B x 5
    float* U_nom = nullptr;             // packed T_i x 2
    float* U_new = nullptr;
    float* weights = nullptr;           // packed K_i
    unsigned long long* iters = nullptr;
    RolloutArgs* d_args = nullptr;
    MmaArgs* d_mm = nullptr;
    UpdateArgs* d_uargs = nullptr;
    int* d_ncta = nullptr;
    CUtensorMap* d_tmaps = nullptr;     // per controller: TMA map over L^-T (FP32 controllers)
    int4* d_items = nullptr;            // (controller, tile, kind, threads per sample)
    int nitems = 0;
    unsigned int* d_head = nullptr;     // the work queue's next item
    int2* d_uitems = nullptr;
    int nuitems = 0;
    std::vector<RolloutArgs> h_args;
    std::vector<MmaArgs> h_mm;
    std::vector<int> rps;               // per controller: producer threads per sample (tensor cores)
    std::vector<double> tile_us;        // per controller: estimated (or measured) time of one tile
    int smem = 0;                       // dynamic shared memory of the persistent launch
    int grid = 1;
    int maxT = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
};

namespace {

bool valid_batch(gpmppi_batch b) { return b && b->magic == kBatchMagic; }

void free_batch(gpmppi_batch b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->states);
    cudaFree(b->U_nom);
    cudaFree(b->U_new);
    cudaFree(b->weights);
    cudaFree(b->iters);
    cudaFree(b->d_args);
    cudaFree(b->d_mm);
    cudaFree(b->d_uargs);
    cudaFree(b->d_ncta);
    cudaFree(b->d_tmaps);
    cudaFree(b->d_items);
    cudaFree(b->d_head);
    cudaFree(b->d_uitems);
    b->magic = 0;
    delete b;
}

void drop_graph(gpmppi_batch b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

int kind_of(gpmppi_ctrl c) { return c->fmt < 0 ? 0 : 1 + c->fmt; }

// samples per tile of controller i
int tile_samples(gpmppi_batch b, int i) {
    gpmppi_ctrl c = b->ctrls[i];
    return c->fmt < 0 ? c->mt : 256 / b->rps[i];
}

int tile_count(gpmppi_batch b, int i) {
    const int ms = tile_samples(b, i);
    return (b->ctrls[i]->p.K + ms - 1) / ms;
}

// time of one tile before anything was measured: proportional to the
// tensor-core MMAs of its horizon (the FP32 path taken ~8x slower per sample)
double tile_estimate(gpmppi_batch b, int i) {
    gpmppi_ctrl c = b->ctrls[i];
    const double T = c->p.T, np = c->gp->g.Np > 0 ? c->gp->g.Np : 1;
    if (c->fmt < 0) return T * np * np * c->mt / 128.0 * 8.0e-6;
    double n2 = 0.0;                      // the GPs' triangles (one GP, or a terrain ensemble)
    for (int t = 0; t < c->mm.tr.M; ++t) {
        const double nt = 128.0 * (c->mm.tr.blk0[t + 1] - c->mm.tr.blk0[t]);
        n2 += nt * nt;
    }
    return T * (n2 > 0.0 ? n2 : 1.0) * (c->mm.lo_set ? 1.5 : 1.0) * 1.0e-6;
}

// A terrain ensemble's weights may change between steps (mppi_set_terrain_weights
// on its controller): the batch's copy of its launch arguments follows before
// the next step (an ordered copy on the step's stream, outside any capture).
int refresh_weights(gpmppi_batch b, cudaStream_t st) {
    bool dirty = false;
    for (int i = 0; i < b->B; ++i) {
        gpmppi_ctrl c = b->ctrls[i];
        if (!c->ens || c->fmt < 0) continue;
        for (int t = 0; t < c->mm.tr.M; ++t)
            if (b->h_mm[i].tr.w[t] != c->mm.tr.w[t]) {
                b->h_mm[i].tr.w[t] = c->mm.tr.w[t];
                dirty = true;
            }
    }
    if (dirty)
        GPM_CUDA(cudaMemcpyAsync(b->d_mm, b->h_mm.data(), sizeof(MmaArgs) * b->B, cudaMemcpyHostToDevice, st));
    return GPMPPI_OK;
}

// the work queue: every controller's tiles, longest tile first
int build_items(gpmppi_batch b) {
    std::vector<int> ids(b->B);
    std::iota(ids.begin(), ids.end(), 0);
    std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return b->tile_us[x] > b->tile_us[y]; });
    std::vector<int4> items;
    int smem = 0;
    for (int i : ids) {
        gpmppi_ctrl c = b->ctrls[i];
        const int n = tile_count(b, i);
        for (int t = 0; t < n; ++t) items.push_back(make_int4(i, t, kind_of(c), c->fmt < 0 ? 0 : b->rps[i]));
        if (c->fmt < 0) {
            smem = std::max(smem, rollout_fp32_smem_bytes(c->gp->g.Np, rollout_fp32_mtp(c->gp->g.Np), c->stages));
        } else {
            MmaArgs mm = c->mm;
            mm.rps = b->rps[i];
            smem = std::max(smem, rollout_mma_smem(mm, c->S, c->O));
        }
    }
    // each controller's tensor-core layout (threads per sample) as chosen
    for (int i = 0; i < b->B; ++i) b->h_mm[i].rps = b->rps[i];
    GPM_CUDA(cudaMemcpy(b->d_mm, b->h_mm.data(), sizeof(MmaArgs) * b->B, cudaMemcpyHostToDevice));
    cudaFree(b->d_items);
    b->d_items = nullptr;
    b->nitems = (int)items.size();
    if (!items.empty()) {
        GPM_CUDA(cudaMalloc(&b->d_items, items.size() * sizeof(int4)));
        GPM_CUDA(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    int nsm = 0;
    GPM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = std::max(1, std::min(nsm, b->nitems));
    b->smem = smem;
    drop_graph(b);
    return GPMPPI_OK;
}

int enqueue_step(gpmppi_batch b, cudaStream_t st) {
    int rc;
    GPM_CUDA(cudaMemsetAsync(b->d_head, 0, sizeof(unsigned int), st));
    if ((rc = launch_rollout_persistent(b->d_args, b->d_mm, b->d_tmaps, b->d_items, b->nitems, b->d_head, b->grid,
                                        b->smem, st)))
        return rc;
    return launch_update_batched(b->d_uargs, b->d_uitems, b->d_ncta, b->iters, b->nuitems, b->maxT, st);
}

// Measured tile times per controller shape, kept for the process: a shape is
// (precision, K, T, Np, lane segments, obstacles) and the value (threads per
// sample, microseconds per tile).
using ShapeKey = std::tuple<int, int, int, int, int, int, int>;
std::map<ShapeKey, std::pair<int, double>> g_tuned;
std::mutex g_tuned_mu;

ShapeKey shape_of(gpmppi_ctrl c) {
    // a terrain ensemble: its total block count and number of GPs
    if (c->ens) return ShapeKey(c->fmt, c->p.K, c->p.T, 128 * c->mm.nblocks, c->S, c->O, c->mm.tr.M);
    return ShapeKey(c->fmt, c->p.K, c->p.T, c->gp->g.Np, c->S, c->O, 1);
}

// time of one wave of tiles of controller i (at most one tile per SM) with
// rps producer threads per sample (tensor cores) or its FP32 tiles
int time_wave(gpmppi_batch b, int i, int rps, int nsm, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
              double* us, int* tiles_out) {
    gpmppi_ctrl c = b->ctrls[i];
    RolloutArgs a = b->h_args[i];
    const int ms = c->fmt < 0 ? c->mt : 256 / rps;
    const int tiles = (c->p.K + ms - 1) / ms;
    a.K = std::min(c->p.K, nsm * ms);           // one wave; u~ is laid out for this K (scratch)
    MmaArgs mm = c->mm;
    mm.rps = rps;
    int rc = GPMPPI_OK;
    float best = 1e30f;
    for (int rep = 0; rep < 3 && !rc; ++rep) {
        cudaEventRecord(e0, st);
        rc = c->fmt < 0 ? launch_rollout_fp32(a, &c->tmW, false, st) : launch_rollout_mma(a, mm, c->fmt, false, st);
        cudaEventRecord(e1, st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "mppi_batch_autotune");
        float ms_ = 0.0f;
        cudaEventElapsedTime(&ms_, e0, e1);
        if (rep > 0) best = std::min(best, ms_);      // the first launch warms up
    }
    if (rc) return rc;
    *us = 1e3 * best;
    *tiles_out = tiles;
    return GPMPPI_OK;
}

}  // namespace

extern "C" {

int mppi_batch_create(const gpmppi_ctrl* ctrls, int32_t B, gpmppi_batch* out) {
    try {
        if (!out) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_create: out must not be NULL");
        *out = nullptr;
        if (!ctrls || B < 1) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_create: need at least one controller");
        int dev = 0;
        GPM_CUDA(cudaGetDevice(&dev));
        int rc;
        for (int i = 0; i < B; ++i) {
            if ((rc = check_ctrl_handle(ctrls[i]))) return rc;
            if (ctrls[i]->device != dev)
                return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_create: controllers must live on the current device");
            if (ctrls[i]->p.variance_mode != GPMPPI_VAR_PER_SAMPLE)
                return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_batch_create: nominal variance mode is not batched");
            for (int j = 0; j < i; ++j)
                if (ctrls[j] == ctrls[i])
                    return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_create: a controller appears twice");
        }
        gpmppi_batch b = new (std::nothrow) gpmppi_batch_s;
        if (!b) return fail(GPMPPI_ERR_OOM, "mppi_batch_create: host allocation failed");
        b->B = B;
        b->device = dev;
        b->ctrls.assign(ctrls, ctrls + B);
        for (int i = 0; i < B; ++i) {
            b->uoff.push_back(b->utotal);
            b->woff.push_back(b->wtotal);
            b->utotal += (size_t)2 * ctrls[i]->p.T;
            b->wtotal += (size_t)ctrls[i]->p.K;
            b->maxT = std::max(b->maxT, (int)ctrls[i]->p.T);
        }
        auto fail_free = [&](int code) {
            free_batch(b);
            return code;
        };
        auto alloc = [&](void** p, size_t bytes) -> int {
            cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
            if (e != cudaSuccess) return cuda_fail(e, "mppi_batch_create: cudaMalloc");
            return GPMPPI_OK;
        };
        if ((rc = alloc((void**)&b->states, sizeof(float) * 5 * B)) ||
            (rc = alloc((void**)&b->U_nom, sizeof(float) * b->utotal)) ||
            (rc = alloc((void**)&b->U_new, sizeof(float) * b->utotal)) ||
            (rc = alloc((void**)&b->weights, sizeof(float) * b->wtotal)) ||
            (rc = alloc((void**)&b->iters, sizeof(unsigned long long) * B)) ||
            (rc = alloc((void**)&b->d_args, sizeof(RolloutArgs) * B)) ||
            (rc = alloc((void**)&b->d_mm, sizeof(MmaArgs) * B)) ||
            (rc = alloc((void**)&b->d_uargs, sizeof(UpdateArgs) * B)) ||
            (rc = alloc((void**)&b->d_ncta, sizeof(int) * B)) ||
            (rc = alloc((void**)&b->d_tmaps, sizeof(CUtensorMap) * B)) ||
            (rc = alloc((void**)&b->d_head, sizeof(unsigned int))))
            return fail_free(rc);
        std::vector<unsigned long long> its(B);
        std::vector<UpdateArgs> uargs(B);
        std::vector<int> ncta(B);
        std::vector<int2> uitems;
        b->h_args.resize(B);
        b->h_mm.resize(B);
        b->rps.assign(B, 2);
        b->tile_us.assign(B, 0.0);
        std::vector<CUtensorMap> tmaps(B);
        const float zero_state[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i < B; ++i) {
            gpmppi_ctrl c = ctrls[i];
            its[i] = c->it;
            RolloutArgs a = make_rollout_args(c, zero_state, b->U_nom + b->uoff[i]);
            a.x0_dev = b->states + 5 * i;
            a.expire_first = 0;                 // the failure-detection hook is not batched
            a.it_dev = b->iters + i;
            a.costs = c->costs;
            b->h_args[i] = a;
            b->h_mm[i] = c->mm;
            tmaps[i] = c->tmW;
            if (c->fmt >= 0) b->rps[i] = c->mm.rps;
            b->tile_us[i] = tile_estimate(b, i);
            {
                std::lock_guard<std::mutex> lock(g_tuned_mu);
                auto hit = g_tuned.find(shape_of(c));
                if (hit != g_tuned.end()) {
                    if (c->fmt >= 0) b->rps[i] = hit->second.first;
                    b->tile_us[i] = hit->second.second;
                }
            }
            UpdateArgs& u = uargs[i];
            u.costs = c->costs;
            u.u_tilde = c->u_tilde;
            u.U = b->U_nom + b->uoff[i];
            u.U_new = b->U_new + b->uoff[i];
            u.weights = b->weights + b->woff[i];
            u.partial = c->partial;
            u.counter = c->counter;
            u.K = c->p.K;
            u.T = c->p.T;
            u.per_cta = 256;
            u.inv_lambda = 1.0f / c->p.lambda;
            ncta[i] = c->n_upd;
            for (int t = 0; t < c->n_upd; ++t) uitems.push_back(make_int2(i, t));
        }
        cudaError_t e = cudaMemcpy(b->iters, its.data(), sizeof(unsigned long long) * B, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_args, b->h_args.data(), sizeof(RolloutArgs) * B, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_mm, b->h_mm.data(), sizeof(MmaArgs) * B, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_uargs, uargs.data(), sizeof(UpdateArgs) * B, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_ncta, ncta.data(), sizeof(int) * B, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_tmaps, tmaps.data(), sizeof(CUtensorMap) * B, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(b->d_head, 0, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(b->states, 0, sizeof(float) * 5 * B);
        if (e == cudaSuccess) e = cudaMemset(b->U_nom, 0, sizeof(float) * b->utotal);
        if (e == cudaSuccess) e = cudaMemset(b->U_new, 0, sizeof(float) * b->utotal);
        if (e == cudaSuccess) e = cudaMemset(b->weights, 0, sizeof(float) * b->wtotal);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_uitems, uitems.size() * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_uitems, uitems.data(), uitems.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_free(cuda_fail(e, "mppi_batch_create: upload"));
        b->nuitems = (int)uitems.size();
        if ((rc = build_items(b))) return fail_free(rc);
        *out = b;
        return GPMPPI_OK;
    } catch (...) {
        return fail(GPMPPI_ERR_CUDA, "mppi_batch_create: unexpected exception");
    }
}

int mppi_batch_buffers(gpmppi_batch b, int32_t i, float** state, float** U_nom, float** U_new,
                       float** weights, float** costs) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_buffers: invalid handle");
    if (i < 0 || i >= b->B) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_buffers: index out of range");
    if (state) *state = b->states + 5 * i;
    if (U_nom) *U_nom = b->U_nom + b->uoff[i];
    if (U_new) *U_new = b->U_new + b->uoff[i];
    if (weights) *weights = b->weights + b->woff[i];
    if (costs) *costs = b->ctrls[i]->costs;
    return GPMPPI_OK;
}

int mppi_batch_step(gpmppi_batch b, void* stream) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_step: invalid handle");
    int dev = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_step: batch belongs to another device");
    int rc;
    if ((rc = refresh_weights(b, (cudaStream_t)stream))) return rc;
    return enqueue_step(b, (cudaStream_t)stream);
}

int mppi_batch_graph(gpmppi_batch b, void* stream) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_graph: invalid handle");
    if (!stream) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_graph: graph replay needs a created stream");
    cudaStream_t st = (cudaStream_t)stream;
    int rc0;
    if ((rc0 = refresh_weights(b, st))) return rc0;
    if (!b->gexec) {
        GPM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        const int rc = enqueue_step(b, st);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "mppi_batch_graph: capture");
        b->graph = g;
        GPM_CUDA(cudaGraphInstantiate(&b->gexec, b->graph, 0));
    }
    GPM_CUDA(cudaGraphLaunch(b->gexec, st));
    return GPMPPI_OK;
}

int mppi_batch_autotune(gpmppi_batch b, void* stream, int32_t* chosen) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_autotune: invalid handle");
    cudaStream_t st = (cudaStream_t)stream;
    int nsm = 0;
    GPM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    cudaEvent_t e0, e1;
    GPM_CUDA(cudaEventCreate(&e0));
    GPM_CUDA(cudaEventCreate(&e1));
    // Per controller shape: one wave of its tiles timed for each tile layout
    // (tensor cores: 2, 4 or 8 producer threads per sample, i.e. 128, 64 or
    // 32 samples per tile; FP32: its one layout); the layout with the least
    // SM time (tiles x time per tile) is kept, and the time per tile orders
    // the work queue.  Only rollouts run (scratch outputs); no update, so the
    // iteration counters do not move.
    int rc = GPMPPI_OK, changed = 0;
    for (int i = 0; i < b->B && !rc; ++i) {
        gpmppi_ctrl c = b->ctrls[i];
        const ShapeKey key = shape_of(c);
        {
            std::lock_guard<std::mutex> lock(g_tuned_mu);
            auto hit = g_tuned.find(key);
            if (hit != g_tuned.end()) {
                if (c->fmt >= 0 && b->rps[i] != hit->second.first) ++changed;
                if (c->fmt >= 0) b->rps[i] = hit->second.first;
                b->tile_us[i] = hit->second.second;
                continue;
            }
        }
        int best_r = c->fmt < 0 ? 0 : b->rps[i];
        double best_cost = 1e300, best_us = b->tile_us[i];
        const int cand[3] = {2, 4, 8};
        for (int r : cand) {
            if (c->fmt < 0 && r != 2) break;            // FP32 tiles have one layout
            double us = 0.0;
            int tiles = 0;
            if ((rc = time_wave(b, i, r, nsm, st, e0, e1, &us, &tiles))) break;
            const double cost = us * tiles;              // SM-microseconds of the controller's tiles
            if (cost < best_cost) {
                best_cost = cost;
                best_us = us;
                best_r = c->fmt < 0 ? 0 : r;
            }
        }
        if (rc) break;
        if (c->fmt >= 0 && b->rps[i] != best_r) ++changed;
        if (c->fmt >= 0) b->rps[i] = best_r;
        b->tile_us[i] = best_us;
        std::lock_guard<std::mutex> lock(g_tuned_mu);
        g_tuned[key] = std::make_pair(best_r, best_us);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = build_items(b))) return rc;
    if (chosen) *chosen = changed;
    return GPMPPI_OK;
}

int mppi_batch_layout(gpmppi_batch b, int32_t i, int32_t* threads_per_sample, float* tile_us) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_layout: invalid handle");
    if (i < 0 || i >= b->B) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_layout: index out of range");
    if (threads_per_sample) *threads_per_sample = b->ctrls[i]->fmt < 0 ? 0 : b->rps[i];
    if (tile_us) *tile_us = (float)b->tile_us[i];
    return GPMPPI_OK;
}

int mppi_batch_get_iteration(gpmppi_batch b, int32_t i, uint64_t* it) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_get_iteration: invalid handle");
    if (i < 0 || i >= b->B || !it) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_get_iteration: bad argument");
    unsigned long long v = 0;
    GPM_CUDA(cudaMemcpy(&v, b->iters + i, sizeof(v), cudaMemcpyDeviceToHost));
    *it = v;
    return GPMPPI_OK;
}

int mppi_batch_destroy(gpmppi_batch b) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_destroy: invalid handle");
    cudaDeviceSynchronize();
    free_batch(b);
    return GPMPPI_OK;
}

}  // extern "C"
