// Batched MPPI iterations over many independent controllers.
//
// One iteration of every controller in the batch runs as (at most) two
// tensor-core rollout launches (one per 16-bit format) whose CTAs each take a
// (controller, sample tile) item, plus one launch of the weights/update for all
// controllers; controllers on the FP32 CUDA-core path are launched one after
// the other in between.  States, nominal controls, outputs and the Philox
// iteration counters live in device buffers owned by the batch, so the whole
// iteration can be captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
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
    if (c->ens) return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_batch_create: terrain ensembles are not batched");
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
    int2* d_items[2] = {nullptr, nullptr};
    int nitems[2] = {0, 0};
    int2* d_uitems = nullptr;
    int nuitems = 0;
    std::vector<RolloutArgs> h_args;
    std::vector<MmaArgs> h_mm;
    std::vector<int> fp32_ids;
    int rps = 2;
    int smem[2] = {0, 0};
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
    cudaFree(b->d_items[0]);
    cudaFree(b->d_items[1]);
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

// (controller, tile) items of the tensor-core controllers of one format,
// largest work first so that the long tiles start in the first wave
int build_items(gpmppi_batch b, int rps) {
    const int mtc = 256 / rps;
    for (int f = 0; f < 2; ++f) {
        std::vector<int> ids;
        for (int i = 0; i < b->B; ++i)
            if (b->ctrls[i]->fmt == f) ids.push_back(i);
        std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) {
            const double wx = (double)b->h_args[x].T * b->h_mm[x].nblocks * (b->h_mm[x].nblocks + 1);
            const double wy = (double)b->h_args[y].T * b->h_mm[y].nblocks * (b->h_mm[y].nblocks + 1);
            return wx > wy;
        });
        std::vector<int2> items;
        for (int i : ids) {
            const int tiles = (b->h_args[i].K + mtc - 1) / mtc;
            for (int t = 0; t < tiles; ++t) items.push_back(make_int2(i, t));
        }
        cudaFree(b->d_items[f]);
        b->d_items[f] = nullptr;
        b->nitems[f] = (int)items.size();
        if (!items.empty()) {
            GPM_CUDA(cudaMalloc(&b->d_items[f], items.size() * sizeof(int2)));
            GPM_CUDA(cudaMemcpy(b->d_items[f], items.data(), items.size() * sizeof(int2),
                                cudaMemcpyHostToDevice));
        }
    }
    b->rps = rps;
    drop_graph(b);
    return GPMPPI_OK;
}

int enqueue_step(gpmppi_batch b, cudaStream_t st) {
    int rc;
    for (int f = 0; f < 2; ++f)
        if ((rc = launch_rollout_mma_batched(b->d_args, b->d_mm, b->d_items[f], b->nitems[f], f, b->rps,
                                             b->smem[f], st)))
            return rc;
    for (int i : b->fp32_ids)
        if ((rc = launch_rollout_fp32(b->h_args[i], &b->ctrls[i]->tmW, false, st))) return rc;
    return launch_update_batched(b->d_uargs, b->d_uitems, b->d_ncta, b->iters, b->nuitems, b->maxT, st);
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
            (rc = alloc((void**)&b->d_ncta, sizeof(int) * B)))
            return fail_free(rc);
        std::vector<unsigned long long> its(B);
        std::vector<UpdateArgs> uargs(B);
        std::vector<int> ncta(B);
        std::vector<int2> uitems;
        b->h_args.resize(B);
        b->h_mm.resize(B);
        const float zero_state[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i < B; ++i) {
            gpmppi_ctrl c = ctrls[i];
            its[i] = c->it;
            RolloutArgs a = make_rollout_args(c, zero_state, b->U_nom + b->uoff[i]);
            a.x0_dev = b->states + 5 * i;
            a.it_dev = b->iters + i;
            a.costs = c->costs;
            b->h_args[i] = a;
            b->h_mm[i] = c->mm;
            if (c->fmt < 0) {
                b->fp32_ids.push_back(i);
            } else {
                b->smem[c->fmt] = std::max(b->smem[c->fmt], rollout_mma_smem(c->mm, c->S, c->O));
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
        if (e == cudaSuccess) e = cudaMemset(b->states, 0, sizeof(float) * 5 * B);
        if (e == cudaSuccess) e = cudaMemset(b->U_nom, 0, sizeof(float) * b->utotal);
        if (e == cudaSuccess) e = cudaMemset(b->U_new, 0, sizeof(float) * b->utotal);
        if (e == cudaSuccess) e = cudaMemset(b->weights, 0, sizeof(float) * b->wtotal);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_uitems, uitems.size() * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_uitems, uitems.data(), uitems.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail_free(cuda_fail(e, "mppi_batch_create: upload"));
        b->nuitems = (int)uitems.size();
        if ((rc = build_items(b, 2))) return fail_free(rc);
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
    return enqueue_step(b, (cudaStream_t)stream);
}

int mppi_batch_graph(gpmppi_batch b, void* stream) {
    if (!valid_batch(b)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_graph: invalid handle");
    if (!stream) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_batch_graph: graph replay needs a created stream");
    cudaStream_t st = (cudaStream_t)stream;
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
    if (b->nitems[0] + b->nitems[1] == 0) {
        if (chosen) *chosen = b->rps;
        return GPMPPI_OK;
    }
    // trial steps advance the iteration counters: keep and restore them
    std::vector<unsigned long long> saved(b->B);
    GPM_CUDA(cudaMemcpy(saved.data(), b->iters, sizeof(unsigned long long) * b->B, cudaMemcpyDeviceToHost));
    cudaEvent_t e0, e1;
    GPM_CUDA(cudaEventCreate(&e0));
    GPM_CUDA(cudaEventCreate(&e1));
    const int cand[3] = {2, 4, 8};
    float best_ms = 1e30f;
    int best = 2, rc = GPMPPI_OK;
    for (int r : cand) {
        if ((rc = build_items(b, r))) break;
        if ((rc = enqueue_step(b, st))) break;             // warm-up
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2 && !rc; ++rep) rc = enqueue_step(b, st);
        cudaEventRecord(e1, st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "mppi_batch_autotune");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = r;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    GPM_CUDA(cudaMemcpy(b->iters, saved.data(), sizeof(unsigned long long) * b->B, cudaMemcpyHostToDevice));
    if ((rc = build_items(b, best))) return rc;
    if (chosen) *chosen = best;
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
