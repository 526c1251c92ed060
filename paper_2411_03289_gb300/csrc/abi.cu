// Host implementation of the C ABI declared in include/gpmppi.h.
//
// Every entry point validates its arguments (shapes, finiteness, pointer
// kinds, handle tags) before touching the GPU, so that bad input becomes an
// error code instead of a device fault, and converts every CUDA error into a
// status code with a thread-local message.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "handles.cuh"

namespace gpm {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GPMPPI_ERR_OOM : GPMPPI_ERR_CUDA;
}

// Device (or managed) memory of the current device?
int check_dev_ptr(const void* p, const char* name, bool nullable) {
    if (p == nullptr) {
        if (nullable) return GPMPPI_OK;
        return fail(GPMPPI_ERR_INVALID_ARG, std::string(name) + " must not be NULL");
    }
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GPMPPI_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(GPMPPI_ERR_INVALID_ARG, std::string(name) + " must be device memory");
    int dev = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return fail(GPMPPI_ERR_INVALID_ARG, std::string(name) + " lives on another device");
    return GPMPPI_OK;
}

// A host array argument: not NULL unless nullable, and not device memory.
int check_host_ptr(const void* p, const char* name, bool nullable) {
    if (p == nullptr) {
        if (nullable) return GPMPPI_OK;
        return fail(GPMPPI_ERR_INVALID_ARG, std::string(name) + " must not be NULL");
    }
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GPMPPI_OK;                    // unknown to CUDA: ordinary host memory
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return fail(GPMPPI_ERR_INVALID_ARG, std::string(name) + " must be host memory");
    return GPMPPI_OK;
}

}  // namespace gpm

using namespace gpm;

namespace {

constexpr uint32_t kGpMagic = kGpMagicValue;
constexpr uint32_t kCtrlMagic = kCtrlMagicValue;
// training sets larger than this use the separate low column set of the
// streaming tensor-core rollout (MmaArgs::lo_set)
constexpr int kLoSetMinN = 768;

bool is_finite(double v) { return std::isfinite(v); }

// Quantile of a chi-squared variable with 2 degrees of freedom (Eq. 14):
// that distribution is exponential with mean 2, so chi2_2(p) = -2 ln(1 - p).
double chi2_2_quantile(double p) { return -2.0 * std::log1p(-p); }

// Standard normal quantile (Eq. 16) by bisection on the upper tail
// erfc(x / sqrt 2) / 2 = 1 - p (p > 1/2) or on Phi(x) = p.
double normal_quantile(double p) {
    double lo = -40.0, hi = 40.0;
    const double q = 1.0 - p;
    for (int i = 0; i < 400; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        const bool below = (p > 0.5) ? (0.5 * std::erfc(mid / std::sqrt(2.0)) > q)
                                     : (0.5 * std::erfc(-mid / std::sqrt(2.0)) < p);
        if (below) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

namespace {

void free_gp(gpmppi_gp h) {
    if (!h) return;
    GpDevice& g = h->g;
    cudaFree(g.alpha);
    cudaFree(g.Xs[0]);
    cudaFree(g.W[0]);
    cudaFree(g.Linv64[0]);
    cudaFree(g.alpha64[0]);
    cudaFree(g.alpha64[1]);
    for (int f = 0; f < 3; ++f) {
        cudaFree(g.mma_hi[f]);
        cudaFree(g.mma_lo[f]);
    }
    cudaFree(g.mma_mid);
    for (int f = 0; f < 2; ++f) cudaFree(g.cl_tiles[f]);
    cudaFree(g.cl_xa);
    cudaFree(g.mma_xa);
    cudaFree(g.Wt);
    cudaFree(g.ubar);
    if (!g.shared) {
        cudaFree(g.Xs[1]);
        cudaFree(g.W[1]);
        cudaFree(g.Linv64[1]);
    }
    h->magic = 0;
    delete h;
}

void free_ctrl(gpmppi_ctrl c) {
    if (!c) return;
    cudaFree(c->obst);
    cudaFree(c->seg);
    cudaFree(c->seg_il2);
    cudaFree(c->costs);
    cudaFree(c->hs_U);
    cudaFree(c->hs_w);
    cudaFree(c->ens_hi);
    cudaFree(c->ens_lo);
    cudaFree(c->ens_mid);
    cudaFree(c->ens_xa);
    cudaFree(c->u_tilde);
    cudaFree(c->partial);
    cudaFree(c->counter);
    cudaFree(c->nom_sxy);
    cudaFree(c->gcell);
    cudaFree(c->gidx);
    cudaFree(c->err);
    cudaFree(c->grad_scr);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->gp && c->gp->magic == kGpMagic) c->gp->g.n_controllers--;
    for (int i = 1; i < c->M; ++i)
        if (c->tgp[i] && c->tgp[i]->magic == kGpMagic) c->tgp[i]->g.n_controllers--;
    c->magic = 0;
    delete c;
}

bool valid_gp(gpmppi_gp h) { return h && h->magic == kGpMagic; }
bool valid_ctrl(gpmppi_ctrl c) { return c && c->magic == kCtrlMagic && valid_gp(c->gp); }

int validate_params(const gpmppi_params& p) {
    auto bad = [](const char* what) { return fail(GPMPPI_ERR_INVALID_ARG, std::string("params: ") + what); };
    if (p.K < 1 || p.K > GPMPPI_MAX_K) return bad("K out of range");
    if (p.T < 1 || p.T > GPMPPI_MAX_T) return bad("T out of range");
    const float fs[] = {p.dt, p.tau_v, p.tau_w, p.sigma[0], p.sigma[1], p.lambda, p.p_x,
                        p.u_min[0], p.u_min[1], p.u_max[0], p.u_max[1], p.alpha[0], p.alpha[1],
                        p.alpha[2], p.alpha[3], p.alpha[4], p.beta[0], p.beta[1], p.beta[2],
                        p.beta[3], p.P_lane, p.P_coll, p.lane_half_width, p.v_desired,
                        p.goal[0], p.goal[1], p.goal_radius, p.P_goal};
    for (float f : fs)
        if (!is_finite(f)) return fail(GPMPPI_ERR_NONFINITE, "params: non-finite value");
    if (!(p.dt > 0.0f) || !(p.tau_v > 0.0f) || !(p.tau_w > 0.0f)) return bad("dt, tau_v, tau_w must be > 0");
    if (p.sigma[0] < 0.0f || p.sigma[1] < 0.0f) return bad("sigma must be >= 0");
    if (!(p.lambda > 0.0f)) return bad("lambda must be > 0");
    if (!(p.p_x > 0.0f && p.p_x < 1.0f)) return bad("p_x must lie in (0, 1)");
    if (p.u_min[0] > p.u_max[0] || p.u_min[1] > p.u_max[1]) return bad("u_min > u_max");
    if (!(p.lane_half_width > 0.0f)) return bad("lane_half_width must be > 0");
    if (p.alpha[2] != 0.0f)
        return fail(GPMPPI_ERR_UNSUPPORTED, "params: the slip term (alpha[2]) is not modelled");
    if (p.goal_radius < 0.0f) return bad("goal_radius must be >= 0");
    if (p.variance_mode != GPMPPI_VAR_PER_SAMPLE && p.variance_mode != GPMPPI_VAR_NOMINAL)
        return bad("unknown variance_mode");
    if (p.precision != GPMPPI_FP32 && p.precision != GPMPPI_BF16_SPLIT && p.precision != GPMPPI_FP16_SPLIT &&
        p.precision != GPMPPI_BF16_SPLIT3)
        return bad("unknown precision");
    return GPMPPI_OK;
}

int current_device(int* dev) {
    GPM_CUDA(cudaGetDevice(dev));
    return GPMPPI_OK;
}

int check_state(const float* state) {
    if (!state) return fail(GPMPPI_ERR_INVALID_ARG, "state must not be NULL");
    for (int i = 0; i < 5; ++i)
        if (!std::isfinite(state[i])) return fail(GPMPPI_ERR_NONFINITE, "state: non-finite value");
    return GPMPPI_OK;
}

}  // namespace

RolloutArgs gpm::make_rollout_args(gpmppi_ctrl c, const float* state, const float* U) {
    const gpmppi_params& p = c->p;
    const GpDevice& g = c->gp->g;
    RolloutArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Xs = g.Xs[0];
    a.alpha = g.alpha;
    a.W = g.W[0];
    a.obst = c->obst;
    a.seg = c->seg;
    a.seg_il2 = c->seg_il2;
    a.U = U;
    a.nom_sxy = (p.variance_mode == GPMPPI_VAR_NOMINAL) ? c->nom_sxy : nullptr;
    a.costs = c->costs;
    a.u_tilde = c->u_tilde;
    a.K = p.K;
    a.T = p.T;
    a.N = g.N;
    a.Np = g.Np;
    a.O = c->O;
    a.S = c->S;
    a.mt = c->mt;
    a.stages = c->stages;
    a.err = c->err;
    a.wait_ns = c->wait_ns;
    a.expire_first = c->expire_first;
    a.sf2 = g.sf2[0];
    for (int i = 0; i < 5; ++i) a.x0[i] = state[i];
    for (int d = 0; d < 4; ++d) a.zscale[d] = g.zscale[0][d];
    a.dt = p.dt;
    a.kv = (float)((double)p.dt / p.tau_v);
    a.kw = (float)((double)p.dt / p.tau_w);
    a.av = (float)(1.0 - (double)p.dt / p.tau_v);
    a.aw = (float)(1.0 - (double)p.dt / p.tau_w);
    a.sig_v = p.sigma[0];
    a.sig_w = p.sigma[1];
    a.umin0 = p.u_min[0];
    a.umin1 = p.u_min[1];
    a.umax0 = p.u_max[0];
    a.umax1 = p.u_max[1];
    a.c_var = p.alpha[0] + p.beta[0];
    a.c_dev = (float)((double)p.alpha[1] / p.lane_half_width);
    a.c_lane = p.alpha[3] * p.P_lane;
    a.c_speed = p.alpha[4];
    a.c_coll = p.beta[1] * p.P_coll;
    a.r = p.lane_half_width;
    a.v_des = p.v_desired;
    a.sq_chi2 = (float)c->sq_chi2;
    a.phi_inv = (float)c->phi_inv;
    a.gcell = c->gcell;
    a.gidx = c->gidx;
    a.gx0 = c->gx0;
    a.gy0 = c->gy0;
    a.ginv = c->ginv;
    a.gnx = c->gnx;
    a.gny = c->gny;
    a.c_goal = p.beta[2];
    a.c_term = (float)((double)p.beta[3] * p.P_goal);
    a.goal_x = p.goal[0];
    a.goal_y = p.goal[1];
    a.goal_r = p.goal_radius;
    a.key0 = (uint32_t)p.seed;
    a.key1 = (uint32_t)(p.seed >> 32);
    a.it0 = (uint32_t)c->it;
    a.it1 = (uint32_t)(c->it >> 32);
    return a;
}

namespace {

// Launch arguments of the ensemble rollout: the single-GP arguments plus the
// per-terrain factors and weights.
EnsArgs make_ens_args(gpmppi_ctrl c, const RolloutArgs& a) {
    EnsArgs e;
    std::memset(&e, 0, sizeof(e));
    e.r = a;
    e.M = c->M;
    e.Npmax = 0;
    for (int i = 0; i < c->M; ++i) {
        const GpDevice& g = c->tgp[i]->g;
        TerrainGp& t = e.gp[i];
        t.Xs = g.Xs[0];
        t.alpha = g.alpha;
        t.W = g.W[0];
        t.N = g.N;
        t.Np = g.Np;
        t.sf2 = g.sf2[0];
        for (int d = 0; d < 4; ++d) t.zscale[d] = g.zscale[0][d];
        t.w = c->tw[i];
        if (g.Np > e.Npmax) e.Npmax = g.Np;
    }
    return e;
}

int check_ctrl_device(gpmppi_ctrl c) {
    int dev = 0;
    int rc = current_device(&dev);
    if (rc) return rc;
    if (dev != c->device) return fail(GPMPPI_ERR_INVALID_ARG, "controller belongs to another device");
    return GPMPPI_OK;
}

}  // namespace

extern "C" {

const char* gpmppi_last_error(void) { return g_err.c_str(); }

int gpmppi_version(void) { return 100; }

int gp_fit(const double* X, const double* Y, int32_t N, const gpmppi_hyper hyper[2], gpmppi_gp* out) {
    try {
        if (!out) return fail(GPMPPI_ERR_INVALID_ARG, "gp_fit: out must not be NULL");
        *out = nullptr;
        if (!hyper) return fail(GPMPPI_ERR_INVALID_ARG, "gp_fit: hyper must not be NULL");
        if (N < 0 || N > GPMPPI_MAX_N) return fail(GPMPPI_ERR_INVALID_ARG, "gp_fit: N out of range");
        if (N > 0 && (!X || !Y)) return fail(GPMPPI_ERR_INVALID_ARG, "gp_fit: X and Y must not be NULL");
        for (int i = 0; i < 4 * N; ++i)
            if (!is_finite(X[i])) return fail(GPMPPI_ERR_NONFINITE, "gp_fit: non-finite X");
        for (int i = 0; i < 2 * N; ++i)
            if (!is_finite(Y[i])) return fail(GPMPPI_ERR_NONFINITE, "gp_fit: non-finite Y");
        for (int o = 0; o < 2; ++o) {
            const gpmppi_hyper& h = hyper[o];
            for (int d = 0; d < 4; ++d)
                if (!is_finite(h.lengthscale[d]) || !(h.lengthscale[d] > 0.0))
                    return fail(GPMPPI_ERR_INVALID_ARG, "gp_fit: lengthscales must be finite and > 0");
            if (!is_finite(h.signal_var) || !(h.signal_var > 0.0))
                return fail(GPMPPI_ERR_INVALID_ARG, "gp_fit: signal_var must be finite and > 0");
            if (!is_finite(h.noise_var) || h.noise_var < 0.0)
                return fail(GPMPPI_ERR_INVALID_ARG, "gp_fit: noise_var must be finite and >= 0");
        }
        gpmppi_gp h = new (std::nothrow) gpmppi_gp_s;
        if (!h) return fail(GPMPPI_ERR_OOM, "gp_fit: host allocation failed");
        h->g.hyper[0] = hyper[0];
        h->g.hyper[1] = hyper[1];
        h->g.shared = std::memcmp(hyper[0].lengthscale, hyper[1].lengthscale, sizeof(double) * 4) == 0 &&
                      hyper[0].signal_var == hyper[1].signal_var &&
                      hyper[0].noise_var == hyper[1].noise_var;
        int rc = current_device(&h->g.device);
        if (rc) {
            delete h;
            return rc;
        }
        cudaStream_t st = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(e, "gp_fit: stream");
        }
        rc = gp_fit_device(h->g, X, Y, N, st);
        cudaStreamDestroy(st);
        if (rc) {
            free_gp(h);
            return rc;
        }
        *out = h;
        return GPMPPI_OK;
    } catch (...) {
        return fail(GPMPPI_ERR_CUDA, "gp_fit: unexpected exception");
    }
}

int gp_destroy(gpmppi_gp gp) {
    if (!valid_gp(gp)) return fail(GPMPPI_ERR_INVALID_ARG, "gp_destroy: invalid handle");
    if (gp->g.n_controllers > 0)
        return fail(GPMPPI_ERR_INVALID_ARG, "gp_destroy: controllers still use this GP");
    free_gp(gp);
    return GPMPPI_OK;
}

int gp_factors(gpmppi_gp gp, int32_t j, double* Linv, double* alpha) {
    if (!valid_gp(gp)) return fail(GPMPPI_ERR_INVALID_ARG, "gp_factors: invalid handle");
    if (j != 0 && j != 1) return fail(GPMPPI_ERR_INVALID_ARG, "gp_factors: output must be 0 or 1");
    const int N = gp->g.N;
    if (N == 0) return GPMPPI_OK;
    if (Linv)
        GPM_CUDA(cudaMemcpy(Linv, gp->g.Linv64[j], sizeof(double) * (size_t)N * N, cudaMemcpyDeviceToHost));
    if (alpha) GPM_CUDA(cudaMemcpy(alpha, gp->g.alpha64[j], sizeof(double) * N, cudaMemcpyDeviceToHost));
    return GPMPPI_OK;
}

int gp_predict(gpmppi_gp gp, const float* Z, int32_t M, float* mean, float* var, void* stream) {
    if (!valid_gp(gp)) return fail(GPMPPI_ERR_INVALID_ARG, "gp_predict: invalid handle");
    if (M < 0) return fail(GPMPPI_ERR_INVALID_ARG, "gp_predict: M must be >= 0");
    if (M == 0) return GPMPPI_OK;
    int rc;
    if ((rc = check_dev_ptr(Z, "gp_predict: Z", false))) return rc;
    if ((rc = check_dev_ptr(mean, "gp_predict: mean", false))) return rc;
    if ((rc = check_dev_ptr(var, "gp_predict: var", false))) return rc;
    return launch_gp_predict(gp->g, Z, M, mean, var, (cudaStream_t)stream);
}

int mppi_create(const gpmppi_params* p, const float* obstacles, int32_t O, const float* path,
                int32_t P, gpmppi_gp gp, gpmppi_ctrl* out) {
    try {
        if (!out) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: out must not be NULL");
        *out = nullptr;
        if (!p) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: params must not be NULL");
        if (!valid_gp(gp)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: invalid GP handle");
        int rc = validate_params(*p);
        if (rc) return rc;
        if (!gp->g.shared)
            return fail(GPMPPI_ERR_UNSUPPORTED,
                        "mppi_create: the two GP outputs must share hyper-parameters");
        if (O < 0 || O > GPMPPI_MAX_OBSTACLES) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: O out of range");
        if (O > 0 && !obstacles) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: obstacles is NULL");
        if (P < 1 || P > GPMPPI_MAX_PATH) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: P out of range");
        if (!path) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: path is NULL");
        for (int i = 0; i < 3 * O; ++i)
            if (!is_finite(obstacles[i])) return fail(GPMPPI_ERR_NONFINITE, "mppi_create: non-finite obstacle");
        for (int i = 0; i < O; ++i)
            if (!(obstacles[3 * i + 2] > 0.0f)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: radius <= 0");
        for (int i = 0; i < 2 * P; ++i)
            if (!is_finite(path[i])) return fail(GPMPPI_ERR_NONFINITE, "mppi_create: non-finite path");
        int dev = 0;
        if ((rc = current_device(&dev))) return rc;
        if (dev != gp->g.device) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create: GP lives on another device");

        // launch geometry
        const int mtp = rollout_fp32_mtp(gp->g.Np);
        int nsm = 0, smem_optin = 0;
        GPM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        GPM_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        // the rollout layouts leave 64 bytes for the batched persistent kernel's
        // own words past the largest layout
        const int layout_limit = smem_optin - 64;
        const int stages = rollout_fp32_stages(gp->g.Np, layout_limit);
        if (stages == 0) return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_create: GP too large for shared memory");

        gpmppi_ctrl c = new (std::nothrow) gpmppi_ctrl_s;
        if (!c) return fail(GPMPPI_ERR_OOM, "mppi_create: host allocation failed");
        c->p = *p;
        c->gp = gp;
        c->device = dev;
        c->O = O;
        c->P = P;
        c->stages = stages;
        std::memset(&c->tmW, 0, sizeof(c->tmW));
        c->S = (P > 1) ? (P - 1) : 1;
        int mt = (p->K + nsm - 1) / nsm;
        if (const char* env = std::getenv("GPMPPI_SAMPLES_PER_CTA")) mt = std::atoi(env);
        c->mt = mt < 1 ? 1 : (mt > mtp ? mtp : mt);
        c->n_upd = (p->K + 255) / 256;
        c->sq_chi2 = std::sqrt(chi2_2_quantile(p->p_x));
        c->phi_inv = normal_quantile(p->p_x);
        gp->g.n_controllers++;

        std::vector<float4> seg(c->S);
        std::vector<float> il2(c->S);
        if (P == 1) {
            seg[0] = make_float4(path[0], path[1], 0.0f, 0.0f);
            il2[0] = 0.0f;
        } else {
            for (int i = 0; i < P - 1; ++i) {
                const double ax = path[2 * i], ay = path[2 * i + 1];
                const double dx = (double)path[2 * i + 2] - ax, dy = (double)path[2 * i + 3] - ay;
                const double l2 = dx * dx + dy * dy;
                seg[i] = make_float4((float)ax, (float)ay, (float)dx, (float)dy);
                il2[i] = l2 > 0.0 ? (float)(1.0 / l2) : 0.0f;
            }
        }
        const size_t K = (size_t)p->K, T = (size_t)p->T;
        auto alloc = [&](void** ptr, size_t bytes) -> int {
            cudaError_t e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
            if (e != cudaSuccess) return cuda_fail(e, "mppi_create: cudaMalloc");
            return GPMPPI_OK;
        };
        if ((rc = alloc((void**)&c->obst, sizeof(float) * 3 * O)) ||
            (rc = alloc((void**)&c->seg, sizeof(float4) * c->S)) ||
            (rc = alloc((void**)&c->seg_il2, sizeof(float) * c->S)) ||
            (rc = alloc((void**)&c->costs, sizeof(float) * K)) ||
            (rc = alloc((void**)&c->u_tilde, sizeof(float2) * K * T)) ||
            (rc = alloc((void**)&c->partial, sizeof(float) * 2 * (T + 1) * c->n_upd)) ||
            (rc = alloc((void**)&c->counter, sizeof(unsigned int))) ||
            (rc = alloc((void**)&c->nom_sxy, sizeof(float) * 3 * T)) ||
            (rc = alloc((void**)&c->err, sizeof(unsigned int)))) {
            free_ctrl(c);
            return rc;
        }
        cudaError_t e = cudaSuccess;
        if (O > 0 && e == cudaSuccess)
            e = cudaMemcpy(c->obst, obstacles, sizeof(float) * 3 * O, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->seg, seg.data(), sizeof(float4) * c->S, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->seg_il2, il2.data(), sizeof(float) * c->S, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(c->counter, 0, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(c->nom_sxy, 0, sizeof(float) * 3 * T);
        if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            free_ctrl(c);
            return cuda_fail(e, "mppi_create: upload");
        }
        {
            // candidate segments per cell of a grid over the path (exact nearest-segment search)
            LaneGridHost lg;
            if ((rc = build_lane_grid(path, P, lg))) {
                free_ctrl(c);
                return rc;
            }
            if (!lg.cells.empty()) {
                cudaError_t e2 = cudaMalloc(&c->gcell, sizeof(int2) * lg.cells.size());
                if (e2 == cudaSuccess) e2 = cudaMalloc(&c->gidx, sizeof(int) * (lg.idx.empty() ? 1 : lg.idx.size()));
                if (e2 == cudaSuccess)
                    e2 = cudaMemcpy(c->gcell, lg.cells.data(), sizeof(int2) * lg.cells.size(), cudaMemcpyHostToDevice);
                if (e2 == cudaSuccess && !lg.idx.empty())
                    e2 = cudaMemcpy(c->gidx, lg.idx.data(), sizeof(int) * lg.idx.size(), cudaMemcpyHostToDevice);
                if (e2 != cudaSuccess) {
                    free_ctrl(c);
                    return cuda_fail(e2, "mppi_create: lane grid");
                }
                c->gx0 = lg.x0;
                c->gy0 = lg.y0;
                c->ginv = lg.inv_h;
                c->gnx = lg.nx;
                c->gny = lg.ny;
            }
        }
        if (gp->g.Np > 0 && (rc = make_w_tensor_map(&c->tmW, gp->g.W[0], gp->g.Np))) {
            free_ctrl(c);
            return rc;
        }
        if (p->precision != GPMPPI_FP32) {
            c->fmt = (p->precision == GPMPPI_FP16_SPLIT) ? 0 : (p->precision == GPMPPI_BF16_SPLIT ? 1 : 2);
            if ((rc = build_mma_tiles(gp->g, c->fmt))) {
                free_ctrl(c);
                return rc;
            }
            const GpDevice& g = gp->g;
            c->mm.Bhi = g.mma_hi[c->fmt];
            c->mm.Blo = g.mma_lo[c->fmt];
            c->mm.Bmid = c->fmt == 2 ? g.mma_mid : nullptr;
            c->mm.parts = c->fmt == 2 ? 3 : 2;
            c->mm.xa = g.mma_xa;
            c->mm.nblocks = g.NpM / 128;
            const double r = (double)g.sf2[0] / (g.mma_cB > 0.0f ? (double)g.mma_cB : 1.0);
            // the single GP: one terrain of weight 1 over every block
            MmaTerrains& tr = c->mm.tr;
            tr = MmaTerrains{};
            tr.M = 1;
            tr.blk0[0] = 0;
            tr.blk0[1] = c->mm.nblocks;
            tr.qscale[0] = (float)(r * r);
            tr.sf2[0] = g.sf2[0];
            tr.w[0] = 1.0f;
            for (int d = 0; d < 4; ++d) tr.zscale[0][d] = g.zscale[0][d];
            c->mm.scene_smem = 1;
            // The tensor core rounds its FP32 accumulator at every MMA, so the
            // variance error grows with the MMAs per output column (3 N / 16
            // with all split products in one column set).  Beyond 768 points
            // the two small products get their own column set (N / 16 MMAs on
            // the large accumulator), which keeps the variance error near
            // 1e-5 sf2 at N = 2048 at the cost of output passes half as wide.
            // The three-term BF16 split always keeps its five small products
            // apart (its stages would not fit shared memory with 512-column
            // passes).
            c->mm.lo_set = (g.N > kLoSetMinN || c->fmt == 2) ? 1 : 0;
            c->mm.stages = rollout_mma_stages(g.NpM, c->S, O, layout_limit, c->mm.lo_set, c->mm.parts, 1);
            if (c->mm.stages < 3) {
                // keep the pipeline deep; read the scene from global memory instead
                const int st_noscene = rollout_mma_stages(g.NpM, 0, 0, layout_limit, c->mm.lo_set, c->mm.parts, 1);
                if (st_noscene > c->mm.stages) {
                    c->mm.stages = st_noscene;
                    c->mm.scene_smem = 0;
                }
            }
            // fewest threads per sample (largest sample tile) that still
            // gives every SM a CTA; small K falls back to 32 samples per CTA
            c->mm.rps = 8;
            if ((p->K + 127) / 128 >= nsm * 4 / 5) c->mm.rps = 2;
            else if ((p->K + 63) / 64 >= nsm * 4 / 5) c->mm.rps = 4;
            if (const char* env = std::getenv("GPMPPI_MMA_THREADS_PER_SAMPLE")) c->mm.rps = std::atoi(env);
            if (c->mm.stages == 0) {
                free_ctrl(c);
                return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_create: tensor-core rollout does not fit shared memory");
            }
            // N <= 512: the cluster rollout keeps the factor resident in shared
            // memory (two-part formats only)
            const char* no_cl = std::getenv("GPMPPI_NO_CLUSTER");
            if (c->fmt < 2 && g.N > 0 && g.N <= 512 && !(no_cl && no_cl[0] == '1')) {
                if ((rc = build_cl_tiles(gp->g, c->fmt))) {
                    free_ctrl(c);
                    return rc;
                }
                ClArgs& cl = c->cla;
                cl.tiles = gp->g.cl_tiles[c->fmt];
                cl.npc = gp->g.cl_npc;
                cl.xa = gp->g.cl_xa;
                cl.ns = cl.npc / 64;
                cl.cs = cl.ns / 2;
                for (int r = 0; r < 4; ++r) {
                    cl.base[r] = gp->g.cl_base[r];
                    cl.bytes[r] = gp->g.cl_bytes[r];
                }
                cl.qscale = c->mm.tr.qscale[0];
                cl.scene_smem = 1;
                if (cl_smem_bytes(cl, c->S, O) > smem_optin) cl.scene_smem = 0;
                c->cl = cl_smem_bytes(cl, c->S, O) <= smem_optin && cl_schedulable(cl, c->S, O, dev);
            }
        }
        *out = c;
        return GPMPPI_OK;
    } catch (...) {
        return fail(GPMPPI_ERR_CUDA, "mppi_create: unexpected exception");
    }
}

int mppi_step(gpmppi_ctrl c, const float state[5], const float* U_nom, float* U_new,
              float* weights, float* costs, void* stream) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_step: invalid handle");
    int rc;
    if ((rc = check_ctrl_device(c))) return rc;
    if ((rc = check_state(state))) return rc;
    if ((rc = check_dev_ptr(U_nom, "mppi_step: U_nom", false))) return rc;
    if ((rc = check_dev_ptr(U_new, "mppi_step: U_new", false))) return rc;
    if ((rc = check_dev_ptr(weights, "mppi_step: weights", true))) return rc;
    if ((rc = check_dev_ptr(costs, "mppi_step: costs", true))) return rc;
    if (U_nom == U_new) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_step: U_new must not alias U_nom");
    cudaStream_t st = (cudaStream_t)stream;
    RolloutArgs a = make_rollout_args(c, state, U_nom);
    if (costs) a.costs = costs;
    if (c->profiling) GPM_CUDA(cudaEventRecord(c->ev[0], st));
    if (c->ens && c->fmt < 0)
        rc = launch_rollout_ens(make_ens_args(c, a), false, st);
    else if (c->cl)
        rc = launch_rollout_cl(a, c->cla, c->fmt, false, st);
    else
        rc = (c->fmt < 0) ? launch_rollout_fp32(a, &c->tmW, false, st)
                          : launch_rollout_mma(a, c->mm, c->fmt, false, st);
    if (rc) return rc;
    if (c->profiling) GPM_CUDA(cudaEventRecord(c->ev[1], st));
    UpdateArgs u;
    u.costs = a.costs;
    u.u_tilde = c->u_tilde;
    u.U = U_nom;
    u.U_new = U_new;
    u.weights = weights;
    u.partial = c->partial;
    u.counter = c->counter;
    u.K = c->p.K;
    u.T = c->p.T;
    u.per_cta = 256;
    u.inv_lambda = 1.0f / c->p.lambda;
    if ((rc = launch_update(u, c->n_upd, st, !c->profiling))) return rc;
    if (c->p.variance_mode == GPMPPI_VAR_NOMINAL) {
        RolloutArgs n = make_rollout_args(c, state, U_new);
        if ((rc = launch_nominal(n, c->nom_sxy, st))) return rc;
    }
    if (c->profiling) {
        GPM_CUDA(cudaEventRecord(c->ev[2], st));
        c->profiled = true;
    }
    c->it++;
    return GPMPPI_OK;
}

int mppi_step_host(gpmppi_ctrl c, const float state[5], const float* U_nom, float* U_new, float* weights,
                   float* costs, void* stream) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_step_host: invalid handle");
    int rc;
    if ((rc = check_ctrl_device(c))) return rc;
    if ((rc = check_state(state))) return rc;
    if ((rc = check_host_ptr(U_nom, "mppi_step_host: U_nom", false))) return rc;
    if ((rc = check_host_ptr(U_new, "mppi_step_host: U_new", false))) return rc;
    if ((rc = check_host_ptr(weights, "mppi_step_host: weights", true))) return rc;
    if ((rc = check_host_ptr(costs, "mppi_step_host: costs", true))) return rc;
    const size_t ub = sizeof(float) * 2 * (size_t)c->p.T, kb = sizeof(float) * (size_t)c->p.K;
    if (!c->hs_U) GPM_CUDA(cudaMalloc(&c->hs_U, 2 * ub));
    if (weights && !c->hs_w) GPM_CUDA(cudaMalloc(&c->hs_w, kb));
    cudaStream_t st = (cudaStream_t)stream;
    float* d_nom = c->hs_U;
    float* d_new = c->hs_U + 2 * (size_t)c->p.T;
    // every exit waits for the copies it enqueued: the caller's host buffers
    // may be released as soon as the call returns
    cudaError_t e = cudaMemcpyAsync(d_nom, U_nom, ub, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "mppi_step_host: copy in");
    rc = mppi_step(c, state, d_nom, d_new, weights ? c->hs_w : nullptr, nullptr, st);
    if (!rc) e = cudaMemcpyAsync(U_new, d_new, ub, cudaMemcpyDeviceToHost, st);
    if (!rc && e == cudaSuccess && weights) e = cudaMemcpyAsync(weights, c->hs_w, kb, cudaMemcpyDeviceToHost, st);
    if (!rc && e == cudaSuccess && costs) e = cudaMemcpyAsync(costs, c->costs, kb, cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "mppi_step_host: copy out");
    if (es != cudaSuccess) return cuda_fail(es, "mppi_step_host: synchronise");
    return GPMPPI_OK;
}

int mppi_rollout_trace(gpmppi_ctrl c, const float state[5], const float* U_nom, float* mu,
                       float* sigma, float* stage, float* margins, float* costs, void* stream) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_rollout_trace: invalid handle");
    int rc;
    if ((rc = check_ctrl_device(c))) return rc;
    if ((rc = check_state(state))) return rc;
    if ((rc = check_dev_ptr(U_nom, "mppi_rollout_trace: U_nom", false))) return rc;
    if ((rc = check_dev_ptr(mu, "mppi_rollout_trace: mu", true))) return rc;
    if ((rc = check_dev_ptr(sigma, "mppi_rollout_trace: sigma", true))) return rc;
    if ((rc = check_dev_ptr(stage, "mppi_rollout_trace: stage", true))) return rc;
    if ((rc = check_dev_ptr(margins, "mppi_rollout_trace: margins", true))) return rc;
    if ((rc = check_dev_ptr(costs, "mppi_rollout_trace: costs", true))) return rc;
    RolloutArgs a = make_rollout_args(c, state, U_nom);
    if (costs) a.costs = costs;
    a.tr_mu = mu;
    a.tr_sig = sigma;
    a.tr_stage = stage;
    a.tr_margin = margins;
    if (c->ens && c->fmt < 0) return launch_rollout_ens(make_ens_args(c, a), true, (cudaStream_t)stream);
    if (c->cl) return launch_rollout_cl(a, c->cla, c->fmt, true, (cudaStream_t)stream);
    if (c->fmt >= 0) return launch_rollout_mma(a, c->mm, c->fmt, true, (cudaStream_t)stream);
    return launch_rollout_fp32(a, &c->tmW, true, (cudaStream_t)stream);
}

int mppi_create_ensemble(const gpmppi_params* p, const float* obstacles, int32_t O, const float* path,
                         int32_t P, const gpmppi_gp* gps, int32_t M, const float* weights,
                         gpmppi_ctrl* out) {
    if (!out) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create_ensemble: out must not be NULL");
    *out = nullptr;
    if (!gps || !weights) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create_ensemble: gps / weights is NULL");
    if (M < 1 || M > kMaxTerrains) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create_ensemble: M out of range");
    if (!p) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create_ensemble: params must not be NULL");
    for (int i = 0; i < M; ++i) {
        if (!valid_gp(gps[i])) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create_ensemble: invalid GP handle");
        if (!gps[i]->g.shared)
            return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_create_ensemble: each terrain's outputs must share hyper-parameters");
        if (gps[i]->g.device != gps[0]->g.device)
            return fail(GPMPPI_ERR_INVALID_ARG, "mppi_create_ensemble: GPs on different devices");
        if (!is_finite(weights[i])) return fail(GPMPPI_ERR_NONFINITE, "mppi_create_ensemble: non-finite weight");
    }
    // M = 1 with weight 1 is the single-GP controller (any precision);
    // everything else runs an ensemble rollout: the FP32 one, or in the split
    // precisions the streaming tensor-core rollout over the GPs' stacked factors
    const bool ens = M > 1 || weights[0] != 1.0f;
    if (ens && p->variance_mode != GPMPPI_VAR_PER_SAMPLE)
        return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_create_ensemble: needs the per-sample variance mode");
    int npmax = 0, optin = 0, dev = 0, rc;
    for (int i = 0; i < M; ++i) npmax = gps[i]->g.Np > npmax ? gps[i]->g.Np : npmax;
    if ((rc = current_device(&dev))) return rc;
    GPM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (ens && p->precision == GPMPPI_FP32 && ens_smem_bytes(npmax) > optin)
        return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_create_ensemble: GPs too large for the ensemble rollout");
    gpmppi_ctrl c = nullptr;
    if ((rc = mppi_create(p, obstacles, O, path, P, gps[0], &c))) return rc;
    c->M = M;
    c->ens = ens;
    for (int i = 0; i < M; ++i) {
        c->tgp[i] = gps[i];
        c->tw[i] = weights[i];
        if (i > 0) gps[i]->g.n_controllers++;
    }
    if (ens && c->fmt >= 0) {
        // the streaming rollout over the stacked factors (not the cluster kernel)
        GpDevice* gd[kMaxTerrains];
        bool lo = c->fmt == 2;
        for (int i = 0; i < M; ++i) {
            gd[i] = &gps[i]->g;
            lo = lo || gps[i]->g.N > kLoSetMinN;
        }
        MmaArgs& mm = c->mm;
        if ((rc = build_mma_ensemble(gd, M, c->fmt, mm.tr, &c->ens_hi, &c->ens_lo, &c->ens_mid, &c->ens_xa))) {
            mppi_destroy(c);
            return rc;
        }
        for (int i = 0; i < M; ++i) mm.tr.w[i] = weights[i];
        mm.Bhi = c->ens_hi;
        mm.Blo = c->ens_lo;
        mm.Bmid = c->ens_mid;
        mm.xa = c->ens_xa;
        mm.nblocks = mm.tr.blk0[M];
        mm.lo_set = lo ? 1 : 0;
        mm.scene_smem = 1;
        const int NpT = mm.nblocks * 128;
        mm.stages = rollout_mma_stages(NpT, c->S, O, optin - 64, mm.lo_set, mm.parts, M);
        if (mm.stages < 3) {
            const int st_noscene = rollout_mma_stages(NpT, 0, 0, optin - 64, mm.lo_set, mm.parts, M);
            if (st_noscene > mm.stages) {
                mm.stages = st_noscene;
                mm.scene_smem = 0;
            }
        }
        c->cl = false;
        if (mm.stages == 0) {
            mppi_destroy(c);
            return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_create_ensemble: the GPs' training sets do not fit shared memory");
        }
    }
    *out = c;
    return GPMPPI_OK;
}

int mppi_set_terrain_weights(gpmppi_ctrl c, const float* weights, int32_t M) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_set_terrain_weights: invalid handle");
    if (!weights || M != c->M) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_set_terrain_weights: M differs from the controller's");
    for (int i = 0; i < M; ++i)
        if (!is_finite(weights[i])) return fail(GPMPPI_ERR_NONFINITE, "mppi_set_terrain_weights: non-finite weight");
    if (!c->ens && weights[0] != 1.0f)
        return fail(GPMPPI_ERR_UNSUPPORTED,
                    "mppi_set_terrain_weights: a single-GP controller keeps weight 1 (create it with weight != 1)");
    for (int i = 0; i < M; ++i) c->tw[i] = weights[i];
    if (c->ens && c->fmt >= 0)
        for (int i = 0; i < M; ++i) c->mm.tr.w[i] = weights[i];
    return GPMPPI_OK;
}

int mppi_grad(gpmppi_ctrl c, const float state[5], const float* U_nom, const float* sample_weights,
              float slope, float* J, float* dU, float* dlengthscale, void* stream) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_grad: invalid handle");
    int rc;
    if ((rc = check_ctrl_device(c))) return rc;
    if ((rc = check_state(state))) return rc;
    if ((rc = check_dev_ptr(U_nom, "mppi_grad: U_nom", false))) return rc;
    if ((rc = check_dev_ptr(sample_weights, "mppi_grad: sample_weights", true))) return rc;
    if ((rc = check_dev_ptr(J, "mppi_grad: J", false))) return rc;
    if ((rc = check_dev_ptr(dU, "mppi_grad: dU", true))) return rc;
    if ((rc = check_dev_ptr(dlengthscale, "mppi_grad: dlengthscale", true))) return rc;
    if (!(slope > 0.0f) || !is_finite(slope)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_grad: slope must be > 0");
    if (dlengthscale && !dU)
        return fail(GPMPPI_ERR_INVALID_ARG, "mppi_grad: dlengthscale needs dU");
    if (c->p.variance_mode != GPMPPI_VAR_PER_SAMPLE)
        return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_grad: needs the per-sample variance mode");
    if (c->ens) return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_grad: terrain ensembles are not differentiated");
    GpDevice& g = c->gp->g;
    const int K = c->p.K, T = c->p.T, Np = g.Np, N = g.N;
    int C = (int)std::ceil(std::sqrt((double)T));
    if (C < 1) C = 1;
    const int nseg = (T + C - 1) / C;
    const int gm = grad_samples_per_cta();
    const int ncta = (K + gm - 1) / gm;
    const int Kpad = ncta * gm;
    int optin = 0;
    GPM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (grad_smem_bytes(Np, C) > optin)
        return fail(GPMPPI_ERR_UNSUPPORTED, "mppi_grad: GP too large for the adjoint kernel's shared memory");
    cudaStream_t st = (cudaStream_t)stream;
    const bool want_l = dlengthscale != nullptr;
    // per-GP factors of the adjoint, built once
    if (!g.Wt) {
        GPM_CUDA(cudaMalloc(&g.Wt, sizeof(float) * (size_t)Np * Np));
        if ((rc = launch_transpose(g.W[0], Np, g.Wt, st))) return rc;
        GPM_CUDA(cudaStreamSynchronize(st));
    }
    if (want_l && !g.ubar) {
        GPM_CUDA(cudaMalloc(&g.ubar, sizeof(float) * 8 * (size_t)Np));
        if ((rc = launch_dk_alpha(g.Xs[0], g.alpha, N, Np, g.sf2[0], g.ubar, st))) return rc;
        GPM_CUDA(cudaStreamSynchronize(st));
    }
    // scratch layout (bytes, each piece 256-aligned)
    const int Q = T * Kpad;
    int nsm = 0;
    GPM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    const int nparts = want_l ? gram_tc_parts(Q, Np, nsm) : 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_v = take(sizeof(float) * (size_t)ncta * C * Np * gm);
    const size_t o_ck = take(sizeof(float) * (size_t)ncta * nseg * gm * 20);
    const size_t o_S = take(sizeof(float) * (size_t)K);
    const size_t o_dU = take(sizeof(float) * (size_t)2 * T * K);
    const size_t o_dl = take(sizeof(float) * (size_t)8 * K);
    size_t o_B = 0, o_q = 0, o_p = 0;
    if (want_l) {
        o_B = take(sizeof(float) * (size_t)Q * Np);
        o_q = take(sizeof(float4) * (size_t)Q);
        o_p = take(sizeof(float) * 8 * (size_t)nparts);
    }
    if (off > c->grad_bytes) {
        cudaFree(c->grad_scr);
        c->grad_scr = nullptr;
        c->grad_bytes = 0;
        GPM_CUDA(cudaMalloc(&c->grad_scr, off));
        c->grad_bytes = off;
    }
    char* base = static_cast<char*>(c->grad_scr);
    GradArgs ga;
    std::memset(&ga, 0, sizeof(ga));
    ga.r = make_rollout_args(c, state, U_nom);
    ga.r.nom_sxy = nullptr;
    ga.Wt = g.Wt;
    ga.ubar = want_l ? g.ubar : nullptr;
    ga.weight = sample_weights;
    ga.slope = slope;
    ga.inv_K = 1.0f / (float)K;
    ga.C = C;
    ga.nseg = nseg;
    ga.Kpad = Kpad;
    ga.backward = dU ? 1 : 0;
    ga.vscr = reinterpret_cast<float*>(base + o_v);
    ga.ckpt = reinterpret_cast<float*>(base + o_ck);
    ga.S_out = reinterpret_cast<float*>(base + o_S);
    ga.dU_out = reinterpret_cast<float*>(base + o_dU);
    ga.dl_out = want_l ? reinterpret_cast<float*>(base + o_dl) : nullptr;
    ga.Bq = want_l ? reinterpret_cast<float*>(base + o_B) : nullptr;
    ga.qbar = want_l ? reinterpret_cast<float4*>(base + o_q) : nullptr;
    if (c->profiling) GPM_CUDA(cudaEventRecord(c->ev[0], st));
    if ((rc = launch_grad(ga, ncta, st))) return rc;
    if (c->profiling) GPM_CUDA(cudaEventRecord(c->ev[1], st));
    if (want_l) {
        // tr(dK/dl_d G_o), G_o = sum_q sbar_o,q b_q b_q^T over the T K queries:
        // the Gram contraction on the tensor cores, traced tile by tile
        if ((rc = launch_gram_tc(ga.Bq, ga.qbar, Q, Np, N, g.Xs[0], g.sf2[0], reinterpret_cast<float*>(base + o_p),
                                 nparts, c->err, nsm, st)))
            return rc;
    }
    GradReduceArgs rr;
    std::memset(&rr, 0, sizeof(rr));
    rr.dU_out = ga.dU_out;
    rr.S_out = ga.S_out;
    rr.dl_out = ga.dl_out;
    rr.parts = want_l ? reinterpret_cast<float*>(base + o_p) : nullptr;
    rr.nparts = nparts;
    rr.weight = sample_weights;
    rr.inv_K = ga.inv_K;
    rr.K = K;
    rr.T = dU ? T : 0;
    rr.dU = dU;
    rr.J = J;
    rr.dl = dlengthscale;
    for (int d = 0; d < 4; ++d) rr.ell[d] = (float)g.hyper[0].lengthscale[d];
    if ((rc = launch_grad_reduce(rr, st))) return rc;
    if (c->profiling) {
        GPM_CUDA(cudaEventRecord(c->ev[2], st));
        c->profiled = true;
    }
    return GPMPPI_OK;
}

int mppi_set_iteration(gpmppi_ctrl c, uint64_t it) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_set_iteration: invalid handle");
    c->it = it;
    return GPMPPI_OK;
}

int mppi_get_iteration(gpmppi_ctrl c, uint64_t* it) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_get_iteration: invalid handle");
    if (!it) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_get_iteration: it must not be NULL");
    *it = c->it;
    return GPMPPI_OK;
}

int mppi_nominal_sxy(gpmppi_ctrl c, float* sxy, void* stream) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_nominal_sxy: invalid handle");
    int rc;
    if ((rc = check_dev_ptr(sxy, "mppi_nominal_sxy: sxy", false))) return rc;
    GPM_CUDA(cudaMemcpyAsync(sxy, c->nom_sxy, sizeof(float) * 3 * c->p.T, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    return GPMPPI_OK;
}

int mppi_set_wait_limit(gpmppi_ctrl c, uint64_t ns, int32_t expire_first) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_set_wait_limit: invalid handle");
    c->wait_ns = ns;
    c->expire_first = expire_first ? 1 : 0;
    return GPMPPI_OK;
}

int mppi_rollout_kind(gpmppi_ctrl c, int32_t* kind) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_rollout_kind: invalid handle");
    if (!kind) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_rollout_kind: kind is NULL");
    *kind = (c->ens && c->fmt < 0) ? GPMPPI_KERNEL_ENSEMBLE
                   : (c->cl ? GPMPPI_KERNEL_TC_CLUSTER : (c->fmt >= 0 ? GPMPPI_KERNEL_TC_STREAM : GPMPPI_KERNEL_FP32));
    return GPMPPI_OK;
}

int mppi_set_profiling(gpmppi_ctrl c, int32_t on) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_set_profiling: invalid handle");
    if (on && !c->ev[0])
        for (cudaEvent_t& e : c->ev) GPM_CUDA(cudaEventCreate(&e));
    c->profiling = on != 0;
    c->profiled = false;
    return GPMPPI_OK;
}

int mppi_last_profile(gpmppi_ctrl c, float* rollout_ms, float* update_ms) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_last_profile: invalid handle");
    if (!c->profiled) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_last_profile: no profiled step");
    GPM_CUDA(cudaEventSynchronize(c->ev[2]));
    float a = 0.0f, b = 0.0f;
    GPM_CUDA(cudaEventElapsedTime(&a, c->ev[0], c->ev[1]));
    GPM_CUDA(cudaEventElapsedTime(&b, c->ev[1], c->ev[2]));
    if (rollout_ms) *rollout_ms = a;
    if (update_ms) *update_ms = b;
    return GPMPPI_OK;
}

int mppi_device_status(gpmppi_ctrl c) {
    if (!valid_ctrl(c)) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_device_status: invalid handle");
    int rc;
    if ((rc = check_ctrl_device(c))) return rc;
    GPM_CUDA(cudaDeviceSynchronize());
    unsigned int word = 0;
    GPM_CUDA(cudaMemcpy(&word, c->err, sizeof(word), cudaMemcpyDeviceToHost));
    if (word == 0) return GPMPPI_OK;
    GPM_CUDA(cudaMemset(c->err, 0, sizeof(unsigned int)));
    return fail(GPMPPI_ERR_TIMEOUT, "a rollout kernel gave up waiting for a tile copy");
}

int mppi_destroy(gpmppi_ctrl c) {
    if (!c || c->magic != kCtrlMagic) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_destroy: invalid handle");
    cudaDeviceSynchronize();
    free_ctrl(c);
    return GPMPPI_OK;
}

int gpmppi_philox(uint64_t seed, const uint32_t* ctr, int32_t M, uint32_t* out, void* stream) {
    if (M < 0) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_philox: M must be >= 0");
    if (M == 0) return GPMPPI_OK;
    int rc;
    if ((rc = check_dev_ptr(ctr, "gpmppi_philox: ctr", false))) return rc;
    if ((rc = check_dev_ptr(out, "gpmppi_philox: out", false))) return rc;
    if ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) & 15u)
        return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_philox: arrays must be 16-byte aligned");
    return launch_philox(seed, ctr, M, out, (cudaStream_t)stream);
}

int gpmppi_control_noise(uint64_t seed, int32_t K, int32_t T, uint64_t it, const float sigma[2],
                         float* eps, void* stream) {
    if (K < 0 || T < 0 || !sigma) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_control_noise: bad arguments");
    if ((size_t)K * T == 0) return GPMPPI_OK;
    int rc;
    if ((rc = check_dev_ptr(eps, "gpmppi_control_noise: eps", false))) return rc;
    if (reinterpret_cast<uintptr_t>(eps) & 7u)
        return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_control_noise: eps must be 8-byte aligned");
    return launch_noise(seed, K, T, it, sigma[0], sigma[1], eps, (cudaStream_t)stream);
}

int gpmppi_mma_selftest(int32_t fmt, int32_t N, int32_t K, int32_t variant, const uint16_t* A,
                        const uint16_t* B, float* D) {
    if (fmt != 0 && fmt != 1) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_mma_selftest: fmt must be 0 or 1");
    if (N != 64 && N != 128 && N != 256) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_mma_selftest: N must be 64, 128 or 256");
    if (K != 16 && K != 32 && K != 48 && K != 64) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_mma_selftest: K must be 16, 32, 48 or 64");
    if (variant < 0 || variant > 2) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_mma_selftest: variant must be 0, 1 or 2");
    if (variant == 1 && N > 128) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_mma_selftest: variant 1 needs N <= 128");
    int rc;
    if ((rc = check_dev_ptr(A, "gpmppi_mma_selftest: A", false))) return rc;
    if ((rc = check_dev_ptr(B, "gpmppi_mma_selftest: B", false))) return rc;
    if ((rc = check_dev_ptr(D, "gpmppi_mma_selftest: D", false))) return rc;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u)
        return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_mma_selftest: A and B must be 16-byte aligned");
    unsigned int* err = nullptr;
    GPM_CUDA(cudaMalloc(&err, sizeof(unsigned int)));
    cudaError_t e = cudaMemset(err, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        rc = launch_mma_selftest(fmt, N, K, variant, A, B, D, err, nullptr);
        if (rc) {
            cudaFree(err);
            return rc;
        }
        e = cudaDeviceSynchronize();
    }
    unsigned int word = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&word, err, sizeof(word), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "gpmppi_mma_selftest");
    if (word) return fail(GPMPPI_ERR_TIMEOUT, "gpmppi_mma_selftest: MMA completion did not arrive");
    return GPMPPI_OK;
}

}  // extern "C"
