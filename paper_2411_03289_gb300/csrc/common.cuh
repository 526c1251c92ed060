// Internal declarations shared by the CUDA translation units of libgpmppi.
//
// Nothing here is part of the C ABI (include/gpmppi.h is).  The device
// helpers below are used by every kernel that draws control noise, so the
// rollout, the update and the debug entry points see bit-identical draws.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gpmppi.h"

namespace gpm {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Round function on the
// counter words (c0,c1,c2,c3) with key (k0,k1):
//   c0' = hi(M1 c2) ^ c1 ^ k0,  c1' = lo(M1 c2),
//   c2' = hi(M0 c0) ^ c3 ^ k1,  c3' = lo(M0 c0),
// and the Weyl key schedule k += (W0, W1) between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const uint32_t lo0 = kPhiloxM0 * c.x;
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Standard normal pair from two Philox words by Box-Muller with the
// uniforms u = (w + 1/2) 2^-32 in (0,1).  -2 ln u0 is evaluated through
// log1p(-(1 - u0)) when u0 >= 1/2, where 1 - u0 = (~w0 + 1/2) 2^-32 is formed
// without cancellation; the angle 2 pi u1 goes through sincospi.
__device__ __forceinline__ float2 box_muller(uint32_t w0, uint32_t w1) {
    float r2;
    if (w0 >= 0x80000000u) {
        const float t = (__uint2float_rn(~w0) + 0.5f) * 0x1p-32f;
        r2 = -2.0f * log1pf(-t);
    } else {
        const float u0 = (__uint2float_rn(w0) + 0.5f) * 0x1p-32f;
        r2 = -2.0f * logf(u0);
    }
    const float rad = sqrtf(r2);
    const float u1 = (__uint2float_rn(w1) + 0.5f) * 0x1p-32f;
    float s, c;
    sincospif(2.0f * u1, &s, &c);
    return make_float2(rad * c, rad * s);
}

// Control perturbation of sample s at step k, iteration (it0 = low word,
// it1 = high word): counter (k, s, it0, it1), key (seed_lo, seed_hi).
__device__ __forceinline__ float2 control_eps(uint32_t k, uint32_t s, uint32_t it0, uint32_t it1,
                                              uint32_t key0, uint32_t key1, float sig_v, float sig_w) {
    const uint4 w = philox4x32_10(make_uint4(k, s, it0, it1), key0, key1);
    const float2 z = box_muller(w.x, w.y);
    return make_float2(sig_v * z.x, sig_w * z.y);
}

// Compensated (Neumaier) accumulation s += x with running correction c: the
// GP mean is a long sum of terms k*_j alpha_j of both signs that largely
// cancel, where plain FP32 accumulation loses digits with the length of the sum.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

// ---------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
// INVALID_ARG unless p is device (or managed) memory of the current device
// (NULL is accepted when nullable).
int check_dev_ptr(const void* p, const char* name, bool nullable);

#define GPM_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ::gpm::cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// device-side layout of a fitted GP
// ---------------------------------------------------------------------------
struct GpDevice {
    int N = 0;        // training points
    int Np = 0;       // N rounded up to a multiple of 16, at least 64 (W is Np x Np)
    int device = 0;
    bool shared = true;          // both outputs share their hyper-parameters
    float sf2[2] = {0, 0};       // signal variances
    // per output o: Xs[o] = N x 4 floats, X scaled by sqrt(log2(e)/2)/l_d so
    // that k = sf2 * exp2(-|xs - zs|^2); W[o] = Np x Np floats, W[j][i] =
    // (L^-1)[i][j] for i >= j, zero elsewhere (row j of L^-T).
    float* Xs[2] = {nullptr, nullptr};
    float* W[2] = {nullptr, nullptr};
    float* alpha = nullptr;      // N x 2 floats (alpha_v, alpha_w) per point
    float zscale[2][4] = {};     // the per-input scale applied to queries
    // FP64 factors kept for export: Linv64[o] N x N, alpha64[o] N
    double* Linv64[2] = {nullptr, nullptr};
    double* alpha64[2] = {nullptr, nullptr};
    // tensor-core tiles of L^-T per operand format (0 = FP16 hi/lo, 1 = BF16
    // hi/lo, 2 = BF16 hi/mid/lo), built on first use by a controller; NpM = N
    // rounded up to 128
    uint16_t* mma_hi[3] = {nullptr, nullptr, nullptr};
    uint16_t* mma_lo[3] = {nullptr, nullptr, nullptr};
    uint16_t* mma_mid = nullptr;   // the middle part of format 2
    float mma_cB = 0.0f;
    int NpM = 0;
    // the streaming rollout's training inputs and alpha in pair layout (NpM x 4
    // floats, then NpM x 2; see k_pack_xa), copied into shared memory in bulk
    float* mma_xa = nullptr;
    // resident tiles of the cluster rollout (N <= 512): per 16-bit format, rank
    // r's pieces at element offset cl_base[r], cl_bytes[r] bytes; NpC = 128,
    // 256 or 512 output columns.  A piece holds one 16-point chunk of the
    // rank's output rows, hi and lo parts as one slab-major operand: rows
    // [hi lower | hi upper | lo upper | lo lower] slice (256) while both
    // slices need the chunk, [hi upper | lo upper] (128) after
    uint16_t* cl_tiles[2] = {nullptr, nullptr};
    int cl_base[4] = {0, 0, 0, 0};
    int cl_bytes[4] = {0, 0, 0, 0};
    int cl_npc = 0;
    // the cluster rollout's training inputs and alpha in pair layout (NpC x 4
    // floats, then NpC x 2), copied into shared memory by one bulk copy
    float* cl_xa = nullptr;
    // adjoint rollout, built on first use: rows of L^-1 (Np x Np) and the
    // vectors (dK/dl_d) alpha_o (8 x Np)
    float* Wt = nullptr;
    float* ubar = nullptr;
    gpmppi_hyper hyper[2];
    int n_controllers = 0;
};

// Everything one rollout launch needs (passed by value as a kernel argument).
struct RolloutArgs {
    const float* Xs;        // N x 4 scaled GP inputs
    const float* alpha;     // N x 2
    const float* W;         // Np x Np
    const float* obst;      // O x 3 (cx, cy, r)
    const float4* seg;      // S segments: (ax, ay, bx - ax, by - ay)
    const float* seg_il2;   // S: 1 / |b - a|^2, or 0 for a degenerate segment
    const float* U;         // T x 2 nominal controls
    const float* nom_sxy;   // T x 3 tightening covariance (nominal mode) or null
    float* costs;           // K
    float2* u_tilde;        // T x K clamped sampled controls (for the update)
    // optional per-(s,k) records
    float* tr_mu;           // K x T x 5
    float* tr_sig;          // K x T x 15
    float* tr_stage;        // K x T
    float* tr_margin;       // K x T x 2
    int K, T, N, Np, O, S;
    int mt;                 // samples per CTA
    int stages;             // per-warp TMA pipeline depth for the L^-T tiles
    unsigned int* err;      // device status word (bit 0: a bounded wait gave up)
    unsigned long long wait_ns;   // FP32 rollout: limit of each tile-copy wait (mppi_set_wait_limit)
    int expire_first;             // FP32 rollout: first wait on a barrier nothing completes (test hook)
    float sf2;
    float x0[5];
    float zscale[4];
    float dt, kv, kw, av, aw;   // kv = dt/tau_v, av = 1 - kv (same for omega)
    float sig_v, sig_w;
    float umin0, umin1, umax0, umax1;
    float c_var;            // (alpha_0 + beta_0): weight of trace(C)
    float c_dev;            // alpha_1 / r
    float c_lane;           // alpha_3 * P_lane
    float c_speed;          // alpha_4
    float c_coll;           // beta_1 * P_coll
    float r, v_des, sq_chi2, phi_inv;
    // candidate segments of the lane-distance grid (lane_grid.cu); gcell null: scan all
    const int2* gcell;      // gny x gnx cells: (offset into gidx, count)
    const int* gidx;
    float gx0, gy0, ginv;   // grid origin and 1 / cell size
    int gnx, gny;
    float c_goal;           // beta_2: weight of the distance to the goal (every stage)
    float c_term;           // beta_3 * P_goal: terminal miss penalty
    float goal_x, goal_y, goal_r;
    uint32_t key0, key1, it0, it1;
    // when set, the initial state and the iteration are read from device
    // memory instead of x0 / it0 / it1 (batched and graph-replayed steps)
    const float* x0_dev;
    const unsigned long long* it_dev;
};

constexpr int kMaxTerrains = 8;

// The GPs of a tensor-core rollout: M = 1 is the single GP, M > 1 the terrain
// ensemble of Eq. 3 (mean sum_t w_t m_t, variance sum_t w_t^2 var_t).  The
// factors are stacked block-diagonally: terrain t owns the 128-column blocks
// [blk0[t], blk0[t+1]) of the output and the training points 128 blk0[t] ..
// 128 blk0[t+1] - 1; with M > 1 every terrain's block count is even, so no
// pair of blocks straddles two terrains.
struct MmaTerrains {
    int M;
    int blk0[kMaxTerrains + 1];
    float qscale[kMaxTerrains];     // (sf2_t / cB_t)^2: |L_t^-1 k*|^2 = qscale_t |V'_t|^2
    float sf2[kMaxTerrains];        // signal variance
    float w[kMaxTerrains];          // mixing weight (1 for the single GP)
    float zscale[kMaxTerrains][4];  // query scaling (the GP's inverse lengthscales)
};

// Tensor-core variance contraction: cB L^-T (cB a power of two per GP) split
// into 16-bit parts, packed by k_pack_mma as 16 KiB pair pieces (256 output
// columns x 32 training points, slab-major operand layout).
struct MmaArgs {
    const uint16_t* Bhi;
    const uint16_t* Blo;
    const uint16_t* Bmid;   // format 2 (BF16 hi/mid/lo) only, else null
    const float* xa;        // training inputs and alpha in pair layout (GpDevice::mma_xa)
    int nblocks;            // 128-column blocks of all GPs together (tr.blk0[tr.M])
    int parts;              // operand parts: 2 (hi, lo) or 3 (hi, mid, lo)
    MmaTerrains tr;         // per-GP ranges and constants
    int stages;             // shared-memory pipeline depth (2..6)
    int rps;                // producer threads per sample (2, 4, 8): 128, 64, 32 samples per CTA
    int scene_smem;         // lane segments and obstacles staged in shared memory
    int lo_set;             // 1: the small split products in their own TMEM column set
                            // (passes of 2 output blocks), 0: all three in one (passes of 4)
};

// The lane segments to scan for the point (px, py): (offset into gidx, count),
// or (-1, S) for every segment when the point lies outside the grid.
__device__ __forceinline__ int2 lane_cands(const RolloutArgs& a, float px, float py) {
    if (a.gcell) {
        const float fx = (px - a.gx0) * a.ginv, fy = (py - a.gy0) * a.ginv;
        if (fx >= 0.0f && fy >= 0.0f && fx < (float)a.gnx && fy < (float)a.gny) {
            const int ix = min((int)fx, a.gnx - 1), iy = min((int)fy, a.gny - 1);
            return __ldg(a.gcell + iy * a.gnx + ix);
        }
    }
    return make_int2(-1, a.S);
}

// i-th segment of a candidate range from lane_cands
__device__ __forceinline__ int lane_seg(const RolloutArgs& a, int2 oc, int i) {
    return oc.x < 0 ? i : __ldg(a.gidx + oc.x + i);
}

// Goal terms of Eq. 12 at stage k (0-based) for the mean position (x, y):
// c_goal |p - goal| at every stage, plus c_term on the last stage when the
// mean is farther than goal_r from the goal.
__device__ __forceinline__ float goal_cost(const RolloutArgs& a, int k, float x, float y) {
    if (a.c_goal == 0.0f && a.c_term == 0.0f) return 0.0f;
    const float dx = x - a.goal_x, dy = y - a.goal_y;
    const float d = sqrtf(dx * dx + dy * dy);
    float c = a.c_goal * d;
    if (k == a.T - 1 && d > a.goal_r) c += a.c_term;
    return c;
}

// Host side of the lane-distance grid (built once per controller).
struct LaneGridHost {
    float x0 = 0, y0 = 0, inv_h = 0;
    int nx = 0, ny = 0;
    std::vector<int2> cells;
    std::vector<int> idx;
};
int build_lane_grid(const float* path, int P, LaneGridHost& g);

// One terrain GP of an ensemble (Eq. 3) as the ensemble rollout reads it.
struct TerrainGp {
    const float* Xs;        // N x 4, scaled by this GP's lengthscales
    const float* alpha;     // N x 2
    const float* W;         // Np x Np rows of L^-T
    int N, Np;
    float sf2;
    float zscale[4];
    float w;                // ensemble weight w_i
};

struct EnsArgs {
    RolloutArgs r;          // scene, controls, constants (the GP fields of r are unused)
    TerrainGp gp[kMaxTerrains];
    int M;
    int Npmax;              // largest Np of the terrains
};

// Adjoint rollout (gradient of the smoothed cost); see adjoint.cu.
struct GradArgs {
    RolloutArgs r;          // scene, GP, controls and constants of the controller
    const float* Wt;        // Np x Np rows of L^-1 (zero above the diagonal and in the padding)
    const float* ubar;      // 8 x Np: (dK/dl_d) alpha_o / (2 ln2 / l_d), row o*4+d; null: no K terms
    const float* weight;    // K sample weights, or null for 1/K
    float slope;            // sigmoid slope of the smoothed indicators
    float inv_K;
    int C, nseg, Kpad;      // checkpoint interval, segments, CTAs x samples per CTA
    int backward;           // 0: objective only
    float* vscr;            // n_cta x C x Np x 8: v = L^-1 k* of the current segment
    float* ckpt;            // n_cta x nseg x 8 x 20: (mu, Sigma) at the segment starts
    float* S_out;           // K smoothed rollout costs
    float* dU_out;          // 2T x K per-sample control adjoints (weighted)
    float* dl_out;          // 8 x K per-sample lengthscale terms, or null
    float* Bq;              // (T Kpad) x Np: b = K^-1 k* per query, or null
    float4* qbar;           // T Kpad: (mbar_v, mbar_w, sbar_v, sbar_w) per query
};

struct GradReduceArgs {
    const float* dU_out;
    const float* S_out;
    const float* dl_out;
    const float* parts;     // nparts x 8 Gram-trace partials
    int nparts;
    const float* weight;
    float inv_K;
    int K, T;
    float* dU;              // T x 2
    float* J;               // 1
    float* dl;              // 2 x 4, or null
    float ell[4];
};

// Cluster rollout (N <= 512): CS CTAs share 128 samples; rank r holds its
// column slices of cB L^-1 resident in shared memory.
struct ClArgs {
    const uint16_t* tiles;  // all ranks' pieces (one 16-bit format)
    int base[4];            // element offset of rank r's pieces
    int bytes[4];           // their size in bytes
    int cs;                 // cluster size (CTAs per 128 samples): NS / 2
    int ns;                 // 64-column slices: NpC / 64
    int npc;                // padded training-set size (128, 256 or 512)
    float qscale;           // (sf2 / cB)^2
    int scene_smem;         // lane segments and obstacles staged in shared memory
    const float* xa;        // training inputs and alpha in pair layout (npc x 6 floats)
};

struct UpdateArgs {
    const float* costs;     // K
    const float2* u_tilde;  // T x K
    const float* U;         // T x 2
    float* U_new;           // T x 2
    float* weights;         // K or null
    float* partial;         // n_cta x (T + 1) x 2 scratch: partial sums, then (rho_b, Z_b) per CTA
    unsigned int* counter;  // one scratch word, zero between launches
    int K, T;
    int per_cta;            // samples per CTA
    float inv_lambda;
};

// launchers (defined in the .cu files)
int launch_rollout_fp32(const RolloutArgs& a, const CUtensorMap* tmap_w, bool trace,
                        cudaStream_t st);
// TMA tensor map over W (Np x Np floats) with the box the FP32 rollout reads
int make_w_tensor_map(CUtensorMap* out, const float* W, int Np);
// pipeline depth that fits shared memory (0 if none fits)
int rollout_fp32_stages(int Np, int smem_optin);
// after_rollout: the previous operation on st is the rollout kernel, and the
// update's launch may overlap its tail (programmatic dependent launch)
int launch_update(const UpdateArgs& a, int n_cta, cudaStream_t st, bool after_rollout);
int launch_update_batched(const UpdateArgs* args, const int2* items, const int* ncta,
                          unsigned long long* iters, int nitems, int maxT, cudaStream_t st);
int rollout_mma_smem(const MmaArgs& mm, int S, int O);
// Batched persistent rollout: `grid` CTAs (one per SM) take items (controller,
// tile, kind: 0 FP32 / 1 FP16 split / 2 BF16 split, producer threads per
// sample) from the queue, advancing *head (zero before the launch).
int launch_rollout_persistent(const RolloutArgs* args, const MmaArgs* mms, const CUtensorMap* tmaps,
                              const int4* items, int nitems, unsigned int* head, int grid, int smem,
                              cudaStream_t st);
int launch_gp_predict(const GpDevice& g, const float* Z, int M, float* mean, float* var,
                      cudaStream_t st);
int gp_fit_device(GpDevice& g, const double* X, const double* Y, int N, cudaStream_t st);
int launch_philox(uint64_t seed, const uint32_t* ctr, int M, uint32_t* out, cudaStream_t st);
int launch_noise(uint64_t seed, int K, int T, uint64_t it, float sv, float sw, float* eps,
                 cudaStream_t st);
int launch_nominal(const RolloutArgs& a, float* sxy_out, cudaStream_t st);
int rollout_fp32_smem_bytes(int Np, int mtp, int stages);
int launch_rollout_mma(const RolloutArgs& a, const MmaArgs& mm, int fmt, bool trace, cudaStream_t st);
int rollout_mma_stages(int NpM, int S, int O, int smem_optin, int lo_set, int parts, int M);
int build_mma_tiles(GpDevice& g, int fmt);
int build_cl_tiles(GpDevice& g, int fmt);
// The M GPs of a terrain ensemble as one block-diagonal factor for the
// streaming tensor-core rollout: fills tr (ranges, scales, weights 1) and
// allocates the stacked tiles and training set (caller frees them).
int build_mma_ensemble(GpDevice* const* gs, int M, int fmt, MmaTerrains& tr, uint16_t** hi, uint16_t** lo,
                       uint16_t** mid, float** xa);
int cl_smem_bytes(const ClArgs& cl, int S, int O);
bool cl_schedulable(const ClArgs& cl, int S, int O, int device);
int launch_rollout_cl(const RolloutArgs& a, const ClArgs& cl, int fmt, bool trace, cudaStream_t st);
int launch_mma_selftest(int fmt, int N, int K, int variant, const uint16_t* A, const uint16_t* B,
                        float* D, unsigned int* err, cudaStream_t st);
int rollout_fp32_mtp(int Np);
int grad_smem_bytes(int Np, int C);
int grad_samples_per_cta();
int launch_grad(const GradArgs& g, int ncta, cudaStream_t st);
// tr(D_d G_o) from G = [G_v; G_w] (2 Np x Np, column-major): one block per 8
// columns, 8 partial sums per block; returns the number of blocks
// the lengthscale Gram traces on the tensor cores (gram_tc.cu): nparts x 8
// partial traces, nparts = gram_tc_parts(Q, Np, nsm)
int gram_tc_parts(int Q, int Np, int nsm);
int launch_gram_tc(const float* Bq, const float4* qbar, int Q, int Np, int N, const float* Xs, float sf2,
                   float* part, int nparts, unsigned int* err, int nsm, cudaStream_t st);
int launch_dk_alpha(const float* Xs, const float* alpha, int N, int Np, float sf2, float* ubar,
                    cudaStream_t st);
int launch_transpose(const float* W, int Np, float* Wt, cudaStream_t st);
int launch_grad_reduce(const GradReduceArgs& r, cudaStream_t st);
int ens_smem_bytes(int Npmax);
int launch_rollout_ens(const EnsArgs& e, bool trace, cudaStream_t st);

}  // namespace gpm
