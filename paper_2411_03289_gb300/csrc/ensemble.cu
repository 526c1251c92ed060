// Rollout with the weighted terrain ensemble of Eq. 3 (Alg. 1 Step 1), FP32.
//
// The residual of every step is the mixture of M terrain GPs: mean
// sum_i w_i m_i(z) and variance sum_i w_i^2 var_i(z) per output (the two
// outputs of a terrain share its hyper-parameters, so var_i is one number).
// One CTA carries GMT samples, one warp each.  Per step and terrain the warps
// write their samples' kernel rows k*_i (with terrain i's lengthscales) into
// shared memory, the CTA forms V_i = K*_i L_i^-T with the balanced triangular
// product (rows of L_i^-T read from L2), and each warp reduces |v_i|^2 and
// its mean partials.  The mixed mean and variance then drive Eq. 6 and 10 and
// the stage cost of Eq. 11-16 with the goal terms of Eq. 12, exactly as in
// the single-GP rollouts; the outputs (costs, u_tilde, optional per-step
// records) have the same layout, so the same update kernel follows.
#include <cfloat>

#include "common.cuh"
#include "warp_rollout.cuh"

namespace gpm {
namespace {

using namespace wr;

constexpr int ESAVE = 32;    // per-warp spill area for the state live across a product

template <bool TRACE>
__global__ void __launch_bounds__(GT, 2) k_rollout_ens(const EnsArgs e) {
    extern __shared__ __align__(16) float esm[];
    const RolloutArgs& a = e.r;
    const int Npm = e.Npmax;
    float* kT = esm;                         // Npm x GMT kernel rows
    float* vT = kT + Npm * GMT;              // Npm x GMT products
    float* saves = vT + Npm * GMT;           // GMT x ESAVE
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    float* save = saves + w * ESAVE;
    const int s = blockIdx.x * GMT + w;
    const bool act = s < a.K;

    float mu[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) mu[i] = a.x0_dev ? a.x0_dev[i] : a.x0[i];
    uint32_t it0 = a.it0, it1 = a.it1;
    if (a.it_dev) {
        const unsigned long long v = *a.it_dev;
        it0 = (uint32_t)v;
        it1 = (uint32_t)(v >> 32);
    }
    float S[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) S[i] = 0.0f;
    float cost = 0.0f;

    for (int k = 0; k < a.T; ++k) {
        // noise and clamp (Eq. 8), lane-replicated
        const float2 eps = control_eps((uint32_t)k, (uint32_t)(act ? s : 0), it0, it1, a.key0, a.key1,
                                       a.sig_v, a.sig_w);
        float ux = fminf(fmaxf(__ldg(a.U + 2 * k) + eps.x, a.umin0), a.umax0);
        float uy = fminf(fmaxf(__ldg(a.U + 2 * k + 1) + eps.y, a.umin1), a.umax1);
        if (act && lane == 0) a.u_tilde[(size_t)k * a.K + s] = make_float2(ux, uy);

        // the terrain mixture (Eq. 3)
        float mbv = 0.0f, mbw = 0.0f, cvar = 0.0f;
        for (int t = 0; t < e.M; ++t) {
            const TerrainGp& gp = e.gp[t];
            const float z0 = mu[3] * gp.zscale[0], z1 = mu[4] * gp.zscale[1], z2 = ux * gp.zscale[2],
                        z3 = uy * gp.zscale[3];
            float mv = 0.0f, mw = 0.0f, cv = 0.0f, cw = 0.0f;
            for (int j = lane; j < gp.Np; j += 32) {
                float kv = 0.0f;
                if (act && j < gp.N) {
                    const float4 x = ldg4(gp.Xs + 4 * j);
                    const float d0 = z0 - x.x, d1 = z1 - x.y, d2 = z2 - x.z, d3 = z3 - x.w;
                    kv = gp.sf2 * exp2f(-(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3));
                    const float2 al = __ldg(reinterpret_cast<const float2*>(gp.alpha) + j);
                    kahan_add(mv, cv, kv * al.x);
                    kahan_add(mw, cw, kv * al.y);
                }
                kT[j * GMT + w] = kv;
            }
            mbv += gp.w * wsum(mv + cv);
            mbw += gp.w * wsum(mw + cw);
            // the warp's state waits in shared memory while the product runs
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < 5; ++i) save[i] = mu[i];
#pragma unroll
                for (int i = 0; i < 15; ++i) save[5 + i] = S[i];
                save[20] = ux;
                save[21] = uy;
                save[22] = mbv;
                save[23] = mbw;
                save[24] = cvar;
                save[25] = cost;
            }
            __syncthreads();
            tri_product<false>(gp.W, gp.Np, kT, vT);
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 5; ++i) mu[i] = save[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) S[i] = save[5 + i];
            ux = save[20];
            uy = save[21];
            mbv = save[22];
            mbw = save[23];
            cvar = save[24];
            cost = save[25];
            float q = 0.0f;
            for (int i = lane; i < gp.Np; i += 32) {
                const float x = vT[i * GMT + w];
                q = fmaf(x, x, q);
            }
            q = wsum(q);
            cvar += gp.w * gp.w * fmaxf(0.0f, gp.sf2 - q);
            // the next terrain's kT writes follow the barrier after this
            // product, and its product's vT writes the barrier before it
        }

        // mean and covariance (Eq. 6, 10) with the mixture
        float sn, cs;
        sincosf(mu[2], &sn, &cs);
        const float a02 = -a.dt * mu[3] * sn, a03 = a.dt * cs;
        const float a12 = a.dt * mu[3] * cs, a13 = a.dt * sn;
        const float nX = mu[0] + a.dt * mu[3] * cs;
        const float nY = mu[1] + a.dt * mu[3] * sn;
        const float nT = mu[2] + a.dt * mu[4];
        const float nV = mu[3] + a.kv * (ux - mu[3]) + mbv;
        const float nW = mu[4] + a.kw * (uy - mu[4]) + mbw;
        mu[0] = nX; mu[1] = nY; mu[2] = nT; mu[3] = nV; mu[4] = nW;
        {
            const float A[5][5] = {{1.f, 0.f, a02, a03, 0.f},
                                   {0.f, 1.f, a12, a13, 0.f},
                                   {0.f, 0.f, 1.f, 0.f, a.dt},
                                   {0.f, 0.f, 0.f, a.av, 0.f},
                                   {0.f, 0.f, 0.f, 0.f, a.aw}};
            float Sf[5][5], B[5][5];
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) Sf[i][j] = (i <= j) ? S[sidx(i, j)] : S[sidx(j, i)];
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    float t2 = 0.0f;
#pragma unroll
                    for (int m = 0; m < 5; ++m) t2 = fmaf(A[i][m], Sf[m][j], t2);
                    B[i][j] = t2;
                }
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = i; j < 5; ++j) {
                    float t2 = 0.0f;
#pragma unroll
                    for (int m = 0; m < 5; ++m) t2 = fmaf(B[i][m], A[j][m], t2);
                    S[sidx(i, j)] = t2;
                }
            S[sidx(3, 3)] += cvar;
            S[sidx(4, 4)] += cvar;
        }

        // stage cost (Eq. 11-16 and the goal terms of Eq. 12)
        if (act) {
            const float sxx = S[sidx(0, 0)], sxy = S[sidx(0, 1)], syy = S[sidx(1, 1)];
            const Lam L = lam_max(sxx, sxy, syy);
            const float rbar = a.r - a.sq_chi2 * L.sq;
            float best;
            int bi;
            lane_nearest(a, mu[0], mu[1], best, bi);
            const float el = sqrtf(best);
            const float lmargin = el - rbar;
            float om = FLT_MAX;
            if (a.O > 0) {
                int oi;
                obstacle_nearest(a, mu[0], mu[1], sxx, sxy, syy, L.sq, om, oi);
            }
            const float disc = exp2f((float)k * log2f(0.9f));
            float stage = a.c_var * (cvar + cvar) + a.c_speed * (a.v_des - mu[3]) * (a.v_des - mu[3]);
            if (a.O > 0 && om <= 0.0f) stage += a.c_coll;
            stage += a.c_dev * el;
            if (lmargin > 0.0f) stage += a.c_lane * disc;
            stage += goal_cost(a, k, mu[0], mu[1]);
            cost += stage;
            if (TRACE && lane == 0) {
                const size_t sk = (size_t)s * a.T + k;
                if (a.tr_mu)
                    for (int i = 0; i < 5; ++i) a.tr_mu[sk * 5 + i] = mu[i];
                if (a.tr_sig)
                    for (int i = 0; i < 15; ++i) a.tr_sig[sk * 15 + i] = S[i];
                if (a.tr_stage) a.tr_stage[sk] = stage;
                if (a.tr_margin) {
                    a.tr_margin[sk * 2] = lmargin;
                    a.tr_margin[sk * 2 + 1] = (a.O > 0) ? om : __int_as_float(0x7f800000);
                }
            }
        }
    }
    if (act && lane == 0 && a.costs) a.costs[s] = cost;
}

}  // namespace

int ens_smem_bytes(int Npmax) {
    return (int)(sizeof(float) * (2 * (size_t)Npmax * GMT + (size_t)GMT * ESAVE));
}

int launch_rollout_ens(const EnsArgs& e, bool trace, cudaStream_t st) {
    const int smem = ens_smem_bytes(e.Npmax);
    const int grid = (e.r.K + GMT - 1) / GMT;
    if (trace) {
        GPM_CUDA(cudaFuncSetAttribute(k_rollout_ens<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_rollout_ens<true><<<grid, GT, smem, st>>>(e);
    } else {
        GPM_CUDA(cudaFuncSetAttribute(k_rollout_ens<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_rollout_ens<false><<<grid, GT, smem, st>>>(e);
    }
    GPM_CUDA(cudaGetLastError());
    return 0;
}

}  // namespace gpm
