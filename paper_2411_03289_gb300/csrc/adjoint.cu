// Adjoint (reverse-mode) rollout: gradient of the smoothed chance-constrained
// MPPI cost with respect to the nominal controls U and the SE-ARD
// lengthscales of the residual GPs.
//
// Objective.  J = sum_s w_s S_s, where S_s is the rollout cost of sample s
// (Alg. 1 Step 1, Eq. 10-16) with the indicators of Eq. 11-12 replaced by
// logistic sigmoids of slope * margin, the control noise held fixed (the
// Philox draws of the current iteration) and w_s = 1/K unless the caller
// passes weights.
//
// One CTA carries GMT samples, one warp per sample, through three passes:
//   1. forward over all T steps: S_s, plus the state (mu, Sigma) every C
//      steps (C = ceil(sqrt(T))) as a checkpoint in global scratch;
//   2. for each segment of C steps, last first: the forward steps again from
//      the segment's checkpoint, keeping per-step states in shared memory and
//      v = L^-1 k* (the GP variance factor) in global scratch;
//   3. the reverse steps of that segment: stage-cost adjoint (lane distance,
//      lambda_max of Sigma_XY, obstacle spread), covariance adjoint
//      (Sigma' = A Sigma A^T + D: Sigma_bar = A^T G A, A_bar = 2 G A Sigma),
//      mean adjoint (Eq. 6), then the GP adjoint: b = L^-T v = K^-1 k* by a
//      second triangular product, k*_bar_j = m_bar . alpha_j - 2 s_bar b_j,
//      and z_bar, the direct lengthscale terms and the terms that flow
//      through alpha = K^-1 y.
// The terms that flow through K^-1 in the variance need G_o = sum_q s_bar_o,q
// b_q b_q^T; the CTAs store b_q and the per-query adjoints, and a Gram kernel
// forms tr(dK/dl_d G_o) tile by tile.  A last kernel reduces the per-sample
// contributions in double in a fixed order, so results are deterministic.
#include <cfloat>

#include "common.cuh"
#include "warp_rollout.cuh"

namespace gpm {
namespace {

using namespace wr;

constexpr float kLn2 = 0.69314718055994530942f;

struct StepInfo {
    float ux, uy;      // clamped perturbed control (Eq. 8)
    float sraw;        // sf2 - |L^-1 k*|^2 before the clamp at zero
    int mask;          // bit c: control component c strictly inside its box
};

// One forward step of sample s (warp w); all threads of the CTA call it.
// mu / S are the warp's (lane-replicated) state, advanced in place.
__device__ void fwd_step(const GradArgs& g, int k, int s, bool act, float mu[5], float S[15],
                         float* kT, float* vT, float* vstore, StepInfo& inf, float* save) {
    const RolloutArgs& a = g.r;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int Np = a.Np;
    const float2 e = control_eps((uint32_t)k, (uint32_t)(act ? s : 0), a.it0, a.it1, a.key0, a.key1,
                                 a.sig_v, a.sig_w);
    const float rx = __ldg(a.U + 2 * k) + e.x, ry = __ldg(a.U + 2 * k + 1) + e.y;
    inf.ux = fminf(fmaxf(rx, a.umin0), a.umax0);
    inf.uy = fminf(fmaxf(ry, a.umin1), a.umax1);
    inf.mask = ((rx > a.umin0 && rx < a.umax0) ? 1 : 0) | ((ry > a.umin1 && ry < a.umax1) ? 2 : 0);
    const float z0 = mu[3] * a.zscale[0], z1 = mu[4] * a.zscale[1], z2 = inf.ux * a.zscale[2],
                z3 = inf.uy * a.zscale[3];
    float mv = 0.0f, mw = 0.0f, cv = 0.0f, cw = 0.0f;
    for (int j = lane; j < Np; j += 32) {
        float kv = 0.0f;
        if (act && j < a.N) {
            const float4 x = ldg4(a.Xs + 4 * j);
            const float d0 = z0 - x.x, d1 = z1 - x.y, d2 = z2 - x.z, d3 = z3 - x.w;
            kv = a.sf2 * exp2f(-(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3));
            const float2 al = __ldg(reinterpret_cast<const float2*>(a.alpha) + j);
            kahan_add(mv, cv, kv * al.x);
            kahan_add(mw, cw, kv * al.y);
        }
        kT[j * GMT + w] = kv;
    }
    mv = wsum(mv + cv);
    mw = wsum(mw + cw);
    // the warp's state waits in shared memory while the product runs, so that
    // its registers are free for the product's tiles
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) save[i] = mu[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) save[5 + i] = S[i];
        save[20] = mv;
        save[21] = mw;
        save[22] = inf.ux;
        save[23] = inf.uy;
        save[24] = __int_as_float(inf.mask);
    }
    __syncthreads();
    tri_product<false>(a.W, Np, kT, vT);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 5; ++i) mu[i] = save[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) S[i] = save[5 + i];
    mv = save[20];
    mw = save[21];
    inf.ux = save[22];
    inf.uy = save[23];
    inf.mask = __float_as_int(save[24]);
    float q = 0.0f;
    for (int i = lane; i < Np; i += 32) {
        const float x = vT[i * GMT + w];
        q = fmaf(x, x, q);
    }
    q = wsum(q);
    if (vstore) {
        const float4* src = reinterpret_cast<const float4*>(vT);
        float4* dst = reinterpret_cast<float4*>(vstore);
        for (int i = tid; i < Np * GMT / 4; i += GT) dst[i] = src[i];
    }
    inf.sraw = a.sf2 - q;
    const float sv = fmaxf(0.0f, inf.sraw);

    float sn, cs;
    sincosf(mu[2], &sn, &cs);
    const float a02 = -a.dt * mu[3] * sn, a03 = a.dt * cs;
    const float a12 = a.dt * mu[3] * cs, a13 = a.dt * sn;
    const float nX = mu[0] + a.dt * mu[3] * cs;
    const float nY = mu[1] + a.dt * mu[3] * sn;
    const float nT = mu[2] + a.dt * mu[4];
    const float nV = mu[3] + a.kv * (inf.ux - mu[3]) + mv;
    const float nW = mu[4] + a.kw * (inf.uy - mu[4]) + mw;
    mu[0] = nX; mu[1] = nY; mu[2] = nT; mu[3] = nV; mu[4] = nW;
    // Sigma' = A Sigma A^T + diag(0, 0, 0, s, s)  (Eq. 10)
    float A[5][5] = {{1.f, 0.f, a02, a03, 0.f},
                     {0.f, 1.f, a12, a13, 0.f},
                     {0.f, 0.f, 1.f, 0.f, a.dt},
                     {0.f, 0.f, 0.f, a.av, 0.f},
                     {0.f, 0.f, 0.f, 0.f, a.aw}};
    float Sf[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) Sf[i][j] = (i <= j) ? S[sidx(i, j)] : S[sidx(j, i)];
    float B[5][5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            float t = 0.0f;
#pragma unroll
            for (int m = 0; m < 5; ++m) t = fmaf(A[i][m], Sf[m][j], t);
            B[i][j] = t;
        }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) {
            float t = 0.0f;
#pragma unroll
            for (int m = 0; m < 5; ++m) t = fmaf(B[i][m], A[j][m], t);
            S[sidx(i, j)] = t;
        }
    S[sidx(3, 3)] += sv;
    S[sidx(4, 4)] += sv;
}

// Smoothed stage cost at the post-step state (warp-wide, lane-replicated).
__device__ float stage_cost(const GradArgs& g, int k, const float mu[5], const float S[15], float sraw) {
    const RolloutArgs& a = g.r;
    const float s = fmaxf(0.0f, sraw);
    float best;
    int bi;
    lane_nearest(a, mu[0], mu[1], best, bi);
    const float e = sqrtf(best);
    const Lam L = lam_max(S[sidx(0, 0)], S[sidx(0, 1)], S[sidx(1, 1)]);
    const float rbar = a.r - a.sq_chi2 * L.sq;                               // Eq. 14
    const float disc = exp2f((float)k * log2f(0.9f));
    float c = a.c_var * (s + s) + a.c_speed * (a.v_des - mu[3]) * (a.v_des - mu[3]) + a.c_dev * e +
              a.c_lane * disc * sigm(g.slope * (e - rbar));
    if (a.O > 0) {
        float om;
        int oi;
        obstacle_nearest(a, mu[0], mu[1], S[sidx(0, 0)], S[sidx(0, 1)], S[sidx(1, 1)], L.sq, om, oi);
        c += a.c_coll * sigm(-g.slope * om);
    }
    if (a.c_goal != 0.0f || a.c_term != 0.0f) {          // Eq. 12 goal terms, F smoothed
        const float dx = mu[0] - a.goal_x, dy = mu[1] - a.goal_y;
        const float d = sqrtf(dx * dx + dy * dy);
        c += a.c_goal * d;
        if (k == a.T - 1) c += a.c_term * sigm(g.slope * (d - a.goal_r));
    }
    return c;
}

// Adjoint of the smoothed stage cost at the post-step state, scaled by wt,
// added to the post-state adjoints mub (mean) and Sb (Sigma, stored upper
// triangle: the derivative with respect to each stored entry).  Returns the
// derivative with respect to the GP variance of each output.
__device__ float stage_cost_adjoint(const GradArgs& g, int k, const float mu[5], const float S[15],
                                    float wt, float mub[5], float Sb[15]) {
    const RolloutArgs& a = g.r;
    const float sxx = S[sidx(0, 0)], sxy = S[sidx(0, 1)], syy = S[sidx(1, 1)];
    const Lam L = lam_max(sxx, sxy, syy);
    float gX = 0.0f, gY = 0.0f, gxx = 0.0f, gxy = 0.0f, gyy = 0.0f;
    // lane deviation and tightened lane indicator (Eq. 11, 13-14)
    float best;
    int bi;
    lane_nearest(a, mu[0], mu[1], best, bi);
    const float e = sqrtf(best);
    float ex = 0.0f, ey = 0.0f;              // d e / d (X, Y)
    if (e > 0.0f && bi < a.S) {
        const float4 sg = __ldg(a.seg + bi);
        const float il2 = __ldg(a.seg_il2 + bi);
        const float qx0 = mu[0] - sg.x, qy0 = mu[1] - sg.y;
        const float t = fminf(fmaxf((qx0 * sg.z + qy0 * sg.w) * il2, 0.0f), 1.0f);
        ex = (qx0 - t * sg.z) / e;
        ey = (qy0 - t * sg.w) / e;
    }
    const float disc = exp2f((float)k * log2f(0.9f));
    const float sl = sigm(g.slope * (e - (a.r - a.sq_chi2 * L.sq)));
    const float gl = a.c_lane * disc * g.slope * sl * (1.0f - sl);    // d cost / d lane margin
    gX += (a.c_dev + gl) * ex;
    gY += (a.c_dev + gl) * ey;
    gxx += gl * a.sq_chi2 * L.dxx;
    gxy += gl * a.sq_chi2 * L.dxy;
    gyy += gl * a.sq_chi2 * L.dyy;
    // collision indicator (Eq. 12, 15-16) through the nearest tightened obstacle
    if (a.O > 0) {
        float om;
        int oi;
        obstacle_nearest(a, mu[0], mu[1], sxx, sxy, syy, L.sq, om, oi);
        const float sc = sigm(-g.slope * om);
        const float gc = -a.c_coll * g.slope * sc * (1.0f - sc);      // d cost / d margin
        if (oi < a.O) {
            const float cx = __ldg(a.obst + 3 * oi), cy = __ldg(a.obst + 3 * oi + 1);
            const float dx = mu[0] - cx, dy = mu[1] - cy;
            const float rho = sqrtf(dx * dx + dy * dy);
            if (rho > 1e-9f) {
                const float nx = dx / rho, ny = dy / rho;
                const float qn = nx * nx * sxx + 2.0f * nx * ny * sxy + ny * ny * syy;
                const float sp = sqrtf(fmaxf(0.0f, qn));
                float mx = nx, my = ny;           // d margin / d (X, Y)
                if (sp > 0.0f) {
                    const float snx = sxx * nx + sxy * ny, sny = sxy * nx + syy * ny;
                    mx -= a.phi_inv * (snx - qn * nx) / (rho * sp);
                    my -= a.phi_inv * (sny - qn * ny) / (rho * sp);
                    const float f = -a.phi_inv * 0.5f / sp;
                    gxx += gc * f * nx * nx;
                    gxy += gc * f * 2.0f * nx * ny;
                    gyy += gc * f * ny * ny;
                }
                gX += gc * mx;
                gY += gc * my;
            } else {
                gxx += gc * (-a.phi_inv) * L.dxx;
                gxy += gc * (-a.phi_inv) * L.dxy;
                gyy += gc * (-a.phi_inv) * L.dyy;
            }
        }
    }
    if (a.c_goal != 0.0f || a.c_term != 0.0f) {
        const float dx = mu[0] - a.goal_x, dy = mu[1] - a.goal_y;
        const float d = sqrtf(dx * dx + dy * dy);
        if (d > 0.0f) {
            float gd = a.c_goal;                            // d cost / d distance
            if (k == a.T - 1) {
                const float sg = sigm(g.slope * (d - a.goal_r));
                gd += a.c_term * g.slope * sg * (1.0f - sg);
            }
            gX += gd * dx / d;
            gY += gd * dy / d;
        }
    }
    mub[0] += wt * gX;
    mub[1] += wt * gY;
    mub[3] += wt * (-2.0f * a.c_speed * (a.v_des - mu[3]));
    Sb[sidx(0, 0)] += wt * gxx;
    Sb[sidx(0, 1)] += wt * gxy;
    Sb[sidx(1, 1)] += wt * gyy;
    return wt * a.c_var;
}

constexpr int SAVE = 40;     // per-warp spill area for state live across a product
constexpr int CARRY = 28;    // per-warp adjoint carry: mu_bar (5), Sigma_bar (15), l_bar (8)

__global__ void __launch_bounds__(GT, 2) k_grad(const GradArgs g) {
    extern __shared__ __align__(16) float gsm[];
    const RolloutArgs& a = g.r;
    const int Np = a.Np, C = g.C, T = a.T;
    float* bufA = gsm;
    float* bufB = bufA + Np * GMT;
    float* rec = bufB + Np * GMT;                                   // (C + 1) x GMT x REC
    StepInfo* info = reinterpret_cast<StepInfo*>(rec + (C + 1) * GMT * REC);   // C x GMT
    float* saves = reinterpret_cast<float*>(info + C * GMT);        // GMT x SAVE
    float* carries = saves + GMT * SAVE;                            // GMT x CARRY
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    float* save = saves + w * SAVE;
    float* carry = carries + w * CARRY;
    const int s = blockIdx.x * GMT + w;
    const bool act = s < a.K;
    const float wt = act ? (g.weight ? __ldg(g.weight + s) : g.inv_K) : 0.0f;
    float* ck = g.ckpt + ((size_t)blockIdx.x * g.nseg * GMT + w) * REC;   // + seg * GMT * REC

    float mu[5], S[15];
#pragma unroll
    for (int i = 0; i < 5; ++i) mu[i] = a.x0[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) S[i] = 0.0f;

    // ---- pass 1: objective and checkpoints --------------------------------
    float Jsum = 0.0f, Jc = 0.0f;
    for (int k = 0; k < T; ++k) {
        if (k % C == 0 && lane == 0) {
            float* dst = ck + (size_t)(k / C) * GMT * REC;
#pragma unroll
            for (int i = 0; i < 5; ++i) dst[i] = mu[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) dst[5 + i] = S[i];
        }
        StepInfo inf;
        fwd_step(g, k, s, act, mu, S, bufA, bufB, nullptr, inf, save);
        if (act) kahan_add(Jsum, Jc, stage_cost(g, k, mu, S, inf.sraw));
    }
    if (act && lane == 0) g.S_out[s] = Jsum + Jc;
    if (!g.backward) return;
    if (lane == 0)
        for (int i = 0; i < CARRY; ++i) carry[i] = 0.0f;
    __syncthreads();     // checkpoint stores and the zeroed carry before the reloads below

    // ---- passes 2 and 3, one segment at a time, last segment first --------
    float* vslot = g.vscr + (size_t)blockIdx.x * C * Np * GMT;
    for (int sg = g.nseg - 1; sg >= 0; --sg) {
        const int k0 = sg * C;
        const int len = min(C, T - k0);
        {
            const float* src = ck + (size_t)sg * GMT * REC;
#pragma unroll
            for (int i = 0; i < 5; ++i) mu[i] = src[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) S[i] = src[5 + i];
        }
        if (lane == 0) {
            float* r0 = rec + w * REC;
#pragma unroll
            for (int i = 0; i < 5; ++i) r0[i] = mu[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) r0[5 + i] = S[i];
        }
        for (int t = 0; t < len; ++t) {
            StepInfo inf;
            fwd_step(g, k0 + t, s, act, mu, S, bufA, bufB, vslot + (size_t)t * Np * GMT, inf, save);
            if (lane == 0) {
                float* r1 = rec + ((t + 1) * GMT + w) * REC;
#pragma unroll
                for (int i = 0; i < 5; ++i) r1[i] = mu[i];
#pragma unroll
                for (int i = 0; i < 15; ++i) r1[5 + i] = S[i];
                info[t * GMT + w] = inf;
            }
        }
        __syncthreads();
        for (int t = len - 1; t >= 0; --t) {
            const int k = k0 + t;
            const float* pre = rec + (t * GMT + w) * REC;
            const float* post = rec + ((t + 1) * GMT + w) * REC;
            float mub[5], Sb[15];
#pragma unroll
            for (int i = 0; i < 5; ++i) mub[i] = carry[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) Sb[i] = carry[5 + i];
            float sbv = 0.0f, sbw = 0.0f;
            {
                float m1[5], S1[15];
#pragma unroll
                for (int i = 0; i < 5; ++i) m1[i] = post[i];
#pragma unroll
                for (int i = 0; i < 15; ++i) S1[i] = post[5 + i];
                // stage cost of step k (scored on the post-step state)
                if (act) {
                    const float gs = stage_cost_adjoint(g, k, m1, S1, wt, mub, Sb);
                    sbv = gs;
                    sbw = gs;
                }
            }
            float m0[5], S0[15];
#pragma unroll
            for (int i = 0; i < 5; ++i) m0[i] = pre[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) S0[i] = pre[5 + i];
            // covariance adjoint: Sigma' = A Sigma A^T + diag(0,0,0,s,s)
            sbv += Sb[sidx(3, 3)];
            sbw += Sb[sidx(4, 4)];
            float sn, cs;
            sincosf(m0[2], &sn, &cs);
            const float v0 = m0[3];
            const float a02 = -a.dt * v0 * sn, a03 = a.dt * cs, a12 = a.dt * v0 * cs, a13 = a.dt * sn;
            const float A[5][5] = {{1.f, 0.f, a02, a03, 0.f},
                                   {0.f, 1.f, a12, a13, 0.f},
                                   {0.f, 0.f, 1.f, 0.f, a.dt},
                                   {0.f, 0.f, 0.f, a.av, 0.f},
                                   {0.f, 0.f, 0.f, 0.f, a.aw}};
            float G[5][5], Sf[5][5];
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const int id = (i <= j) ? sidx(i, j) : sidx(j, i);
                    G[i][j] = (i == j) ? Sb[id] : 0.5f * Sb[id];
                    Sf[i][j] = S0[id];
                }
            float GA[5][5];
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    float t2 = 0.0f;
#pragma unroll
                    for (int m = 0; m < 5; ++m) t2 = fmaf(G[i][m], A[m][j], t2);
                    GA[i][j] = t2;
                }
            // A_bar = 2 G A Sigma at the entries of A that depend on the state
            float Ab02 = 0.f, Ab03 = 0.f, Ab12 = 0.f, Ab13 = 0.f;
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                Ab02 = fmaf(GA[0][m], Sf[m][2], Ab02);
                Ab03 = fmaf(GA[0][m], Sf[m][3], Ab03);
                Ab12 = fmaf(GA[1][m], Sf[m][2], Ab12);
                Ab13 = fmaf(GA[1][m], Sf[m][3], Ab13);
            }
            Ab02 *= 2.0f; Ab03 *= 2.0f; Ab12 *= 2.0f; Ab13 *= 2.0f;
            // Sigma_bar = A^T G A, returned to the stored-entry convention
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = i; j < 5; ++j) {
                    float t2 = 0.0f;
#pragma unroll
                    for (int m = 0; m < 5; ++m) t2 = fmaf(A[m][i], GA[m][j], t2);
                    Sb[sidx(i, j)] = (i == j) ? t2 : 2.0f * t2;
                }
            // mean adjoint (Eq. 6 with the GP mean), with the A_bar terms
            const float mbv = mub[3], mbw = mub[4];
            float nm[5];
            nm[0] = mub[0];
            nm[1] = mub[1];
            nm[2] = mub[2] + mub[0] * (-a.dt * v0 * sn) + mub[1] * (a.dt * v0 * cs) +
                    Ab02 * (-a.dt * v0 * cs) + Ab03 * (-a.dt * sn) + Ab12 * (-a.dt * v0 * sn) +
                    Ab13 * (a.dt * cs);
            nm[3] = mub[0] * (a.dt * cs) + mub[1] * (a.dt * sn) + mub[3] * a.av +
                    Ab02 * (-a.dt * sn) + Ab12 * (a.dt * cs);
            nm[4] = mub[2] * a.dt + mub[4] * a.aw;
            const StepInfo inf0 = info[t * GMT + w];
            if (!(inf0.sraw > 0.0f)) {       // variance clamped at zero: no gradient through it
                sbv = 0.0f;
                sbw = 0.0f;
            }
            // the adjoints wait in shared memory while the product runs
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < 5; ++i) save[i] = nm[i];
#pragma unroll
                for (int i = 0; i < 15; ++i) save[5 + i] = Sb[i];
                save[20] = sbv;
                save[21] = sbw;
                save[22] = mbv;
                save[23] = mbw;
            }
            // b = L^-T v = K^-1 k* for all samples of the CTA
            {
                const float4* src = reinterpret_cast<const float4*>(vslot + (size_t)t * Np * GMT);
                float4* dst = reinterpret_cast<float4*>(bufA);
                for (int i = tid; i < Np * GMT / 4; i += GT) dst[i] = src[i];
            }
            __syncthreads();
            tri_product<true>(g.Wt, Np, bufA, bufB);
            __syncthreads();
            const float sbv2 = save[20], sbw2 = save[21], mbv2 = save[22], mbw2 = save[23];
            if (g.Bq) {
                // b_q for the Gram contraction G_o = sum_q sbar_o,q b_q b_q^T (the
                // adjoints sbar go with it in qbar; a padding sample's are zero)
                const size_t q0 = (size_t)k * g.Kpad + (size_t)blockIdx.x * GMT;
                for (int ws = 0; ws < GMT; ++ws) {
                    float* dst = g.Bq + (q0 + ws) * Np;
                    for (int j = tid; j < Np; j += GT) dst[j] = bufB[j * GMT + ws];
                }
                if (lane == 0)
                    g.qbar[q0 + w] = act ? make_float4(mbv2, mbw2, sbv2, sbw2) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // GP adjoint: z_bar and the lengthscale terms
            float nv3 = save[3], nv4 = save[4];
            if (act) {
                const StepInfo inf = info[t * GMT + w];
                float ubx = mbv2 * a.kv, uby = mbw2 * a.kw;
                const float z0 = pre[3] * a.zscale[0], z1 = pre[4] * a.zscale[1],
                            z2 = inf.ux * a.zscale[2], z3 = inf.uy * a.zscale[3];
                float zb[4] = {0.f, 0.f, 0.f, 0.f};
                float lb[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int j = lane; j < a.N; j += 32) {
                    const float4 x = ldg4(a.Xs + 4 * j);
                    const float d[4] = {z0 - x.x, z1 - x.y, z2 - x.z, z3 - x.w};
                    const float kj = a.sf2 * exp2f(-(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3]));
                    const float bj = bufB[j * GMT + w];
                    const float2 al = __ldg(reinterpret_cast<const float2*>(a.alpha) + j);
                    const float wv = kj * (mbv2 * al.x - 2.0f * sbv2 * bj);
                    const float ww = kj * (mbw2 * al.y - 2.0f * sbw2 * bj);
                    const float wz = wv + ww;
#pragma unroll
                    for (int dd = 0; dd < 4; ++dd) {
                        zb[dd] = fmaf(wz, d[dd], zb[dd]);
                        const float d2 = d[dd] * d[dd];
                        lb[dd] = fmaf(wv, d2, lb[dd]);
                        lb[4 + dd] = fmaf(ww, d2, lb[4 + dd]);
                    }
                    if (g.ubar) {
#pragma unroll
                        for (int dd = 0; dd < 4; ++dd) {
                            lb[dd] = fmaf(-mbv2 * bj, __ldg(g.ubar + (size_t)dd * Np + j), lb[dd]);
                            lb[4 + dd] = fmaf(-mbw2 * bj, __ldg(g.ubar + (size_t)(4 + dd) * Np + j), lb[4 + dd]);
                        }
                    }
                }
#pragma unroll
                for (int dd = 0; dd < 4; ++dd) zb[dd] = -2.0f * kLn2 * a.zscale[dd] * wsum(zb[dd]);
#pragma unroll
                for (int i = 0; i < 8; ++i) lb[i] = wsum(lb[i]);
                nv3 += zb[0];
                nv4 += zb[1];
                ubx += zb[2];
                uby += zb[3];
                if (lane == 0) {
                    g.dU_out[(size_t)(2 * k) * a.K + s] = (inf.mask & 1) ? ubx : 0.0f;
                    g.dU_out[(size_t)(2 * k + 1) * a.K + s] = (inf.mask & 2) ? uby : 0.0f;
#pragma unroll
                    for (int i = 0; i < 8; ++i) carry[20 + i] += lb[i];
                }
            }
            // carry the pre-step adjoints to step k - 1
            __syncwarp();
            if (lane == 0) {
                carry[0] = save[0];
                carry[1] = save[1];
                carry[2] = save[2];
                carry[3] = nv3;
                carry[4] = nv4;
#pragma unroll
                for (int i = 0; i < 15; ++i) carry[5 + i] = save[5 + i];
            }
            __syncwarp();
        }
        __syncthreads();     // rec / info / scratch reuse by the next segment
    }
    if (act && lane == 0 && g.dl_out) {
#pragma unroll
        for (int i = 0; i < 8; ++i) g.dl_out[(size_t)i * a.K + s] = carry[20 + i];
    }
}

// ---- Gram trace: sum_ij dK/dl_d[i][j] G_o[i][j], G_o = sum_q sbar_o,q b_q b_q^T ----
// tr(D_d G_o) for d = 0..3, o = v, w, with D_d[i][j] = sf2 2^-|xs_i - xs_j|^2
// (xs_id - xs_jd)^2 (dK/dl_d up to the factor 2 ln2 / l_d) and G = [G_v; G_w]
// (2 Np x Np, column-major, symmetric blocks): warp w of block b takes column
// j = 8 b + w, lanes the rows i (coalesced); 8 partial sums per block.
// ubar[(o*4+d)][i] = sum_j Kf_ij (xs_id - xs_jd)^2 alpha_o[j]: (dK/dl_d) alpha_o
// up to the factor 2 ln2 / l_d; one warp per row i.
__global__ void k_dk_alpha(const float* __restrict__ Xs, const float* __restrict__ alpha, int N, int Np,
                           float sf2, float* __restrict__ ubar) {
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= Np) return;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < N) {
        const float4 xi = ldg4(Xs + 4 * i);
        for (int j = lane; j < N; j += 32) {
            const float4 xj = ldg4(Xs + 4 * j);
            const float d[4] = {xi.x - xj.x, xi.y - xj.y, xi.z - xj.z, xi.w - xj.w};
            const float dd[4] = {d[0] * d[0], d[1] * d[1], d[2] * d[2], d[3] * d[3]};
            const float kf = sf2 * exp2f(-(dd[0] + dd[1] + dd[2] + dd[3]));
            const float2 al = __ldg(reinterpret_cast<const float2*>(alpha) + j);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                acc[e] = fmaf(kf * dd[e], al.x, acc[e]);
                acc[4 + e] = fmaf(kf * dd[e], al.y, acc[4 + e]);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float v = wsum(acc[e]);
        if (lane == 0) ubar[(size_t)e * Np + i] = v;
    }
}

// Wt[i][j] = W[j][i]: rows of L^-1 from rows of L^-T
__global__ void k_transpose(const float* __restrict__ W, int Np, float* __restrict__ Wt) {
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int x = bx + threadIdx.x;
    for (int r = threadIdx.y; r < 32; r += 8)
        if (by + r < Np && x < Np) tile[r][threadIdx.x] = W[(size_t)(by + r) * Np + x];
    __syncthreads();
    const int y = by + threadIdx.x;
    for (int r = threadIdx.y; r < 32; r += 8)
        if (bx + r < Np && y < Np) Wt[(size_t)(bx + r) * Np + y] = tile[threadIdx.x][r];
}

// Final reductions in double, fixed order: blocks [0, 2T) -> dU, block 2T -> J,
// blocks 2T+1 .. 2T+8 -> dl (when requested).
__global__ void k_grad_reduce(const GradReduceArgs r) {
    __shared__ double red[256];
    const int b = blockIdx.x, tid = threadIdx.x;
    double acc = 0.0;
    float* dst = nullptr;
    double scale = 1.0;
    if (b < 2 * r.T) {
        for (int s = tid; s < r.K; s += 256) acc += (double)r.dU_out[(size_t)b * r.K + s];
        dst = r.dU + b;
    } else if (b == 2 * r.T) {
        for (int s = tid; s < r.K; s += 256)
            acc += (double)(r.weight ? r.weight[s] : r.inv_K) * (double)r.S_out[s];
        dst = r.J;
    } else {
        const int e = b - 2 * r.T - 1;
        for (int s = tid; s < r.K; s += 256) acc += (double)r.dl_out[(size_t)e * r.K + s];
        for (int p = tid; p < r.nparts; p += 256) acc += (double)r.parts[(size_t)p * 8 + e];
        dst = r.dl + e;
        scale = 2.0 * 0.69314718055994530942 / r.ell[e & 3];
    }
    red[tid] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0 && dst) *dst = (float)(red[0] * scale);
}

}  // namespace

int grad_smem_bytes(int Np, int C) {
    return (int)(sizeof(float) * (2 * (size_t)Np * GMT + (size_t)(C + 1) * GMT * REC) +
                 sizeof(StepInfo) * (size_t)C * GMT + sizeof(float) * GMT * (SAVE + CARRY));
}

int grad_samples_per_cta() { return GMT; }

int launch_grad(const GradArgs& g, int ncta, cudaStream_t st) {
    const int smem = grad_smem_bytes(g.r.Np, g.C);
    GPM_CUDA(cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_grad<<<ncta, GT, smem, st>>>(g);
    GPM_CUDA(cudaGetLastError());
    return 0;
}

int launch_dk_alpha(const float* Xs, const float* alpha, int N, int Np, float sf2, float* ubar,
                    cudaStream_t st) {
    k_dk_alpha<<<(Np + 7) / 8, 256, 0, st>>>(Xs, alpha, N, Np, sf2, ubar);
    GPM_CUDA(cudaGetLastError());
    return 0;
}

int launch_transpose(const float* W, int Np, float* Wt, cudaStream_t st) {
    k_transpose<<<dim3((Np + 31) / 32, (Np + 31) / 32), dim3(32, 8), 0, st>>>(W, Np, Wt);
    GPM_CUDA(cudaGetLastError());
    return 0;
}

int launch_grad_reduce(const GradReduceArgs& r, cudaStream_t st) {
    const int nb = 2 * r.T + 1 + (r.dl ? 8 : 0);
    k_grad_reduce<<<nb, 256, 0, st>>>(r);
    GPM_CUDA(cudaGetLastError());
    return 0;
}

}  // namespace gpm
