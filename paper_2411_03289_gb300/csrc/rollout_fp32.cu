// Fused MPPI rollout, FP32 on the CUDA cores (Alg. 1 Step 1).
//
// One CTA owns `mt` samples and carries them through all T steps of the
// horizon (the recurrence of Eq. 10 is sequential in k).  Per step k:
//   P1  (warp 0, lane = sample) Philox noise, clamp (Eq. 8), GP query z
//   P2  (all)  k*_j = sf2 exp(-|z - x_j|^2 / 2l^2) into shared memory, and the
//              mean partials k* . alpha (Eq. 3)
//   P3  (all)  V = K* L^-T as a register-tiled triangular product; each thread
//              squares and sums its tile, giving partial |L^-1 k*|^2
//   P4  (warp 0) GP mean / variance, mean dynamics (Eq. 6, 10), covariance
//              A Sigma A^T + diag(0,0,0,s,s) (Eq. 10), obstacle chance
//              constraint (Eq. 15-16), variance and speed terms (Eq. 11-12)
//   P5  (all)  distance to the lane polyline, split over segments
//   P6  (warp 0) lane deviation and tightened lane indicator (Eq. 11, 13-14)
// The triangular product dominates: N(N+1)/2 FMAs per sample-step.
#include <cfloat>

#include "common.cuh"

namespace gpm {
namespace {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

template <int MTP>
struct Smem {
    // byte offsets inside the dynamic shared buffer
    static __host__ __device__ int ks(int) { return 0; }
    static __host__ __device__ int qpart(int Np) { return Np * MTP * 4; }
    static __host__ __device__ int mpart(int Np) { return qpart(Np) + (Np / 16) * MTP * 4; }
    static __host__ __device__ int epart(int Np) { return mpart(Np) + THREADS * 8; }
    static __host__ __device__ int zq(int Np) { return epart(Np) + THREADS * 4; }
    static __host__ __device__ int pos(int Np) { return zq(Np) + MTP * 16; }
    static __host__ __device__ int total(int Np) { return pos(Np) + MTP * 8; }
};

template <int MTP, bool TRACE>
__global__ void __launch_bounds__(THREADS, 1) k_rollout_fp32(const RolloutArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Np = a.Np;
    float* Ks = reinterpret_cast<float*>(smem_raw + Smem<MTP>::ks(Np));
    float* qpart = reinterpret_cast<float*>(smem_raw + Smem<MTP>::qpart(Np));
    float2* mpart = reinterpret_cast<float2*>(smem_raw + Smem<MTP>::mpart(Np));
    float* epart = reinterpret_cast<float*>(smem_raw + Smem<MTP>::epart(Np));
    float4* zq = reinterpret_cast<float4*>(smem_raw + Smem<MTP>::zq(Np));
    float2* pos = reinterpret_cast<float2*>(smem_raw + Smem<MTP>::pos(Np));

    constexpr int SUB = 32 / MTP;          // lanes sharing one sample in P2 / P5
    constexpr int NMG = MTP / 4;           // 4-sample groups in P3
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s0 = blockIdx.x * a.mt;
    const int mvalid = min(a.mt, a.K - s0);
    const int npairs = Np / 16;
    const int items = NMG * npairs;

    // per-sample state, live in warp 0 lanes < MTP
    const bool owner = (warp == 0) && (lane < MTP);
    const bool active = owner && (lane < mvalid);
    const int s_me = s0 + ((lane < mvalid) ? lane : 0);
    float mu0 = a.x0[0], mu1 = a.x0[1], mu2 = a.x0[2], mu3 = a.x0[3], mu4 = a.x0[4];
    // symmetric Sigma, upper triangle
    float S00 = 0, S01 = 0, S02 = 0, S03 = 0, S04 = 0, S11 = 0, S12 = 0, S13 = 0, S14 = 0,
          S22 = 0, S23 = 0, S24 = 0, S33 = 0, S34 = 0, S44 = 0;
    float cost = 0.0f, disc = 1.0f, stage = 0.0f, rbar = 0.0f, omargin = FLT_MAX;
    float2 ut = make_float2(0.f, 0.f);

    for (int k = 0; k < a.T; ++k) {
        // ---------------- P1: noise, clamp, query --------------------------
        if (owner) {
            const float2 e = control_eps((uint32_t)k, (uint32_t)s_me, a.it0, a.it1, a.key0, a.key1,
                                         a.sig_v, a.sig_w);
            ut.x = fminf(fmaxf(__ldg(a.U + 2 * k) + e.x, a.umin0), a.umax0);
            ut.y = fminf(fmaxf(__ldg(a.U + 2 * k + 1) + e.y, a.umin1), a.umax1);
            zq[lane] = make_float4(mu3 * a.zscale[0], mu4 * a.zscale[1], ut.x * a.zscale[2],
                                   ut.y * a.zscale[3]);
            if (active) a.u_tilde[(size_t)k * a.K + s_me] = ut;
        }
        __syncthreads();

        // ---------------- P2: kernel row and mean partials ----------------
        {
            const int m = lane % MTP;
            const float4 z = zq[m];
            float mv = 0.0f, mw = 0.0f;
            for (int j = warp * SUB + lane / MTP; j < Np; j += THREADS / MTP) {
                float kv = 0.0f;
                if (j < a.N) {
                    const float4 x = ldg4(a.Xs + 4 * j);
                    const float e0 = z.x - x.x, e1 = z.y - x.y, e2 = z.z - x.z, e3 = z.w - x.w;
                    kv = a.sf2 * exp2f(-(e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3));
                    const float2 al = __ldg(reinterpret_cast<const float2*>(a.alpha) + j);
                    mv = fmaf(kv, al.x, mv);
                    mw = fmaf(kv, al.y, mw);
                }
                Ks[j * MTP + m] = kv;
            }
            mpart[tid] = make_float2(mv, mw);
        }
        __syncthreads();

        // ---------------- P3: |L^-1 k*|^2 by a triangular product ----------
        for (int it = tid; it < items; it += THREADS) {
            const int mg = it % NMG;
            const int p = it / NMG;
            const int colA = 8 * p;
            const int colB = Np - 8 - 8 * p;
            // warp-uniform trip counts: extra rows of W are zero (upper part)
            const unsigned am = __activemask();
            const int endA = __reduce_max_sync(am, colA + 8);
            const int endB = __reduce_max_sync(am, colB + 8);
            float accA[4][8], accB[4][8];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    accA[r][c] = 0.0f;
                    accB[r][c] = 0.0f;
                }
            const float* kp = Ks + 4 * mg;
            const float* wA = a.W + colA;
            const float* wB = a.W + colB;
#pragma unroll 2
            for (int j = 0; j < endA; ++j) {
                const float4 kv = *reinterpret_cast<const float4*>(kp + j * MTP);
                const float4 a0 = ldg4(wA + (size_t)j * Np), a1 = ldg4(wA + (size_t)j * Np + 4);
                const float4 b0 = ldg4(wB + (size_t)j * Np), b1 = ldg4(wB + (size_t)j * Np + 4);
                const float kr[4] = {kv.x, kv.y, kv.z, kv.w};
                const float wa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float wb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        accA[r][c] = fmaf(kr[r], wa[c], accA[r][c]);
                        accB[r][c] = fmaf(kr[r], wb[c], accB[r][c]);
                    }
            }
#pragma unroll 4
            for (int j = endA; j < endB; ++j) {
                const float4 kv = *reinterpret_cast<const float4*>(kp + j * MTP);
                const float4 b0 = ldg4(wB + (size_t)j * Np), b1 = ldg4(wB + (size_t)j * Np + 4);
                const float kr[4] = {kv.x, kv.y, kv.z, kv.w};
                const float wb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) accB[r][c] = fmaf(kr[r], wb[c], accB[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float q = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    q = fmaf(accA[r][c], accA[r][c], q);
                    q = fmaf(accB[r][c], accB[r][c], q);
                }
                qpart[p * MTP + 4 * mg + r] = q;
            }
        }
        __syncthreads();

        // ---------------- P4: dynamics, covariance, obstacles --------------
        if (owner) {
            const int m = lane;
            float mv = 0.0f, mw = 0.0f;
            for (int w = 0; w < WARPS; ++w)
#pragma unroll
                for (int u = 0; u < SUB; ++u) {
                    const float2 pm = mpart[w * 32 + u * MTP + m];
                    mv += pm.x;
                    mw += pm.y;
                }
            float q = 0.0f;
            for (int p = 0; p < npairs; ++p) q += qpart[p * MTP + m];
            const float s = fmaxf(0.0f, a.sf2 - q);

            // Jacobian of the nominal model at the pre-step mean (Eq. 10)
            float sn, cs;
            sincosf(mu2, &sn, &cs);
            const float a02 = -a.dt * mu3 * sn, a03 = a.dt * cs;
            const float a12 = a.dt * mu3 * cs, a13 = a.dt * sn;
            // mean update (Eq. 6 with the GP mean)
            const float nX = mu0 + a.dt * mu3 * cs;
            const float nY = mu1 + a.dt * mu3 * sn;
            const float nT = mu2 + a.dt * mu4;
            const float nV = mu3 + a.kv * (ut.x - mu3) + mv;
            const float nW = mu4 + a.kw * (ut.y - mu4) + mw;
            mu0 = nX; mu1 = nY; mu2 = nT; mu3 = nV; mu4 = nW;

            // B = A Sigma (rows), then Sigma' = B A^T + diag(0,0,0,s,s)
            const float B00 = S00 + a02 * S02 + a03 * S03, B01 = S01 + a02 * S12 + a03 * S13,
                        B02 = S02 + a02 * S22 + a03 * S23, B03 = S03 + a02 * S23 + a03 * S33,
                        B04 = S04 + a02 * S24 + a03 * S34;
            const float B11 = S11 + a12 * S12 + a13 * S13, B12 = S12 + a12 * S22 + a13 * S23,
                        B13 = S13 + a12 * S23 + a13 * S33, B14 = S14 + a12 * S24 + a13 * S34;
            const float B22 = S22 + a.dt * S24, B23 = S23 + a.dt * S34, B24 = S24 + a.dt * S44;
            const float B33 = a.av * S33, B34 = a.av * S34;
            const float B44 = a.aw * S44;
            S00 = B00 + a02 * B02 + a03 * B03;
            S01 = B01 + a12 * B02 + a13 * B03;
            S02 = B02 + a.dt * B04;
            S03 = a.av * B03;
            S04 = a.aw * B04;
            S11 = B11 + a12 * B12 + a13 * B13;
            S12 = B12 + a.dt * B14;
            S13 = a.av * B13;
            S14 = a.aw * B14;
            S22 = B22 + a.dt * B24;
            S23 = a.av * B23;
            S24 = a.aw * B24;
            S33 = a.av * B33 + s;
            S34 = a.aw * B34;
            S44 = a.aw * B44 + s;

            float sxx = S00, sxy = S01, syy = S11;
            if (a.nom_sxy) {
                sxx = __ldg(a.nom_sxy + 3 * k);
                sxy = __ldg(a.nom_sxy + 3 * k + 1);
                syy = __ldg(a.nom_sxy + 3 * k + 2);
            }
            const float lmax =
                fmaxf(0.0f, 0.5f * (sxx + syy) + hypotf(0.5f * (sxx - syy), sxy));
            rbar = a.r - a.sq_chi2 * sqrtf(lmax);                      // Eq. 14
            // obstacles (Eq. 15-16)
            omargin = FLT_MAX;
            for (int o = 0; o < a.O; ++o) {
                const float cx = __ldg(a.obst + 3 * o), cy = __ldg(a.obst + 3 * o + 1),
                            R = __ldg(a.obst + 3 * o + 2);
                const float dx = mu0 - cx, dy = mu1 - cy;
                const float rho = sqrtf(dx * dx + dy * dy);
                float spread;
                if (rho > 1e-9f) {
                    const float nx = dx / rho, ny = dy / rho;
                    spread = sqrtf(fmaxf(0.0f, nx * nx * sxx + 2.0f * nx * ny * sxy + ny * ny * syy));
                } else {
                    spread = sqrtf(lmax);
                }
                omargin = fminf(omargin, (rho - R) - a.phi_inv * spread);
            }
            stage = a.c_var * (s + s) + a.c_speed * (a.v_des - mu3) * (a.v_des - mu3);
            if (omargin <= 0.0f) stage += a.c_coll;
            pos[m] = make_float2(mu0, mu1);
        }
        __syncthreads();

        // ---------------- P5: distance to the lane polyline ----------------
        {
            const int m = lane % MTP;
            const float2 pp = pos[m];
            float best = FLT_MAX;
            for (int g = warp * SUB + lane / MTP; g < a.S; g += THREADS / MTP) {
                const float4 sg = __ldg(a.seg + g);
                const float il2 = __ldg(a.seg_il2 + g);
                const float px = pp.x - sg.x, py = pp.y - sg.y;
                const float t = fminf(fmaxf((px * sg.z + py * sg.w) * il2, 0.0f), 1.0f);
                const float qx = px - t * sg.z, qy = py - t * sg.w;
                best = fminf(best, qx * qx + qy * qy);
            }
            epart[tid] = best;
        }
        __syncthreads();

        // ---------------- P6: lane deviation and indicator ----------------
        if (owner) {
            const int m = lane;
            float e2 = FLT_MAX;
            for (int w = 0; w < WARPS; ++w)
#pragma unroll
                for (int u = 0; u < SUB; ++u) e2 = fminf(e2, epart[w * 32 + u * MTP + m]);
            const float e = sqrtf(e2);
            const float lmargin = e - rbar;
            stage += a.c_dev * e;
            if (lmargin > 0.0f) stage += a.c_lane * disc;
            cost += stage;
            disc *= 0.9f;
            if (TRACE && active) {
                const size_t sk = (size_t)s_me * a.T + k;
                if (a.tr_mu) {
                    float* o = a.tr_mu + sk * 5;
                    o[0] = mu0; o[1] = mu1; o[2] = mu2; o[3] = mu3; o[4] = mu4;
                }
                if (a.tr_sig) {
                    float* o = a.tr_sig + sk * 15;
                    o[0] = S00; o[1] = S01; o[2] = S02; o[3] = S03; o[4] = S04;
                    o[5] = S11; o[6] = S12; o[7] = S13; o[8] = S14;
                    o[9] = S22; o[10] = S23; o[11] = S24;
                    o[12] = S33; o[13] = S34; o[14] = S44;
                }
                if (a.tr_stage) a.tr_stage[sk] = stage;
                if (a.tr_margin) {
                    a.tr_margin[sk * 2] = lmargin;
                    a.tr_margin[sk * 2 + 1] = (a.O > 0) ? omargin : __int_as_float(0x7f800000);
                }
            }
        }
    }
    if (active && a.costs) a.costs[s_me] = cost;
}

template <int MTP, bool TRACE>
int launch_t(const RolloutArgs& a, cudaStream_t st) {
    const int smem = Smem<MTP>::total(a.Np);
    auto kern = k_rollout_fp32<MTP, TRACE>;
    GPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = (a.K + a.mt - 1) / a.mt;
    kern<<<grid, THREADS, smem, st>>>(a);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

}  // namespace

int rollout_fp32_mtp(int Np) {
    if (Np <= 1024) return 32;
    if (Np <= 2048) return 16;
    return 8;
}

int rollout_fp32_smem_bytes(int Np, int mtp) {
    switch (mtp) {
        case 32: return Smem<32>::total(Np);
        case 16: return Smem<16>::total(Np);
        default: return Smem<8>::total(Np);
    }
}

int launch_rollout_fp32(const RolloutArgs& a, bool trace, cudaStream_t st) {
    const int mtp = rollout_fp32_mtp(a.Np);
    if (a.mt < 1 || a.mt > mtp) return fail(GPMPPI_ERR_INVALID_ARG, "rollout: bad samples per CTA");
    if (trace) {
        switch (mtp) {
            case 32: return launch_t<32, true>(a, st);
            case 16: return launch_t<16, true>(a, st);
            default: return launch_t<8, true>(a, st);
        }
    }
    switch (mtp) {
        case 32: return launch_t<32, false>(a, st);
        case 16: return launch_t<16, false>(a, st);
        default: return launch_t<8, false>(a, st);
    }
}

}  // namespace gpm
