// The FP32 CUDA-core rollout (Alg. 1 Step 1) as a device body, shared by
// the single-controller kernel (rollout_fp32.cu) and the batched persistent
// kernel (rollout_mma.cu).  See rollout_fp32.cu for the phases.
#pragma once

#include <cudaTypedefs.h>

#include <cfloat>

#include "common.cuh"

namespace gpm {
namespace f32r {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

// ---- TMA / mbarrier primitives (PTX) ---------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// non-blocking probe of a phase
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for a phase with a time limit; on expiry record the error and report
// failure (the caller then stops waiting for further copies).  A limit of 0
// gives up at once unless the phase is already complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                                  unsigned int* err) {
    if (mbar_test_wait(bar, parity)) return true;
    if (limit_ns == 0) {
        atomicOr(err, 1u);
        return false;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) {
            atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}


// Geometry of the L^-T tiles: a warp owns 32 consecutive (sample-group, pair)
// items, i.e. PPW = 32 / NMG pairs; its A tile covers columns [8 p0, 8 p0 + 8 PPW)
// and its B tile columns [Np - 8 (p0 + PPW), Np - 8 p0), R rows per stage.
template <int MTP>
struct Tile {
    static constexpr int NMG = MTP / 4;
    static constexpr int PPW = 32 / NMG;
    static constexpr int TW = 8 * PPW;                 // tile width (floats)
    static constexpr int R = (MTP == 8) ? 4 : 8;       // rows per stage
    static constexpr int BYTES = TW * R * 4;           // one tile
};

template <int MTP>
struct Smem {
    // byte offsets inside the dynamic shared buffer
    static __host__ __device__ int ks(int) { return 0; }
    static __host__ __device__ int qpart(int Np) { return Np * MTP * 4; }
    static __host__ __device__ int mpart(int Np) { return qpart(Np) + (Np / 16) * MTP * 4; }
    static __host__ __device__ int epart(int Np) { return mpart(Np) + THREADS * 8; }
    static __host__ __device__ int zq(int Np) { return epart(Np) + THREADS * 4; }
    static __host__ __device__ int pos(int Np) { return zq(Np) + MTP * 16; }
    static __host__ __device__ int tiles(int Np) { return ((pos(Np) + MTP * 8 + 1023) / 1024) * 1024; }
    // per warp and stage: the A tile then the B tile
    static __host__ __device__ int bars(int Np, int stages) {
        return tiles(Np) + WARPS * stages * 2 * Tile<MTP>::BYTES;
    }
    // one more mbarrier for the failure-detection hook (nothing arrives on it)
    static __host__ __device__ int never(int Np, int stages) { return bars(Np, stages) + WARPS * stages * 8; }
    static __host__ __device__ int total(int Np, int stages) { return never(Np, stages) + 8; }
};

// Named barrier over the 256 threads of the rollout (the whole CTA of the
// single-controller launch; warps 0-7 of the batched persistent kernel).
__device__ __forceinline__ void sync256() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

// One CTA's rollout of the samples [tile mt, tile mt + mt): the body of the
// single-controller kernel and of the batched persistent kernel.  tmW: the
// tensor map over L^-T (a kernel parameter or in global memory).
template <int MTP, bool TRACE>
__device__ __forceinline__ void rollout_fp32_body(const RolloutArgs& a, const CUtensorMap* tmW, int tile,
                                                  unsigned char* smem_raw) {
    const int Np = a.Np;
    float* Ks = reinterpret_cast<float*>(smem_raw + Smem<MTP>::ks(Np));
    float* qpart = reinterpret_cast<float*>(smem_raw + Smem<MTP>::qpart(Np));
    float2* mpart = reinterpret_cast<float2*>(smem_raw + Smem<MTP>::mpart(Np));
    float* epart = reinterpret_cast<float*>(smem_raw + Smem<MTP>::epart(Np));
    float4* zq = reinterpret_cast<float4*>(smem_raw + Smem<MTP>::zq(Np));
    float2* pos = reinterpret_cast<float2*>(smem_raw + Smem<MTP>::pos(Np));
    unsigned char* tiles = smem_raw + Smem<MTP>::tiles(Np);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + Smem<MTP>::bars(Np, a.stages));

    constexpr int SUB = 32 / MTP;          // lanes sharing one sample in P2 / P5
    constexpr int NMG = MTP / 4;           // 4-sample groups in P3
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s0 = tile * a.mt;
    const int mvalid = min(a.mt, a.K - s0);
    const int npairs = Np / 16;
    const int items = NMG * npairs;

    // per-sample state, live in warp 0 lanes < MTP
    const bool owner = (warp == 0) && (lane < MTP);
    const bool active = owner && (lane < mvalid);
    const int s_me = s0 + ((lane < mvalid) ? lane : 0);
    float mu0 = a.x0[0], mu1 = a.x0[1], mu2 = a.x0[2], mu3 = a.x0[3], mu4 = a.x0[4];
    uint32_t it0 = a.it0, it1 = a.it1;
    if (a.x0_dev) {
        mu0 = a.x0_dev[0]; mu1 = a.x0_dev[1]; mu2 = a.x0_dev[2]; mu3 = a.x0_dev[3]; mu4 = a.x0_dev[4];
    }
    if (a.it_dev) {
        const unsigned long long v = *a.it_dev;
        it0 = (uint32_t)v;
        it1 = (uint32_t)(v >> 32);
    }
    // symmetric Sigma, upper triangle
    float S00 = 0, S01 = 0, S02 = 0, S03 = 0, S04 = 0, S11 = 0, S12 = 0, S13 = 0, S14 = 0,
          S22 = 0, S23 = 0, S24 = 0, S33 = 0, S34 = 0, S44 = 0;
    float cost = 0.0f, disc = 1.0f, stage = 0.0f, rbar = 0.0f, omargin = FLT_MAX;
    float2 ut = make_float2(0.f, 0.f);

    // per-warp tile pipeline: S stages, one full-barrier each
    using TL = Tile<MTP>;
    const int S = a.stages;
    uint64_t* wbar = bars + warp * S;
    unsigned char* wtile = tiles + (size_t)warp * S * 2 * TL::BYTES;
    if (lane == 0)
        for (int st = 0; st < S; ++st) mbar_init(wbar + st, 1);
    fence_mbar_init();
    sync256();
    uint32_t nrun = 0;          // tile stages consumed by this warp so far
    uint32_t nissued = 0;       // tile stages requested by this warp (lane 0)
    bool tma_ok = true;         // warp-uniform; false once a copy failed to arrive in time
    // Failure-detection hook (a.expire_first): before any copy, warp 0 waits,
    // bounded by a.wait_ns, on an mbarrier that nothing arrives on.  The wait
    // runs out, records the timeout and turns the warp's copies off, exactly as
    // a copy that never lands would; the rest of the rollout runs on (its
    // results are then unspecified) and the kernel ends normally.
    if (a.expire_first && warp == 0) {
        // (in the dynamic layout: a static shared variable would move the
        // dynamic region off the alignment the tensor copies need)
        uint64_t* never_bar = reinterpret_cast<uint64_t*>(smem_raw + Smem<MTP>::never(Np, S));
        int ok = 1;
        if (lane == 0) {
            mbar_init(never_bar, 1);
            ok = mbar_wait_bounded(never_bar, 0u, a.wait_ns, a.err) ? 1 : 0;
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(never_bar)) : "memory");
        }
        tma_ok = __shfl_sync(0xffffffffu, ok, 0) != 0;
    }

    for (int k = 0; k < a.T; ++k) {
        // ---------------- P1: noise, clamp, query --------------------------
        if (owner) {
            const float2 e = control_eps((uint32_t)k, (uint32_t)s_me, it0, it1, a.key0, a.key1,
                                         a.sig_v, a.sig_w);
            ut.x = fminf(fmaxf(__ldg(a.U + 2 * k) + e.x, a.umin0), a.umax0);
            ut.y = fminf(fmaxf(__ldg(a.U + 2 * k + 1) + e.y, a.umin1), a.umax1);
            zq[lane] = make_float4(mu3 * a.zscale[0], mu4 * a.zscale[1], ut.x * a.zscale[2],
                                   ut.y * a.zscale[3]);
            if (active) a.u_tilde[(size_t)k * a.K + s_me] = ut;
        }
        sync256();

        // ---------------- P2: kernel row and mean partials ----------------
        {
            const int m = lane % MTP;
            const float4 z = zq[m];
            float mv = 0.0f, mw = 0.0f, cv = 0.0f, cw = 0.0f;
            for (int j = warp * SUB + lane / MTP; j < Np; j += THREADS / MTP) {
                float kv = 0.0f;
                if (j < a.N) {
                    const float4 x = ldg4(a.Xs + 4 * j);
                    const float e0 = z.x - x.x, e1 = z.y - x.y, e2 = z.z - x.z, e3 = z.w - x.w;
                    kv = a.sf2 * exp2f(-(e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3));
                    const float2 al = __ldg(reinterpret_cast<const float2*>(a.alpha) + j);
                    kahan_add(mv, cv, kv * al.x);
                    kahan_add(mw, cw, kv * al.y);
                }
                Ks[j * MTP + m] = kv;
            }
            mpart[tid] = make_float2(mv + cv, mw + cw);
        }
        sync256();

        // ---------------- P3: |L^-1 k*|^2 by a triangular product ----------
        for (int g = warp; g * 32 < items; g += WARPS) {
            const int mg = lane % NMG;
            const int pl = lane / NMG;
            const int p0 = g * TL::PPW;
            const int p = p0 + pl;
            const int last = min(TL::PPW, npairs - p0);    // pairs in this group
            const int endA = 8 * (p0 + last);                // rows holding A coefficients
            const int endB = Np - 8 * p0;                    // rows holding B coefficients
            const int xA = 8 * p0;
            const int xB = Np - 8 * (p0 + TL::PPW);          // may be < 0 for tiny N: zero fill
            const int nchA = endA / TL::R;                   // endA, endB are multiples of 8
            const int nch = endB / TL::R;
            auto issue = [&](int c) {
                const uint32_t n = nrun + (uint32_t)c;
                const int st = (int)(n % (uint32_t)S);
                unsigned char* base = wtile + (size_t)st * 2 * TL::BYTES;
                const bool withA = c < nchA;
                ++nissued;
                mbar_expect_tx(wbar + st, (withA ? 2u : 1u) * (uint32_t)TL::BYTES);
                if (withA) tma_load_2d(base, tmW, xA, c * TL::R, wbar + st);
                tma_load_2d(base + TL::BYTES, tmW, xB, c * TL::R, wbar + st);
            };
            if (lane == 0 && tma_ok)
                for (int c = 0; c < min(S, nch); ++c) issue(c);
            float accA[4][8], accB[4][8];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    accA[r][c] = 0.0f;
                    accB[r][c] = 0.0f;
                }
            const float* kp = Ks + 4 * mg;
            const int offA = 8 * pl;
            const int offB = 8 * (TL::PPW - 1 - pl);
            for (int c = 0; c < nch; ++c) {
                const uint32_t n = nrun + (uint32_t)c;
                const int st = (int)(n % (uint32_t)S);
                bool ok = tma_ok;
                if (ok) ok = mbar_wait_bounded(wbar + st, (n / (uint32_t)S) & 1u, a.wait_ns, a.err);
                tma_ok = __all_sync(0xffffffffu, ok);
                const float* tA = reinterpret_cast<const float*>(wtile + (size_t)st * 2 * TL::BYTES);
                const float* tB = tA + TL::TW * TL::R;
                const int j0 = c * TL::R;
                if (c < nchA) {
#pragma unroll
                    for (int r = 0; r < TL::R; ++r) {
                        const float4 kv = *reinterpret_cast<const float4*>(kp + (j0 + r) * MTP);
                        const float4 a0 = *reinterpret_cast<const float4*>(tA + r * TL::TW + offA);
                        const float4 a1 = *reinterpret_cast<const float4*>(tA + r * TL::TW + offA + 4);
                        const float4 b0 = *reinterpret_cast<const float4*>(tB + r * TL::TW + offB);
                        const float4 b1 = *reinterpret_cast<const float4*>(tB + r * TL::TW + offB + 4);
                        const float kr[4] = {kv.x, kv.y, kv.z, kv.w};
                        const float wa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                        const float wb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                            for (int cc = 0; cc < 8; ++cc) {
                                accA[rr][cc] = fmaf(kr[rr], wa[cc], accA[rr][cc]);
                                accB[rr][cc] = fmaf(kr[rr], wb[cc], accB[rr][cc]);
                            }
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < TL::R; ++r) {
                        const float4 kv = *reinterpret_cast<const float4*>(kp + (j0 + r) * MTP);
                        const float4 b0 = *reinterpret_cast<const float4*>(tB + r * TL::TW + offB);
                        const float4 b1 = *reinterpret_cast<const float4*>(tB + r * TL::TW + offB + 4);
                        const float kr[4] = {kv.x, kv.y, kv.z, kv.w};
                        const float wb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                            for (int cc = 0; cc < 8; ++cc)
                                accB[rr][cc] = fmaf(kr[rr], wb[cc], accB[rr][cc]);
                    }
                }
                __syncwarp();
                if (lane == 0 && tma_ok && c + S < nch) {
                    fence_proxy_async_smem();     // our reads of this stage precede the refill
                    issue(c + S);
                }
            }
            nrun += (uint32_t)nch;
            if (p < npairs) {
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
        }
        sync256();

        // ---------------- P4: dynamics, covariance, obstacles --------------
        if (owner) {
            const int m = lane;
            float mv = 0.0f, mw = 0.0f, cv = 0.0f, cw = 0.0f;
            for (int w = 0; w < WARPS; ++w)
#pragma unroll
                for (int u = 0; u < SUB; ++u) {
                    const float2 pm = mpart[w * 32 + u * MTP + m];
                    kahan_add(mv, cv, pm.x);
                    kahan_add(mw, cw, pm.y);
                }
            mv += cv;
            mw += cw;
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
        sync256();

        // ---------------- P5: distance to the lane polyline ----------------
        {
            const int m = lane % MTP;
            const float2 pp = pos[m];
            float best = FLT_MAX;
            const int2 oc = lane_cands(a, pp.x, pp.y);     // candidate segments of this position
            for (int i = warp * SUB + lane / MTP; i < oc.y; i += THREADS / MTP) {
                const int g = lane_seg(a, oc, i);
                const float4 sg = __ldg(a.seg + g);
                const float il2 = __ldg(a.seg_il2 + g);
                const float px = pp.x - sg.x, py = pp.y - sg.y;
                const float t = fminf(fmaxf((px * sg.z + py * sg.w) * il2, 0.0f), 1.0f);
                const float qx = px - t * sg.z, qy = py - t * sg.w;
                best = fminf(best, qx * qx + qy * qy);
            }
            epart[tid] = best;
        }
        sync256();

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
            stage += goal_cost(a, k, mu0, mu1);                       // Eq. 12 goal terms
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
    // after a failed copy, give the copies still in flight a bounded time to
    // land before the CTA's shared memory is released
    if (!tma_ok && lane == 0) {
        const uint64_t t0 = global_ns();
        for (uint32_t n = (nissued > (uint32_t)S ? nissued - (uint32_t)S : 0u); n < nissued; ++n)
            while (!mbar_try_wait(wbar + n % (uint32_t)S, (n / (uint32_t)S) & 1u) &&
                   global_ns() - t0 < 200000000ull) {
            }
    }
}

}  // namespace f32r
}  // namespace gpm
