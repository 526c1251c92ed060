// Fused MPPI rollout with the GP variance contraction on the tensor cores
// (tcgen05, split 16-bit operands, FP32 accumulation in TMEM).
//
// Same method as the FP32 rollout (Alg. 1 Step 1: noise, clamp, GP mean and
// variance, Eq. 10 mean/covariance, Eq. 11-16 costs); only the dense part
// of the variance, V = K* L^-T with |V_m|^2 = |L^-1 k*_m|^2, moves to the
// tensor cores.  Operands are split into a high and a low 16-bit part
// (x = hi + lo, both FP16 or both BF16) and three products hi*hi + hi*lo +
// lo*hi are accumulated in FP32, which keeps the variance close to FP32
// accuracy; the queries are scaled to a_j = k*_j / sf2 in [0, 1] and L^-T by a
// power of two cB so that both fit the 16-bit range.
//
// CTA = 128 samples (the MMA M), 256 threads: thread t serves sample t % 128
// and half h = t / 128 of every shared loop.  The output columns of V are
// processed in passes of up to 512 (one TMEM allocation), 64 columns per MMA
// block; the reduction dimension in chunks of 32 training points through two
// shared-memory stages.  Per chunk the threads compute the kernel-row tile
// (exp2 on the SFU), one thread fetches the pre-arranged L^-T tiles with bulk
// copies and issues 3 x 2 MMAs per active block (blocks entirely above the
// triangle are skipped) and commits them to the stage's mbarrier.  At the end
// of a pass each thread reads its sample's TMEM row and sums the squares.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cfloat>

#include "common.cuh"
#include "tc05.cuh"

namespace gpm {
namespace {

constexpr int MT = 128;               // samples per CTA
constexpr int THREADS = 256;
constexpr int KC = 32;                // training points per chunk
constexpr int BLK = 64;               // output columns per MMA block
constexpr int BLOCKS_PER_PASS = 8;    // 512 TMEM columns
constexpr int A_PART = MT * KC * 2;                         // 8 KiB
constexpr int B_TILE = BLK * KC * 2;                        // 4 KiB
constexpr int STAGE = 2 * A_PART + BLOCKS_PER_PASS * 2 * B_TILE;   // 80 KiB
constexpr uint64_t kWaitNs = 2000000000ull;

struct SmemM {
    static constexpr int bars = 2 * STAGE;              // mma_done[2], bfull[2]
    static constexpr int tslot = bars + 32;
    static constexpr int flag = tslot + 4;
    static constexpr int qh = bars + 64;                // 2 x 128 floats
    static constexpr int mh = qh + 2 * MT * 4;          // 2 x 128 float2
    static constexpr int ep = mh + 2 * MT * 8;          // 2 x 128 floats
    static constexpr int om = ep + 2 * MT * 4;          // 2 x 128 floats
    static constexpr int total = om + 2 * MT * 4;
};

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_addr(bar))
        : "memory");
}

template <int FMT>
__device__ __forceinline__ uint32_t pack2(float a, float b, float* ra, float* rb) {
    // hi parts of two values packed in one 32-bit word; returns the residuals
    if (FMT == 0) {
        const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
        *ra = a - __half2float(ha);
        *rb = b - __half2float(hb);
        return (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
    } else {
        const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
        *ra = a - __bfloat162float(ha);
        *rb = b - __bfloat162float(hb);
        return (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    }
}

template <int FMT>
__device__ __forceinline__ uint32_t pack2_lo(float a, float b) {
    if (FMT == 0)
        return (uint32_t)__half_as_ushort(__float2half_rn(a)) |
               ((uint32_t)__half_as_ushort(__float2half_rn(b)) << 16);
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

template <int FMT, bool TRACE>
__global__ void __launch_bounds__(THREADS, 1) k_rollout_mma(const RolloutArgs a, const MmaArgs mm) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* mma_done = reinterpret_cast<uint64_t*>(sm + SmemM::bars);
    uint64_t* bfull = mma_done + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + SmemM::tslot);
    volatile int* okflag = reinterpret_cast<volatile int*>(sm + SmemM::flag);
    float* qh = reinterpret_cast<float*>(sm + SmemM::qh);
    float2* mh = reinterpret_cast<float2*>(sm + SmemM::mh);
    float* ep = reinterpret_cast<float*>(sm + SmemM::ep);
    float* omh = reinterpret_cast<float*>(sm + SmemM::om);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = tid & (MT - 1);
    const int h = tid >> 7;
    const int s0 = blockIdx.x * MT;
    const int mvalid = min(MT, a.K - s0);
    const bool active = m < mvalid;
    const int s_me = s0 + (active ? m : 0);
    const int NB = mm.nblocks;                 // 64-column blocks of L^-T
    const int npass = (NB + BLOCKS_PER_PASS - 1) / BLOCKS_PER_PASS;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) tc::mbar_init(mma_done + i, 1);
        *okflag = 1;
        tc::fence_mbar_init();
    }
    if (warp == 0 && NB > 0) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint32_t idesc = tc::idesc_f16(FMT, MT, BLK);

    float mu0 = a.x0[0], mu1 = a.x0[1], mu2 = a.x0[2], mu3 = a.x0[3], mu4 = a.x0[4];
    float S00 = 0, S01 = 0, S02 = 0, S03 = 0, S04 = 0, S11 = 0, S12 = 0, S13 = 0, S14 = 0,
          S22 = 0, S23 = 0, S24 = 0, S33 = 0, S34 = 0, S44 = 0;
    float cost = 0.0f, disc = 1.0f;
    uint32_t n = 0;                 // chunks issued so far (all passes, all steps)
    bool ok = true;                 // no bounded wait gave up (CTA-uniform via okflag)

    for (int k = 0; k < a.T; ++k) {
        // ---------------- P1: noise, clamp, query (both halves) ------------
        const float2 e = control_eps((uint32_t)k, (uint32_t)s_me, a.it0, a.it1, a.key0, a.key1,
                                     a.sig_v, a.sig_w);
        float2 ut;
        ut.x = fminf(fmaxf(__ldg(a.U + 2 * k) + e.x, a.umin0), a.umax0);
        ut.y = fminf(fmaxf(__ldg(a.U + 2 * k + 1) + e.y, a.umin1), a.umax1);
        if (h == 0 && active) a.u_tilde[(size_t)k * a.K + s_me] = ut;
        const float z0 = mu3 * a.zscale[0], z1 = mu4 * a.zscale[1];
        const float z2 = ut.x * a.zscale[2], z3 = ut.y * a.zscale[3];

        // ---------------- P2/P3: kernel row, mean, variance on tcgen05 ------
        float qpart = 0.0f, mv = 0.0f, mw = 0.0f, cv = 0.0f, cw = 0.0f;
        for (int g = 0; g < npass; ++g) {
            const int b0 = g * BLOCKS_PER_PASS;
            const int b1 = min(NB, b0 + BLOCKS_PER_PASS);
            const int nchunk = 2 * b1;           // block b needs chunks 0 .. 2b+1
            const bool last_pass = (g == npass - 1);
            for (int c = 0; c < nchunk; ++c, ++n) {
                const int st = (int)(n & 1u);
                const uint32_t use = n >> 1;
                unsigned char* stage = sm + st * STAGE;
                if (n >= 2 && ok) ok = tc::mbar_wait(mma_done + st, (use - 1) & 1u, kWaitNs, a.err);
                if (tid == 0 && ok) {
                    int nact = 0;
                    for (int b = b0; b < b1; ++b) nact += (c < 2 * b + 2) ? 1 : 0;
                    tc::mbar_expect_tx(bfull + st, (uint32_t)(nact * 2 * B_TILE));
                    for (int b = b0; b < b1; ++b) {
                        if (c >= 2 * b + 2) continue;
                        unsigned char* dst = stage + 2 * A_PART + (b - b0) * 2 * B_TILE;
                        const size_t tile = ((size_t)b * mm.nchunks + c) * (B_TILE / 2);
                        bulk_copy(dst, mm.Bhi + tile, B_TILE, bfull + st);
                        bulk_copy(dst + B_TILE, mm.Blo + tile, B_TILE, bfull + st);
                    }
                }
                // kernel-row tile: this thread's 16 training points = slabs 2h, 2h+1
                {
                    uint32_t hw[8], lw[8];
                    const int jb = c * KC + 16 * h;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float av[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int j = jb + 2 * q + u;
                            float v = 0.0f;
                            if (j < a.N) {
                                const float4 x = __ldg(reinterpret_cast<const float4*>(a.Xs) + j);
                                const float d0 = z0 - x.x, d1 = z1 - x.y, d2 = z2 - x.z, d3 = z3 - x.w;
                                v = exp2f(-(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3));
                                if (last_pass) {
                                    const float2 al = __ldg(reinterpret_cast<const float2*>(a.alpha) + j);
                                    kahan_add(mv, cv, v * al.x);
                                    kahan_add(mw, cw, v * al.y);
                                }
                            }
                            av[u] = v;
                        }
                        float r0, r1;
                        hw[q] = pack2<FMT>(av[0], av[1], &r0, &r1);
                        lw[q] = pack2_lo<FMT>(r0, r1);
                    }
                    unsigned char* Ahi = stage;
                    unsigned char* Alo = stage + A_PART;
                    const int sl = 2 * h;
                    *reinterpret_cast<uint4*>(Ahi + sl * MT * 16 + m * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(Ahi + (sl + 1) * MT * 16 + m * 16) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
                    *reinterpret_cast<uint4*>(Alo + sl * MT * 16 + m * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    *reinterpret_cast<uint4*>(Alo + (sl + 1) * MT * 16 + m * 16) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
                }
                tc::fence_proxy_async();
                __syncthreads();
                ok = ok && (*okflag != 0);
                if (tid == 0 && ok) {
                    if (!tc::mbar_wait(bfull + st, use & 1u, kWaitNs, a.err)) {
                        ok = false;
                        *okflag = 0;
                    } else {
                        tc::fence_after_sync();
                        const uint32_t aHi = tc::smem_addr(stage), aLo = aHi + A_PART;
                        for (int b = b0; b < b1; ++b) {
                            if (c >= 2 * b + 2) continue;
                            const uint32_t bHi = aHi + 2 * A_PART + (b - b0) * 2 * B_TILE;
                            const uint32_t bLo = bHi + B_TILE;
                            const uint32_t d = taddr + (uint32_t)((b - b0) * BLK);
#pragma unroll
                            for (int ks = 0; ks < 2; ++ks) {
                                const uint32_t ao = ks * 2 * MT * 16, bo = ks * 2 * BLK * 16;
                                const uint64_t dAh = tc::smem_desc(aHi + ao, MT * 16, 128);
                                const uint64_t dAl = tc::smem_desc(aLo + ao, MT * 16, 128);
                                const uint64_t dBh = tc::smem_desc(bHi + bo, BLK * 16, 128);
                                const uint64_t dBl = tc::smem_desc(bLo + bo, BLK * 16, 128);
                                const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                                tc::mma_f16(d, dAh, dBh, idesc, acc0);
                                tc::mma_f16(d, dAh, dBl, idesc, 1u);
                                tc::mma_f16(d, dAl, dBh, idesc, 1u);
                            }
                        }
                        tc::mma_commit(mma_done + st);
                    }
                }
            }
            // pass end: every MMA of the pass has landed in TMEM
            const uint32_t lastn = n - 1;
            if (ok) ok = tc::mbar_wait(mma_done + (lastn & 1u), (lastn >> 1) & 1u, kWaitNs, a.err);
            ok = __all_sync(0xffffffffu, ok);     // tcgen05.ld below is warp-collective
            tc::fence_after_sync();
            if (ok) {
                const int half_cols = (b1 - b0) * BLK / 2;
                const uint32_t row = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
                for (int cc = 0; cc < half_cols; cc += 32) {
                    float v[32];
                    tc::tmem_ld32(row + (uint32_t)(h * half_cols + cc), v);
                    // two-level sum of squares: 4 partials of 8, then the batch
                    float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        p0 = fmaf(v[i], v[i], p0);
                        p1 = fmaf(v[8 + i], v[8 + i], p1);
                        p2 = fmaf(v[16 + i], v[16 + i], p2);
                        p3 = fmaf(v[24 + i], v[24 + i], p3);
                    }
                    qpart += (p0 + p1) + (p2 + p3);
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            if (!ok) *okflag = 0;
        }
        qh[h * MT + m] = qpart;
        mh[h * MT + m] = make_float2(mv + cv, mw + cw);
        __syncthreads();
        ok = ok && (*okflag != 0);
        const float q = (qh[m] + qh[MT + m]) * mm.qscale;
        const float2 m0 = mh[m], m1 = mh[MT + m];
        const float mean_v = a.sf2 * (m0.x + m1.x), mean_w = a.sf2 * (m0.y + m1.y);
        const float s = fmaxf(0.0f, a.sf2 - q);

        // ---------------- P4: dynamics, covariance, obstacles ---------------
        float sn, cs;
        sincosf(mu2, &sn, &cs);
        const float a02 = -a.dt * mu3 * sn, a03 = a.dt * cs;
        const float a12 = a.dt * mu3 * cs, a13 = a.dt * sn;
        const float nX = mu0 + a.dt * mu3 * cs;
        const float nY = mu1 + a.dt * mu3 * sn;
        const float nT = mu2 + a.dt * mu4;
        const float nV = mu3 + a.kv * (ut.x - mu3) + mean_v;
        const float nW = mu4 + a.kw * (ut.y - mu4) + mean_w;
        mu0 = nX; mu1 = nY; mu2 = nT; mu3 = nV; mu4 = nW;
        {
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
        }
        float sxx = S00, sxy = S01, syy = S11;
        if (a.nom_sxy) {
            sxx = __ldg(a.nom_sxy + 3 * k);
            sxy = __ldg(a.nom_sxy + 3 * k + 1);
            syy = __ldg(a.nom_sxy + 3 * k + 2);
        }
        const float lmax = fmaxf(0.0f, 0.5f * (sxx + syy) + hypotf(0.5f * (sxx - syy), sxy));
        const float rbar = a.r - a.sq_chi2 * sqrtf(lmax);
        float om = FLT_MAX;
        for (int o = h; o < a.O; o += 2) {
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
            om = fminf(om, (rho - R) - a.phi_inv * spread);
        }
        // ---------------- P5: lane distance (segments split by half) -------
        float best = FLT_MAX;
        for (int gsg = h; gsg < a.S; gsg += 2) {
            const float4 sg = __ldg(a.seg + gsg);
            const float il2 = __ldg(a.seg_il2 + gsg);
            const float px = mu0 - sg.x, py = mu1 - sg.y;
            const float t = fminf(fmaxf((px * sg.z + py * sg.w) * il2, 0.0f), 1.0f);
            const float qx = px - t * sg.z, qy = py - t * sg.w;
            best = fminf(best, qx * qx + qy * qy);
        }
        omh[h * MT + m] = om;
        ep[h * MT + m] = best;
        __syncthreads();
        const float omargin = fminf(omh[m], omh[MT + m]);
        const float e_lane = sqrtf(fminf(ep[m], ep[MT + m]));
        // ---------------- P6: stage cost ------------------------------------
        float stage = a.c_var * (s + s) + a.c_speed * (a.v_des - mu3) * (a.v_des - mu3);
        if (omargin <= 0.0f) stage += a.c_coll;
        const float lmargin = e_lane - rbar;
        stage += a.c_dev * e_lane;
        if (lmargin > 0.0f) stage += a.c_lane * disc;
        cost += stage;
        disc *= 0.9f;
        if (TRACE && active && h == 0) {
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
    if (active && h == 0 && a.costs) a.costs[s_me] = cost;
    // release TMEM; after a failed wait give copies and MMAs in flight a
    // bounded time to land first
    if (!ok && tid == 0 && n > 0) {
        const uint64_t t0 = tc::global_ns();
        for (uint32_t i = (n >= 2 ? n - 2 : 0); i < n; ++i) {
            while (!tc::mbar_try_wait(mma_done + (i & 1u), (i >> 1) & 1u) &&
                   tc::global_ns() - t0 < 200000000ull) {
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0 && NB > 0) tc::tmem_dealloc(taddr, 512);
}

}  // namespace

int rollout_mma_smem_bytes() { return SmemM::total; }

int launch_rollout_mma(const RolloutArgs& a, const MmaArgs& mm, int fmt, bool trace, cudaStream_t st) {
    const int smem = SmemM::total;
    const int grid = (a.K + MT - 1) / MT;
#define GPM_LAUNCH_MMA(F, TR)                                                                     \
    do {                                                                                          \
        auto kern = k_rollout_mma<F, TR>;                                                         \
        GPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));  \
        kern<<<grid, THREADS, smem, st>>>(a, mm);                                                 \
    } while (0)
    if (fmt == 0) {
        if (trace) GPM_LAUNCH_MMA(0, true); else GPM_LAUNCH_MMA(0, false);
    } else {
        if (trace) GPM_LAUNCH_MMA(1, true); else GPM_LAUNCH_MMA(1, false);
    }
#undef GPM_LAUNCH_MMA
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

}  // namespace gpm
