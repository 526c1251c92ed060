// Lengthscale gradient through the GP variance (the K^-1 dependence of
// Eq. 3's s = sf2 - k*^T K^-1 k*): the traces
//   tr(D_d G_o),  G_o = sum_q sbar_o,q b_q b_q^T,  D_d = dK/dl_d,
// over all T K queries q of the adjoint rollout, with b_q = K^-1 k*_q and
// sbar_o,q the adjoint of output o's variance at that query.  G_o is a Gram
// matrix of the b_q (a contraction over the queries), formed here on the
// tensor cores tile by tile and contracted with D_d in the tile's epilogue,
// so G never reaches global memory and no scaled copies of b are stored.
//
// Output tiles are 128 rows (block ib of the training points) x 256 columns
// (blocks jb, jb + 1 with jb >= ib: G and D are symmetric, so only the upper
// block triangle is formed and off-diagonal blocks count twice), for both
// outputs at once: A_o = sbar_o,q b_q restricted to the row block (the MMA's
// A, K-major over 16 queries), B = b_q restricted to the two column blocks.
// The query range is split between CTAs (split K); each CTA writes 8
// partial traces (2 outputs x 4 lengthscales), which the gradient's final
// reduction sums in a fixed order.
//
// Precision: b and sbar b are split into BF16 hi + lo parts (16 significand
// bits, the full FP32 exponent range, so no scaling is needed) and three
// products hi.hi + hi.lo + lo.hi are accumulated in FP32 in tensor memory.
// The tensor core's accumulator rounds at every MMA, so the accumulation is
// cut into segments of SEG chunks: after each segment the epilogue takes the
// traces of the segment's partial G (FP32, summed into FP64 per thread) and
// the accumulator restarts.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc05.cuh"

namespace gpm {
namespace {

constexpr int GQ = 16;                        // queries per chunk (one MMA K-step)
constexpr int GROWS = 128;                    // rows of a tile (the MMA M)
constexpr int GCOLS = 256;                    // columns of a tile: two blocks (the MMA N)
constexpr int GPROD = 256;                    // producer threads (8 warps), also the epilogue
constexpr int GTHREADS = GPROD + 32;          // + the MMA-issuing warp
constexpr int GSTAGES = 4;
constexpr int A_TILE = GROWS * GQ * 2;        // 4 KiB: one 16-bit part of one A operand
constexpr int B_TILE = GCOLS * GQ * 2;        // 8 KiB: one 16-bit part of B
constexpr int GSTAGE = 4 * A_TILE + 2 * B_TILE;   // A_v hi, lo, A_w hi, lo, B hi, lo: 32 KiB
constexpr int SEG = 128;                      // chunks accumulated before the traces are taken
constexpr uint64_t kGramWaitNs = 2000000000ull;

// shared memory: stages, the column blocks' scaled inputs, barriers
constexpr int SM_XS = GSTAGES * GSTAGE;                 // 256 float4
constexpr int SM_BARS = SM_XS + GCOLS * 16;             // full[GSTAGES], empty[GSTAGES], seg_done, tmem_free
constexpr int SM_TSLOT = SM_BARS + 8 * (2 * GSTAGES + 2);
constexpr int SM_ABORT = SM_TSLOT + 4;
constexpr int SM_RED = ((SM_ABORT + 4 + 15) / 16) * 16; // 8 warps x 4 doubles
constexpr int SM_TOTAL = SM_RED + 8 * 4 * 8;

struct GramArgs {
    const float* Bq;        // Q x Np
    const float4* qbar;     // Q: (mbar_v, mbar_w, sbar_v, sbar_w)
    const float* Xs;        // N x 4 scaled inputs
    float* part;            // nparts x 8
    unsigned int* err;
    int Q, Np, N, nb, ntiles, qs;
    float sf2;
};

// BF16 hi + lo of the pair (a, b), packed two per 32-bit word (a low)
__device__ __forceinline__ void split_bf16(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    float ra, rb;
    tc::split_resid<1>(hi, a, b, ra, rb);
    const __nv_bfloat162 l = __floats2bfloat162_rn(ra, rb);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ bool gwait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, unsigned int* err) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    const uint64_t t0 = tc::global_ns();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (tc::global_ns() - t0 > kGramWaitNs) {
            *abort_flag = 1;
            if (err) atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}

// One chunk's six MMAs (three split products for each output) and the commit
// that frees its stage, issued by one lane chosen by elect.sync (the warp is
// converged); the first product into each accumulator overwrites it unless
// acc0 != 0.
__device__ __forceinline__ void mma6_elect(uint32_t dv, uint32_t dw, uint64_t avh, uint64_t avl, uint64_t awh,
                                           uint64_t awl, uint64_t bh, uint64_t bl, uint32_t idesc, uint32_t acc0,
                                           uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e, p0, p1;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p0, %9, 0;\n\t"
        "setp.ne.b32 p1, 1, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %6, %8, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %7, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %6, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %6, %8, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %7, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %5, %6, %8, p1;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%10];\n\t}" ::"r"(dv),
        "r"(dw), "l"(avh), "l"(avl), "l"(awh), "l"(awl), "l"(bh), "l"(bl), "r"(idesc), "r"(acc0),
        "r"(tc::smem_addr(bar))
        : "memory");
}

// 2^x, the hardware approximation (relative error near 2^-22)
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

__global__ void __launch_bounds__(GTHREADS, 1) k_gram_tc(const GramArgs g) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float4* xs_s = reinterpret_cast<float4*>(sm + SM_XS);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + SM_BARS);
    uint64_t* empty = full + GSTAGES;
    uint64_t* seg_done = empty + GSTAGES;
    uint64_t* tmem_free = seg_done + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + SM_TSLOT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + SM_ABORT);
    double* red = reinterpret_cast<double*>(sm + SM_RED);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // tile -> (row block ib, first column block jb): row block ib has
    // ceil((nb - ib) / 2) tiles
    const int split = blockIdx.x / g.ntiles;
    int t = blockIdx.x % g.ntiles, ib = 0;
    while (ib < g.nb - 1 && t >= (g.nb - ib + 1) / 2) {
        t -= (g.nb - ib + 1) / 2;
        ++ib;
    }
    const int jb = ib + 2 * t;
    const int I0 = GROWS * ib, J0 = GROWS * jb, J1 = J0 + GROWS;
    const int q_begin = split * g.qs;
    const int q_end = min(g.Q, q_begin + g.qs);
    const int nchunk = q_end > q_begin ? (q_end - q_begin + GQ - 1) / GQ : 0;

    if (tid == 0) {
        for (int i = 0; i < GSTAGES; ++i) {
            tc::mbar_init(full + i, GPROD / 32);
            tc::mbar_init(empty + i, 1);
        }
        tc::mbar_init(seg_done, 1);
        tc::mbar_init(tmem_free, GPROD / 32);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // scaled inputs of the tile's columns (rows past N: far away, never used)
    for (int j = tid; j < GCOLS; j += GTHREADS) {
        const int jj = (j < GROWS ? J0 + j : J1 + j - GROWS);
        xs_s[j] = jj < g.N ? __ldg(reinterpret_cast<const float4*>(g.Xs) + jj)
                           : make_float4(1e4f, 1e4f, 1e4f, 1e4f);
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;

    if (warp == GPROD / 32) {
        // ========================= MMA issuer ==================================
        const uint32_t idesc = tc::idesc_f16(1, GROWS, GCOLS);
        const uint64_t dA0 = tc::smem_desc(tc::smem_addr(sm), GROWS * 16, 128);
        const uint64_t dB0 = tc::smem_desc(tc::smem_addr(sm + 4 * A_TILE), GCOLS * 16, 128);
        bool ok = true;
        int c = 0;
        for (; c < nchunk && ok; ++c) {
            const int st = c % GSTAGES;
            const uint32_t use = (uint32_t)(c / GSTAGES);
            const int seg = c / SEG;
            if (c % SEG == 0 && seg > 0) {
                ok = __all_sync(0xffffffffu, gwait(tmem_free, (uint32_t)(seg - 1) & 1u, abort_flag, g.err));
                if (!ok) break;
                tc::fence_after_sync();
            }
            ok = __all_sync(0xffffffffu, gwait(full + st, use & 1u, abort_flag, g.err));
            if (!ok) break;
            tc::fence_after_sync();
            const uint64_t so = (uint64_t)((st * GSTAGE) >> 4);
            const uint64_t aVh = dA0 + so, aVl = aVh + (A_TILE >> 4);
            const uint64_t aWh = aVh + ((2 * A_TILE) >> 4), aWl = aVh + ((3 * A_TILE) >> 4);
            const uint64_t bH = dB0 + so, bL = bH + (B_TILE >> 4);
            const uint32_t acc0 = (c % SEG) ? 1u : 0u;
            mma6_elect(taddr, taddr + (uint32_t)GCOLS, aVh, aVl, aWh, aWl, bH, bL, idesc, acc0, empty + st);
            if (c % SEG == SEG - 1 || c == nchunk - 1) tc::mma_commit_elect(seg_done);
        }
        // after an abort, let MMAs in flight land before the memory is released
        if (!ok && lane == 0) {
            const uint64_t t0 = tc::global_ns();
            for (int i = (c >= GSTAGES ? c - GSTAGES : 0); i < c; ++i)
                while (!tc::mbar_try_wait(empty + (i % GSTAGES), (uint32_t)(i / GSTAGES) & 1u) &&
                       tc::global_ns() - t0 < 200000000ull) {
                }
        }
        __syncwarp();
    } else {
        // ==================== producers, then the epilogue =======================
        const int r = tid & (GROWS - 1);        // row of the A tiles, of each B block
        const int h = tid >> 7;                 // K half: queries 8h .. 8h + 7 of a chunk
        const bool in_i = I0 + r < g.Np, in_j0 = J0 + r < g.Np, in_j1 = J1 + r < g.Np;
        // epilogue role: TMEM lane quarter lq (rows 32 lq ..), output o
        const int lq = warp & 3, o = warp >> 2;
        const int il = 32 * lq + lane, i = I0 + il;
        const float4 xi = i < g.N ? __ldg(reinterpret_cast<const float4*>(g.Xs) + i)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        bool ok = true;
        for (int c = 0; c < nchunk; ++c) {
            const int st = c % GSTAGES;
            const uint32_t use = (uint32_t)(c / GSTAGES);
            const int q0 = q_begin + c * GQ + 8 * h;
            float av[8], aw[8], b0[8], b1[8];
            // the adjoints and the rows of b are loaded independently (all 32
            // loads in flight at once); a query whose adjoints are both zero
            // (padding samples, whose b may be anything) is then selected away
            float4 qb[8];
            float bi[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int q = q0 + e;
                const bool in = q < q_end;
                const float* row = g.Bq + (size_t)(in ? q : q_begin) * g.Np;
                qb[e] = in ? __ldg(g.qbar + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                bi[e] = (in && in_i) ? __ldg(row + I0 + r) : 0.0f;
                b0[e] = (in && in_j0) ? __ldg(row + J0 + r) : 0.0f;
                b1[e] = (in && in_j1) ? __ldg(row + J1 + r) : 0.0f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool live = (qb[e].z != 0.0f) || (qb[e].w != 0.0f);
                av[e] = live ? bi[e] * qb[e].z : 0.0f;
                aw[e] = live ? bi[e] * qb[e].w : 0.0f;
                b0[e] = live ? b0[e] : 0.0f;
                b1[e] = live ? b1[e] : 0.0f;
            }
            uint32_t vh[4], vl[4], wh[4], wl[4], h0[4], l0[4], h1[4], l1[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                split_bf16(av[2 * p], av[2 * p + 1], vh[p], vl[p]);
                split_bf16(aw[2 * p], aw[2 * p + 1], wh[p], wl[p]);
                split_bf16(b0[2 * p], b0[2 * p + 1], h0[p], l0[p]);
                split_bf16(b1[2 * p], b1[2 * p + 1], h1[p], l1[p]);
            }
            // the stage is free once the MMAs that read it completed
            if (c >= GSTAGES && !gwait(empty + st, (use - 1) & 1u, abort_flag, g.err)) ok = false;
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            unsigned char* s = sm + st * GSTAGE;
            // slab h of row r (16 bytes) in each part
            const int ao = h * GROWS * 16 + r * 16, bo = h * GCOLS * 16 + r * 16;
            *reinterpret_cast<uint4*>(s + ao) = make_uint4(vh[0], vh[1], vh[2], vh[3]);
            *reinterpret_cast<uint4*>(s + A_TILE + ao) = make_uint4(vl[0], vl[1], vl[2], vl[3]);
            *reinterpret_cast<uint4*>(s + 2 * A_TILE + ao) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
            *reinterpret_cast<uint4*>(s + 3 * A_TILE + ao) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
            *reinterpret_cast<uint4*>(s + 4 * A_TILE + bo) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
            *reinterpret_cast<uint4*>(s + 4 * A_TILE + bo + GROWS * 16) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
            *reinterpret_cast<uint4*>(s + 4 * A_TILE + B_TILE + bo) = make_uint4(l0[0], l0[1], l0[2], l0[3]);
            *reinterpret_cast<uint4*>(s + 4 * A_TILE + B_TILE + bo + GROWS * 16) =
                make_uint4(l1[0], l1[1], l1[2], l1[3]);
            tc::fence_proxy_async();           // generic stores -> the tensor core's reads
            __syncwarp();
            if (lane == 0) arrive(full + st);
            if (c % SEG == SEG - 1 || c == nchunk - 1) {
                // ---- epilogue of segment c / SEG: traces against dK/dl_d ----
                const int seg = c / SEG;
                bool sok = gwait(seg_done, (uint32_t)seg & 1u, abort_flag, g.err);
                sok = __all_sync(0xffffffffu, sok);
                tc::fence_after_sync();
                if (!sok) {
                    ok = false;
                    break;
                }
                float tr[4] = {0.f, 0.f, 0.f, 0.f};
                const uint32_t row_addr = taddr + ((uint32_t)(32 * lq) << 16) + (uint32_t)(o * GCOLS);
#pragma unroll 1
                for (int cc = 0; cc < GCOLS; cc += 32) {
                    float v[32];
                    tc::tmem_ld32(row_addr + (uint32_t)cc, v);
                    // off-diagonal blocks stand for both (i, j) and (j, i)
                    const float wblk = (cc < GROWS && jb == ib) ? 1.0f : 2.0f;
                    if (i < g.N) {
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const float4 xj = xs_s[cc + e];
                            const float d0 = xi.x - xj.x, d1 = xi.y - xj.y, d2 = xi.z - xj.z, d3 = xi.w - xj.w;
                            const float q0s = d0 * d0, q1s = d1 * d1, q2s = d2 * d2, q3s = d3 * d3;
                            const float kg = g.sf2 * ex2_approx(-(q0s + q1s + q2s + q3s)) * v[e] * wblk;
                            tr[0] = fmaf(kg, q0s, tr[0]);
                            tr[1] = fmaf(kg, q1s, tr[1]);
                            tr[2] = fmaf(kg, q2s, tr[2]);
                            tr[3] = fmaf(kg, q3s, tr[3]);
                        }
                    }
                }
#pragma unroll
                for (int d = 0; d < 4; ++d) acc[d] += (double)tr[d];
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) arrive(tmem_free);
                (void)seg;
            }
        }
        // per output: sum over the four lane-quarter warps in a fixed order
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            double v = acc[d];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp * 4 + d] = v;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(GPROD) : "memory");
        if (tid < 8) {
            const int oo = tid >> 2, d = tid & 3;
            double s = 0.0;
            for (int w = 0; w < 4; ++w) s += red[(4 * oo + w) * 4 + d];
            g.part[(size_t)blockIdx.x * 8 + oo * 4 + d] = (float)s;
        }
        (void)ok;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

// tiles of the upper block triangle (two column blocks each)
int gram_tiles(int Np) {
    const int nb = (Np + GROWS - 1) / GROWS;
    int n = 0;
    for (int ib = 0; ib < nb; ++ib) n += (nb - ib + 1) / 2;
    return n;
}

// queries per CTA (a multiple of the chunk), for about four waves of CTAs
int gram_queries_per_cta(int Q, int Np, int nsm) {
    const int ntiles = gram_tiles(Np);
    int nsplit = (4 * nsm + ntiles - 1) / ntiles;
    if (nsplit < 1) nsplit = 1;
    int qs = (Q + nsplit - 1) / nsplit;
    qs = ((qs + GQ - 1) / GQ) * GQ;
    return qs < GQ ? GQ : qs;
}

}  // namespace

int gram_tc_parts(int Q, int Np, int nsm) {
    const int qs = gram_queries_per_cta(Q, Np, nsm);
    const int nsplit = Q > 0 ? (Q + qs - 1) / qs : 1;
    return gram_tiles(Np) * nsplit;
}

int launch_gram_tc(const float* Bq, const float4* qbar, int Q, int Np, int N, const float* Xs, float sf2,
                   float* part, int nparts, unsigned int* err, int nsm, cudaStream_t st) {
    GramArgs g;
    g.Bq = Bq;
    g.qbar = qbar;
    g.Xs = Xs;
    g.part = part;
    g.err = err;
    g.Q = Q;
    g.Np = Np;
    g.N = N;
    g.nb = (Np + GROWS - 1) / GROWS;
    g.ntiles = gram_tiles(Np);
    g.qs = gram_queries_per_cta(Q, Np, nsm);
    g.sf2 = sf2;
    const int nsplit = Q > 0 ? (Q + g.qs - 1) / g.qs : 1;
    const int grid = g.ntiles * nsplit;
    if (grid != nparts) return fail(GPMPPI_ERR_INVALID_ARG, "gram: partial-trace count mismatch");
    GPM_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_TOTAL));
    k_gram_tc<<<grid, GTHREADS, SM_TOTAL, st>>>(g);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

}  // namespace gpm
