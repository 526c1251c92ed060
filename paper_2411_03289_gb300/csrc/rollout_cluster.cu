// Tensor-core rollout for training sets of up to 512 points: a cluster of CS
// CTAs (CS = NpC / 128) carries 128 samples through the horizon, each CTA
// holding its share of the variance factor resident in shared memory.
//
// Same method and arithmetic as the streaming tensor-core rollout
// (Alg. 1 Step 1; V = K* L^-T on the tensor cores with FP16/BF16 hi/lo split
// operands, |V_m|^2 = |L^-1 k*_m|^2).  What changes is where the operands
// live.  The output columns of V are cut into 64-column slices and rank r of
// the cluster owns slices r and NS - 1 - r (equal triangular work for every
// rank).  Their pieces of cB L^-1 (the hi and lo rows of a chunk side by
// side, at most 144 KiB) are copied into shared memory once, before the first
// step, so a step moves no factor tiles at all.  The MMAs read that resident
// B from shared memory and the kernel-row tiles A from tensor memory, where
// the producer warps write them (tcgen05.st, one sample per TMEM lane) into a
// four-stage ring.  Shared memory thus carries only B to the tensor core: a
// 128 x 128 x 16 MMA with both operands there reads 8 KiB per 64 clocks, the
// whole shared-memory bandwidth, and streaming the factor through it every
// step halved the MMA rate.
//
// Per step: every rank computes the queries and kernel rows of all 128
// samples (and its share of the GP mean), issues the MMAs of its slices and
// sends its mean share to every peer through distributed shared memory as
// soon as the share is complete (asynchronous stores that complete bytes on
// the receiver's mbarrier).  All ranks then advance the same 128 states
// identically (same inputs, same order of summation).  The variance is off
// that chain: a rank reads its partial |V_m|^2 from TMEM one step later,
// while the next step's kernel rows are in flight, and sends it to the rank
// that scores sample m.  The cost phase (lane distance, obstacles,
// Eq. 11-16) is split between the ranks by sample, so rank r scores and
// writes the samples m = r (mod CS).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cfloat>

#include "common.cuh"
#include "tc05.cuh"

namespace gpm {
namespace {

using tc::f2add;
using tc::f2fma;
using tc::f2mul;
using tc::f2pack;
using tc::f2sub;
using tc::f2unpack;

constexpr int MT = 128;               // samples per cluster (the MMA M)
constexpr int NPROD = 256;            // producer threads: two per sample
constexpr int NCOST = 64;             // scoring threads (two warps)
constexpr int THREADS = NPROD + 32 + NCOST;   // + the MMA-issuing warp and the scoring warps
constexpr int NSTAGE = 4;             // kernel-row tile ring (in tensor memory)
constexpr int GCH = 4;                // chunks per stage: one hand-off per four chunks
static_assert(GCH == 4, "the issue loop issues a stage as four chunks");
constexpr int BURST = 4;              // chunks whose kernel rows a thread computes together
static_assert(BURST == GCH, "a producer burst fills exactly one stage");
// TMEM columns: the accumulators D in columns [0, 256) (hi.hi + lo.hi of the
// lower and upper slice in 0-63 and 64-127, hi.lo of the upper slice in
// 128-191, of the lower in 192-255), the A ring after them; a chunk's A tile
// takes 16 columns (hi in 8, lo in 8: 16 elements of 16 bits per lane and part)
constexpr uint32_t TM_COLS = 512;
constexpr uint32_t A_COL = 256;
constexpr uint32_t A_CHUNK_COLS = 16;
constexpr uint32_t A_STAGE_COLS = GCH * A_CHUNK_COLS;
static_assert(A_COL + NSTAGE * A_STAGE_COLS <= TM_COLS, "A ring exceeds the TMEM allocation");
constexpr int B_MAX = 144 * 1024;     // largest resident share (NS = 8)
constexpr uint64_t kWaitNs = 2000000000ull;
// hand-off record of one scored sample and step: post-step mean (5), pre-step
// speed, sin and cos of the pre-step heading (the GP variance s arrives
// separately, as the |V_m|^2 partials of every rank)
constexpr int SST = 8;
// With four ranks the last rank computes the kernel rows of rank 0's last four
// chunks and copies them into rank 0's shared memory (hi and lo, 128 rows x 16
// points each, in the slab-major operand layout): rank 0, the rank every step
// waits for, computes 28 chunks instead of 32.
constexpr int AR_CHUNKS = 4;
constexpr int AR_CHUNK_BYTES = 2 * MT * 16 * 2;     // 8 KiB: hi 4 KiB, then lo
constexpr int AR_BYTES = AR_CHUNKS * AR_CHUNK_BYTES;

struct ClLayout {
    int b, bars, tslot, abort_flag, xq, xm, ar, sst, xs, al, seg, il2, obs, total;
};

// shared-memory layout; the resident B share is sized for the largest rank;
// S lane segments and O obstacles are staged when they fit (else S = O = 0);
// nown = 128 / CS samples scored per rank
__host__ __device__ inline ClLayout cl_layout(int npc, int S, int O) {
    const int nown = MT / (npc / 128);
    ClLayout L;
    L.b = 0;
    // a_full, empty [NSTAGE], b_res, pass_done, tmem_free, xbar[2], st_full[2], st_empty[2],
    // ar_full, x_res, qbar[4], ar_free
    L.bars = B_MAX;
    L.tslot = L.bars + 8 * (2 * NSTAGE + 16);
    L.abort_flag = L.tslot + 4;
    // received partial |V|^2 of the samples this rank scores,
    // [4 (step mod 4)][2 CS (sending rank, thread half)][nown] floats, and the
    // GP mean partials (v, w) of every producer thread of every rank,
    // [2 (step parity)][8 (rank, thread half)][MT] float2
    L.xq = ((L.abort_flag + 4 + 15) / 16) * 16;
    L.xm = L.xq + 4 * 2 * MT * 4;
    // kernel rows received by rank 0 (staged by the last rank) with four ranks
    L.ar = ((L.xm + 2 * 8 * MT * 8 + 127) / 128) * 128;
    L.sst = L.ar + (npc == 512 ? AR_BYTES : 0);  // [2][nown][SST] floats: per-step hand-off to the scoring warps
    L.xs = ((L.sst + 2 * nown * SST * 4 + 127) / 128) * 128;
    L.al = L.xs + npc * 16;
    L.seg = L.al + npc * 8;                      // S float4
    L.il2 = L.seg + S * 16;                      // S floats
    L.obs = L.il2 + ((S + 3) / 4) * 16;          // O x 3 floats
    L.total = L.obs + O * 12;
    return L;
}

// Issue order of a rank's 4-chunk groups, shared by the producers and the MMA
// warp: group 0 first (its MMAs initialise the accumulators), then the groups
// holding the rank's GP-mean chunks [4 gm0, 4 gm1), then the rest, each part
// ascending.  The mean share is thus complete, and on its way to the peers,
// while the remaining groups are computed.  Returns the first chunk of the
// i-th group.
__device__ __forceinline__ int burst_chunk(int i, int gm0, int gm1) {
    if (i == 0) return 0;
    const int a0 = gm0 > 1 ? gm0 : 1;
    const int nm = gm1 - a0 > 0 ? gm1 - a0 : 0;
    if (i - 1 < nm) return GCH * (a0 + i - 1);
    int g = i - nm;
    if (g >= a0) g += nm;
    return GCH * g;
}
// index of the group after which a rank's GP-mean share is complete (-1: the
// rank sums no chunk of its own groups)
__device__ __forceinline__ int last_mean_burst(int gm0, int gm1) {
    if (gm1 <= gm0) return -1;
    const int a0 = gm0 > 1 ? gm0 : 1;
    return gm1 - a0 > 0 ? gm1 - a0 : 0;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_addr(bar))
        : "memory");
}

// 2^x (the hardware approximation; results below the normal range flush to 0,
// far below what a 16-bit split operand can carry)
__device__ __forceinline__ float ex2_ftz(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// hi + lo split of the pair (a, b): hi = rn16(a, b), lo = rn16((a, b) - hi)
template <int FMT>
__device__ __forceinline__ void split2(uint64_t ab, uint32_t* hi, uint32_t* lo) {
    float a, b;
    f2unpack(ab, a, b);
    float ra, rb;
    if (FMT == 0) {
        const __half2 h = __floats2half2_rn(a, b);
        *hi = *reinterpret_cast<const uint32_t*>(&h);
        tc::split_resid<0>(*hi, a, b, ra, rb);
        const __half2 l = __floats2half2_rn(ra, rb);
        *lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        *hi = *reinterpret_cast<const uint32_t*>(&h);
        tc::split_resid<1>(*hi, a, b, ra, rb);
        const __nv_bfloat162 l = __floats2bfloat162_rn(ra, rb);
        *lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

__device__ __forceinline__ bool try_wait_cluster(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc::smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (CTA-local phases: the tensor pipe, the producers).
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                              unsigned int* err) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    const uint64_t t0 = tc::global_ns();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (tc::global_ns() - t0 > kWaitNs) {
            *abort_flag = 1;
            if (err) atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}

// Bounded wait on a phase completed by remote arrivals (acquire at cluster scope).
__device__ __forceinline__ bool wait_cluster(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                             unsigned int* err) {
    if (try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = tc::global_ns();
    while (!try_wait_cluster(bar, parity)) {
        if (tc::global_ns() - t0 > kWaitNs) {
            *abort_flag = 1;
            if (err) atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}

// The same, also giving up once another role of this CTA has aborted (the
// scoring warps' wait for the variance partials).
__device__ __forceinline__ bool wait_cluster_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                      unsigned int* err) {
    if (try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = tc::global_ns();
    while (!try_wait_cluster(bar, parity)) {
        if (*abort_flag) return false;
        if (tc::global_ns() - t0 > kWaitNs) {
            *abort_flag = 1;
            if (err) atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}

// named barrier over the 128 producer threads of one thread half (u = 0, 1)
__device__ __forceinline__ void half_sync(int u) {
    asm volatile("bar.sync %0, 128;" ::"r"(1 + u) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// address of the same shared-memory object in CTA `peer` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t peer) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::smem_addr(p)), "r"(peer));
    return r;
}

// asynchronous stores into a cluster CTA's shared memory that complete their
// transaction bytes (4 or 8) on the mbarrier at bar (same CTA as addr)
__device__ __forceinline__ void st_async_f32(uint32_t addr, float v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_f32x2(uint32_t addr, float2 v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "f"(v.x), "f"(v.y), "r"(bar)
                 : "memory");
}
// bulk copy from this CTA's shared memory into a cluster CTA's shared memory,
// completing its bytes on the mbarrier at bar (same CTA as dst)
__device__ __forceinline__ void bulk_copy_peer(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "r"(tc::smem_addr(src)), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int FMT, bool TRACE>
__global__ void __launch_bounds__(THREADS, 1) k_rollout_cl(const RolloutArgs a, const ClArgs cl) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const ClLayout L = cl_layout(cl.npc, cl.scene_smem ? a.S : 0, cl.scene_smem ? a.O : 0);
    unsigned char* bres = sm + L.b;
    uint64_t* a_full = reinterpret_cast<uint64_t*>(sm + L.bars);
    uint64_t* empty = a_full + NSTAGE;
    uint64_t* b_res = empty + NSTAGE;
    uint64_t* pass_done = b_res + 1;
    uint64_t* tmem_free = pass_done + 1;
    uint64_t* xbar = tmem_free + 1;             // [2]
    uint64_t* st_full = xbar + 2;               // [2] post-step states handed to the scoring warps
    uint64_t* st_empty = st_full + 2;           // [2] ... and released by them
    uint64_t* ar_full = st_empty + 2;           // rank 0: the kernel rows copied in by the last rank
    uint64_t* x_res = ar_full + 1;              // the training set copied in
    uint64_t* qbar = x_res + 1;                 // [4] partial |V|^2 of the scored samples, by step mod 4
    uint64_t* ar_free = qbar + 4;               // last rank: rank 0's MMAs have consumed the copied rows
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tslot);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + L.abort_flag);
    float* xq = reinterpret_cast<float*>(sm + L.xq);
    float2* xm = reinterpret_cast<float2*>(sm + L.xm);
    unsigned char* ar = sm + L.ar;
    float* sst = reinterpret_cast<float*>(sm + L.sst);
    float4* xs_s = reinterpret_cast<float4*>(sm + L.xs);
    float4* al_s = reinterpret_cast<float4*>(sm + L.al);
    float4* seg_s = reinterpret_cast<float4*>(sm + L.seg);
    float* il2_s = reinterpret_cast<float*>(sm + L.il2);
    float* obs_s = reinterpret_cast<float*>(sm + L.obs);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int CS = cl.cs, NS = cl.ns;
    const uint32_t rank = cluster_rank();
    const int tile = blockIdx.x / CS;
    const int nboth = 4 * ((int)rank + 1);      // chunks needed by both of this rank's slices
    const int nch = 4 * (NS - (int)rank);       // chunks needed by its upper slice
    // GP-mean chunks [mc0, mc1) of this rank: rank 0 (the most kernel-row
    // chunks) the last four, each further rank the eight below, the last rank
    // all the rest; every range lies inside the rank's own kernel-row chunks
    int mc1 = 4 * NS, mc0 = 4 * (NS - 1);
    for (int r = 1; r <= (int)rank; ++r) {
        mc1 = mc0;
        mc0 = mc1 - 8;
    }
    if ((int)rank == CS - 1) mc0 = 0;
    // With four ranks: rank 0 computes no GP-mean terms and not the kernel rows
    // of its last four chunks; the last rank computes those rows (chunks
    // [me0, me1), with their GP-mean terms) first in every step and copies them
    // into rank 0's shared memory; rank 1 sums chunks 24-27, rank 2 12-23, the
    // last rank 0-11.
    const bool rows_out = CS == 4 && (int)rank == CS - 1;
    const bool rows_in = CS == 4 && rank == 0;
    int me0 = 0, me1 = 0;
    if (CS == 4) {
        mc0 = rank == 1 ? 24 : (rank == 2 ? 12 : 0);
        mc1 = rank == 0 ? 0 : (rank == 1 ? 28 : (rank == 2 ? 24 : 12));
        if (rows_out) {
            me0 = 4 * NS - AR_CHUNKS;
            me1 = 4 * NS;
        }
    }
    const int nch_p = rows_in ? nch - AR_CHUNKS : nch;   // chunks whose rows the producers write to TMEM
    // the rank's GP-mean groups inside its own groups, and the burst that completes them
    const int gm0 = mc0 / GCH, gm1 = (mc1 < nch_p ? mc1 : nch_p) / GCH;
    // (rank 0 with four ranks sums no mean chunk and sends its empty share at
    // the start of the step)
    const int ilast = last_mean_burst(gm0, gm1);
    const uint32_t bbytes = (uint32_t)cl.bytes[rank];

    if (tid == 0) {
        for (int i = 0; i < NSTAGE; ++i) {
            tc::mbar_init(a_full + i, NPROD / 32);
            tc::mbar_init(empty + i, 1);
        }
        tc::mbar_init(b_res, 1);
        tc::mbar_init(pass_done, 1);
        tc::mbar_init(tmem_free, NPROD / 32);
        // one local arrival (with the expected bytes) per phase; the partials
        // arrive as transaction bytes
        tc::mbar_init(xbar, 1);
        tc::mbar_init(xbar + 1, 1);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(st_full + i, 4);             // the four warps holding the writers
            tc::mbar_init(st_empty + i, NCOST / 32);
        }
        tc::mbar_init(ar_full, 1);
        tc::mbar_init(x_res, 1);
        for (int i = 0; i < 4; ++i) tc::mbar_init(qbar + i, 1);   // armed by the scoring warps
        tc::mbar_init(ar_free, 1);                      // one arrival per step, from rank 0's tensor pipe
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // training inputs and alpha arrive by one bulk copy (TMA engine) in pair
    // layout: for points 2p and 2p + 1, xs_s[2p] = (x0, x0', x1, x1'),
    // xs_s[2p + 1] = (x2, x2', x3, x3') and al_s[p] = (a_v, a_v', a_w, a_w')
    // (primes: point 2p + 1); rows past N hold a far point and alpha 0
    const int Ssm = cl.scene_smem ? a.S : 0, Osm = cl.scene_smem ? a.O : 0;
    for (int i = tid; i < Ssm; i += THREADS) {
        seg_s[i] = __ldg(a.seg + i);
        il2_s[i] = __ldg(a.seg_il2 + i);
    }
    for (int i = tid; i < 3 * Osm; i += THREADS) obs_s[i] = __ldg(a.obst + i);
    const float4* segp = cl.scene_smem ? seg_s : a.seg;
    const float* il2p = cl.scene_smem ? il2_s : a.seg_il2;
    const float* obsp = cl.scene_smem ? obs_s : a.obst;
    if (warp == 0) tc::tmem_alloc(tslot, TM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
        // this rank's resident share of the factor, one copy for the whole horizon
        tc::mbar_expect_tx(b_res, bbytes);
        bulk_copy(bres, cl.tiles + cl.base[rank], bbytes, b_res);
        tc::mbar_expect_tx(x_res, (uint32_t)(cl.npc * 24));
        bulk_copy(xs_s, cl.xa, (uint32_t)(cl.npc * 16), x_res);
        bulk_copy(al_s, cl.xa + 4 * cl.npc, (uint32_t)(cl.npc * 8), x_res);
    }
    // The perturbed controls of the whole horizon (Alg. 1: nominal plus noise,
    // clamped) do not depend on the state, so they are drawn here, while the
    // resident share is in flight: rank r the samples m = r (mod CS) of all T
    // steps, written to u~ in global memory, which every rank's producers then
    // read a step ahead.  The cluster barrier below publishes them.
    {
        const int nown = MT / CS;
        for (int i = tid; i < nown * a.T; i += THREADS) {
            const int k = i / nown, m = (int)rank + CS * (i % nown);
            const int s = tile * MT + m;
            if (s >= a.K) continue;
            const float2 e = control_eps((uint32_t)k, (uint32_t)s, a.it0, a.it1, a.key0, a.key1, a.sig_v, a.sig_w);
            float2 uk;
            uk.x = fminf(fmaxf(__ldg(a.U + 2 * k) + e.x, a.umin0), a.umax0);
            uk.y = fminf(fmaxf(__ldg(a.U + 2 * k + 1) + e.y, a.umin1), a.umax1);
            a.u_tilde[(size_t)k * a.K + s] = uk;
        }
    }
    // every CTA's barriers are initialised before any peer arrives on them, and
    // every rank's perturbed controls are visible to the whole cluster
    cluster_sync_all();
    const uint32_t taddr = *tslot;

    if (warp == NPROD / 32) {
        // ================= MMA issuer (one warp, one elected lane) ==============
        // The whole warp runs the loop (its operand arithmetic stays
        // warp-uniform); elect.sync picks the lane that issues each instruction.
        // Per chunk two MMAs: A_hi x [B_hi | B_lo] (N doubled: the hi.hi and
        // hi.lo products land in separate TMEM columns) and A_lo x B_hi
        // (accumulated onto hi.hi); the pass-end read adds the two column sets.
        const uint32_t idesc256 = tc::idesc_f16(FMT, MT, 256);
        const uint32_t idesc128 = tc::idesc_f16(FMT, MT, 128);
        const uint32_t idesc64 = tc::idesc_f16(FMT, MT, 64);
        // base descriptors of the resident B pieces (256 rows while both slices
        // need a chunk, 128 rows after); all offsets below are multiples of 16
        // bytes inside shared memory, so they add to the start-address field
        const uint64_t dB256 = tc::smem_desc(tc::smem_addr(bres), 256 * 16, 128);
        const uint64_t dB128 = tc::smem_desc(tc::smem_addr(bres), 128 * 16, 128);
        // the received kernel rows (rank 0 with four ranks): A tiles of 128 rows
        // in shared memory, chunk positions 0, 2, 1, 3 for chunks me + 0 .. 3
        const uint64_t dAr = tc::smem_desc(tc::smem_addr(ar), MT * 16, 128);
        bool ok = __all_sync(0xffffffffu, wait_or_abort(b_res, 0, abort_flag, a.err));
        tc::fence_after_sync();
        uint32_t n = 0;
        for (int k = 0; k < a.T && ok; ++k) {
            if (rows_in) {
                if (lane == 0) tc::mbar_expect_tx(ar_full, (uint32_t)AR_BYTES);
                __syncwarp();
            }
            if (k > 0) {
                if (!__all_sync(0xffffffffu, wait_or_abort(tmem_free, (uint32_t)(k - 1) & 1u, abort_flag, a.err))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
            }
            // stage order: the producers' burst order (burst_chunk; its first
            // group initialises the accumulators), with the stage of received
            // rows second (they arrive early: the last rank computes them first)
            for (int si = 0; si < nch / GCH; ++si) {
                const int c = !rows_in ? burst_chunk(si, gm0, gm1)
                                       : (si == 1 ? nch_p : burst_chunk(si == 0 ? 0 : si - 1, gm0, gm1));
                if (c >= nch_p) {
                    // the last stage from the rows the last rank copied in (upper
                    // slice alone: rank 0's last chunks are above nboth)
                    if (!__all_sync(0xffffffffu, wait_or_abort(ar_full, (uint32_t)k & 1u, abort_flag, a.err))) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint64_t b0 = dB128 + (uint64_t)((nboth * 8192 + (c - nboth) * 4096) >> 4);
                    tc::mma_stage4_sa_elect(taddr + 64u, dAr, dAr + (uint64_t)((2 * AR_CHUNK_BYTES) >> 4),
                                            dAr + (uint64_t)(AR_CHUNK_BYTES >> 4),
                                            dAr + (uint64_t)((3 * AR_CHUNK_BYTES) >> 4),
                                            (uint64_t)((AR_CHUNK_BYTES / 2) >> 4), b0, 4096 >> 4, idesc128, idesc64);
                    // tell the last rank when these MMAs have read the rows: it may
                    // then overwrite its staging area and this buffer
                    tc::mma_commit_mc_elect(ar_free, (uint16_t)(1u << (CS - 1)));
                    continue;
                }
                const int st = (int)(n % NSTAGE);
                const uint32_t use = n / NSTAGE;
                if (!__all_sync(0xffffffffu, wait_or_abort(a_full + st, use & 1u, abort_flag, a.err))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t aS = taddr + A_COL + (uint32_t)st * A_STAGE_COLS;
                // a stage's four chunks are all below nboth or all above (nboth is a
                // multiple of 4)
                if (c < nboth) {
                    // rows [hi lower | hi upper | lo upper | lo lower]: D columns
                    // 0-127 hi.hi (+ lo.hi), 128-191 hi.lo upper, 192-255 hi.lo lower
                    const uint64_t b0 = dB256 + (uint64_t)((c * 8192) >> 4);
                    tc::mma_stage4_elect(taddr, aS, b0, 8192 >> 4, empty + st, c > 0 ? 1u : 0u, idesc256, idesc128);
                } else {
                    // rows [hi upper | lo upper]: D columns 64-127 and 128-191
                    const uint64_t b0 = dB128 + (uint64_t)((nboth * 8192 + (c - nboth) * 4096) >> 4);
                    tc::mma_stage4_elect(taddr + 64u, aS, b0, 4096 >> 4, empty + st, 1u, idesc128, idesc64);
                }
                ++n;
            }
            if (!ok) break;
            tc::mma_commit_elect(pass_done);
        }
        // let MMAs in flight land before the shared memory can be released
        if (!ok) {
            const uint64_t t0 = tc::global_ns();
            for (uint32_t i = (n >= (uint32_t)NSTAGE ? n - (uint32_t)NSTAGE : 0); i < n; ++i)
                while (!tc::mbar_try_wait(empty + (i % NSTAGE), (i / NSTAGE) & 1u) &&
                       tc::global_ns() - t0 < 200000000ull) {
                }
        }
        __syncwarp();
    } else if (warp < NPROD / 32) {
        // ========================== producer warps =============================
        const int m = tid & (MT - 1);          // sample within the cluster (= its TMEM lane)
        const int u = tid >> 7;                // which of its two threads (half of each chunk)
        // this warp's TMEM lanes 32 (warp % 4) .., at the A ring's first column
        const uint32_t a_lane = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + A_COL;
        const int s_me = tile * MT + m;
        const int s_q = s_me < a.K ? s_me : 0;
        const int nown = MT / CS;              // samples scored by this rank

        float mu0 = a.x0[0], mu1 = a.x0[1], mu2 = a.x0[2], mu3 = a.x0[3], mu4 = a.x0[4];
        uint32_t n = 0;
        // the perturbed control of step kk, drawn before the horizon (plain
        // loads: other ranks wrote it during this launch)
        const float2* u_row = a.u_tilde + s_q;
        float2 ut_next = u_row[0];
        wait_or_abort(x_res, 0u, abort_flag, a.err);     // the training set in shared memory

        // This rank's partial |V_m|^2 of step kq, read once the MMAs of step kq
        // have completed (the producers call it after the first burst of step
        // kq + 1, and after the last step), and sent to the rank that scores
        // sample m: slot (kq mod 4, rank, u) of its buffer, completing bytes on
        // its barrier qbar[kq mod 4].  Freeing the accumulators lets the MMAs
        // of step kq + 1 start.
        auto read_q = [&](int kq) {
            bool ok = wait_or_abort(pass_done, (uint32_t)kq & 1u, abort_flag, a.err);
            ok = __all_sync(0xffffffffu, ok);    // tcgen05.ld is warp-collective
            tc::fence_after_sync();
            float qpart = 0.0f;
            if (ok) {
                // warp w reads TMEM lanes 32 (w % 4) ..; thread half u the 64
                // columns of its slice: V = (hi.hi + lo.hi) + hi.lo
                const uint32_t row = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
                const uint32_t c0 = (uint32_t)(64 * u), c1 = u ? 128u : 192u;
                // (packed pairs of columns: four independent sums of two lanes each)
                uint64_t p0 = 0ull, p1 = 0ull, p2 = 0ull, p3 = 0ull;
#pragma unroll
                for (int cc = 0; cc < 64; cc += 32) {
                    float v[32], w[32];
                    tc::tmem_ld32x2(row + c0 + (uint32_t)cc, row + c1 + (uint32_t)cc, v, w);
#pragma unroll
                    for (int i = 0; i < 32; i += 8) {
                        const uint64_t x0 = f2add(f2pack(v[i], v[i + 1]), f2pack(w[i], w[i + 1]));
                        const uint64_t x1 = f2add(f2pack(v[i + 2], v[i + 3]), f2pack(w[i + 2], w[i + 3]));
                        const uint64_t x2 = f2add(f2pack(v[i + 4], v[i + 5]), f2pack(w[i + 4], w[i + 5]));
                        const uint64_t x3 = f2add(f2pack(v[i + 6], v[i + 7]), f2pack(w[i + 6], w[i + 7]));
                        p0 = f2fma(x0, x0, p0);
                        p1 = f2fma(x1, x1, p1);
                        p2 = f2fma(x2, x2, p2);
                        p3 = f2fma(x3, x3, p3);
                    }
                }
                float a0, a1, b0, b1, c0f, c1f, d0, d1;
                f2unpack(p0, a0, a1);
                f2unpack(p1, b0, b1);
                f2unpack(p2, c0f, c1f);
                f2unpack(p3, d0, d1);
                qpart = ((a0 + a1) + (b0 + b1)) + ((c0f + c1f) + (d0 + d1));
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_free);
            const uint32_t owner = (uint32_t)(m % CS);
            const int slot = ((kq & 3) * 2 * CS + 2 * (int)rank + u) * nown + m / CS;
            st_async_f32(peer_addr(xq + slot, owner), qpart, peer_addr(qbar + (kq & 3), owner));
        };

        const int nbu = nch_p / BURST;

        for (int k = 0; k < a.T; ++k) {
            // ---------------- query ------------------------------------------------
            const float2 ut = ut_next;
            // the next step's control, its load in flight during the bursts
            if (k + 1 < a.T) ut_next = u_row[(size_t)(k + 1) * a.K];
            const float z0 = mu3 * a.zscale[0], z1 = mu4 * a.zscale[1];
            const float z2 = ut.x * a.zscale[2], z3 = ut.y * a.zscale[3];

            // ---------------- kernel-row tiles ---------------------------------------
            // A burst is BURST = 4 chunks; each thread computes two whole chunks of
            // 16 points (32 independent exp2 in flight).  The GP mean is split
            // between the ranks: rank r sums chunks [mc0, mc1) (and [me0, me1)).
            float mv = 0.0f, mw = 0.0f, cv = 0.0f, cw = 0.0f;
            const uint64_t zz0 = f2pack(z0, z0), zz1 = f2pack(z1, z1);
            const uint64_t zz2 = f2pack(z2, z2), zz3 = f2pack(z3, z3);
            // kernel-row entries of the 16 points of chunk c, as 8 packed pairs:
            // av[q] = (2^-d(z, x_2p), 2^-d(z, x_2p+1)) for pair p = 8 c + q
            auto kernel_row = [&](int c, uint64_t (&av)[8]) {
                const int pb = c * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const ulonglong2 xa = *reinterpret_cast<const ulonglong2*>(xs_s + 2 * (pb + q));
                    const ulonglong2 xb = *reinterpret_cast<const ulonglong2*>(xs_s + 2 * (pb + q) + 1);
                    const uint64_t d0 = f2sub(zz0, xa.x), d1 = f2sub(zz1, xa.y);
                    const uint64_t d2 = f2sub(zz2, xb.x), d3 = f2sub(zz3, xb.y);
                    uint64_t t = f2mul(d0, d0);
                    t = f2fma(d1, d1, t);
                    t = f2fma(d2, d2, t);
                    t = f2fma(d3, d3, t);
                    float t0, t1;
                    f2unpack(t, t0, t1);
                    av[q] = f2pack(ex2_ftz(-t0), ex2_ftz(-t1));
                }
            };
            auto mean_part = [&](int c, const uint64_t (&av)[8]) {
                const int pb = c * 8;
                uint64_t pv = 0ull, pw = 0ull;     // (even, odd) partial sums
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const ulonglong2 al = *reinterpret_cast<const ulonglong2*>(al_s + pb + q);
                    pv = f2fma(av[q], al.x, pv);
                    pw = f2fma(av[q], al.y, pw);
                }
                float pv0, pv1, pw0, pw1;
                f2unpack(pv, pv0, pv1);
                f2unpack(pw, pw0, pw1);
                kahan_add(mv, cv, pv0 + pv1);
                kahan_add(mw, cw, pw0 + pw1);
            };
            if (rows_out) {
                // rank 0's last four chunks: rows (and their GP-mean terms) into this
                // CTA's staging area, then one bulk copy per thread half into rank
                // 0's shared memory (chunk positions 0, 1 for u = 0, 2, 3 for u = 1),
                // once rank 0's MMAs have consumed the previous step's copy
                if (k > 0) wait_cluster_or_abort(ar_free, (uint32_t)(k - 1) & 1u, abort_flag, a.err);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int cc = me0 + 2 * j + u;
                    uint64_t av[8];
                    kernel_row(cc, av);
                    mean_part(cc, av);
                    uint32_t h[8], l[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) split2<FMT>(av[q], &h[q], &l[q]);
                    unsigned char* pc = ar + (2 * u + j) * AR_CHUNK_BYTES + m * 16;
                    *reinterpret_cast<uint4*>(pc) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(pc + MT * 16) = make_uint4(h[4], h[5], h[6], h[7]);
                    *reinterpret_cast<uint4*>(pc + AR_CHUNK_BYTES / 2) = make_uint4(l[0], l[1], l[2], l[3]);
                    *reinterpret_cast<uint4*>(pc + AR_CHUNK_BYTES / 2 + MT * 16) = make_uint4(l[4], l[5], l[6], l[7]);
                }
                tc::fence_proxy_async();               // generic writes before the bulk copy reads them
                half_sync(u);
                if (m == 0)
                    bulk_copy_peer(peer_addr(ar + 2 * u * AR_CHUNK_BYTES, 0u), ar + 2 * u * AR_CHUNK_BYTES,
                                   2u * AR_CHUNK_BYTES, peer_addr(ar_full, 0u));
            }
            // the GP mean share goes to every rank (its own included) as soon as
            // it is complete: slot (rank, u) of sample m in every rank's buffer,
            // completing bytes on that rank's exchange barrier xbar[k & 1]
            const int buf = k & 1;
            if (tid == 0) tc::mbar_expect_tx(xbar + buf, (uint32_t)(CS * 2 * MT * 8));
            auto send_mean = [&]() {
                const int slot = (buf * 8 + 2 * (int)rank + u) * MT + m;
                const float2 mm = make_float2(mv + cv, mw + cw);
                for (int p = 0; p < CS; ++p)
                    st_async_f32x2(peer_addr(xm + slot, (uint32_t)p), mm, peer_addr(xbar + buf, (uint32_t)p));
            };
            // the part of the step that needs no GP result (unicycle with velocity
            // lag; the covariance recursion, which the mean never reads, runs in
            // the scoring warps), computed during the bursts
            float sn = 0.0f, cs = 1.0f, nX = 0.0f, nY = 0.0f, nT = 0.0f, nV0 = 0.0f, nW0 = 0.0f;
            auto dynamics = [&]() {
                sincosf(mu2, &sn, &cs);
                nX = mu0 + a.dt * mu3 * cs;
                nY = mu1 + a.dt * mu3 * sn;
                nT = mu2 + a.dt * mu4;
                nV0 = mu3 + a.kv * (ut.x - mu3);
                nW0 = mu4 + a.kw * (ut.y - mu4);
            };
            if (ilast < 0) send_mean();
            for (int bi = 0; bi < nbu; ++bi) {    // nch_p is a multiple of 4 (and of BURST)
                const int c = burst_chunk(bi, gm0, gm1);
                // the sample's two threads take alternate chunks of the burst:
                // thread half u the chunks c + u and c + 2 + u, all 16 points each
                uint64_t av[2][8];
#pragma unroll
                for (int j = 0; j < 2; ++j) kernel_row(c + 2 * j + u, av[j]);
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (c + 2 * j + u >= mc0 && c + 2 * j + u < mc1) mean_part(c + 2 * j + u, av[j]);
                // per chunk: hi parts in columns 0-7, lo parts in 8-15
                uint32_t hl[2][16];
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int q = 0; q < 8; ++q) split2<FMT>(av[j][q], &hl[j][q], &hl[j][8 + q]);
                // a burst fills one stage (BURST == GCH)
                const int st = (int)(n % NSTAGE);
                const uint32_t use = n / NSTAGE;
                if (n >= (uint32_t)NSTAGE) {
                    // the MMAs that read this stage's columns have completed
                    wait_or_abort(empty + st, (use - 1) & 1u, abort_flag, a.err);
                    __syncwarp();                      // tcgen05.st is warp-collective
                    tc::fence_after_sync();
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    // chunk c + 2 j + u of sample m (TMEM lane m): 16 packed columns
                    const uint32_t col =
                        a_lane + (uint32_t)st * A_STAGE_COLS + (uint32_t)(2 * j + u) * A_CHUNK_COLS;
                    tc::tmem_st16(col, hl[j]);
                }
                // hand the stage to the MMA warp once the stores have landed
                tc::tmem_wait_st();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(a_full + st);
                ++n;
                // the previous step's variance partials, then this step's
                // mean-free dynamics
                if (bi == 0) {
                    if (k > 0) read_q(k - 1);
                    dynamics();
                }
                if (bi == ilast) send_mean();
            }
            if (nch_p < BURST) {                         // (no burst in this rank's steps)
                if (k > 0) read_q(k - 1);
                dynamics();
            }
            const float v_pre = mu3;
            // ---------------- the GP mean: every rank's shares -------------------------
            wait_cluster(xbar + buf, (uint32_t)(k >> 1) & 1u, abort_flag, a.err);
            float2 msum = make_float2(0.0f, 0.0f);
            float2 pm[8];
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p < 2 * CS) pm[p] = xm[(buf * 8 + p) * MT + m];
#pragma unroll
            for (int p = 0; p < 8; ++p)              // fixed order: identical on every rank
                if (p < 2 * CS) {
                    msum.x += pm[p].x;
                    msum.y += pm[p].y;
                }
            const float mean_v = a.sf2 * msum.x, mean_w = a.sf2 * msum.y;

            // ---------------- mean dynamics: add the GP mean -----------------------
            mu0 = nX; mu1 = nY; mu2 = nT; mu3 = nV0 + mean_v; mu4 = nW0 + mean_w;
            // ---------------- hand the step to the scoring warps -------------------
            // (rank r scores the samples m = r mod CS; the buffer of step k is
            // reused at step k + 2, once the scoring warps released it)
            if (warp < 4) {
                float* sstk = sst + (k & 1) * nown * SST;
                if (k >= 2) {
                    wait_or_abort(st_empty + (k & 1), (uint32_t)((k >> 1) - 1) & 1u, abort_flag, a.err);
                    __syncwarp();
                }
                if ((m % CS) == (int)rank) {
                    float* o = sstk + (m / CS) * SST;
                    o[0] = mu0; o[1] = mu1; o[2] = mu2; o[3] = mu3; o[4] = mu4;
                    o[5] = v_pre; o[6] = sn; o[7] = cs;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(st_full + (k & 1));
            }
        }
        // the variance partials of the last step
        if (a.T > 0) read_q(a.T - 1);
    } else {
        // ======================= scoring warps (Eq. 10-16) ======================
        // One step behind the producers: the covariance recursion (Eq. 10) and
        // the chance-constrained cost of the samples this rank scores, RC lanes
        // per sample (2 with CS = 4, else 1; two passes of 64 samples with
        // CS = 1).  The GP variance of a step is summed here from the ranks'
        // |V_m|^2 partials, which arrive during the producers' next step.
        const int nown = MT / CS;
        const int ct = tid - (NPROD + 32);
        const int RC = nown >= NCOST ? 1 : NCOST / nown;
        const int spp = NCOST / RC;                 // samples per pass
        const int cpart = ct % RC;
        float cost[2] = {0.0f, 0.0f};
        float Sg[2][15];                            // covariance upper triangles (sidx order)
#pragma unroll
        for (int js = 0; js < 2; ++js)
#pragma unroll
            for (int i = 0; i < 15; ++i) Sg[js][i] = 0.0f;
        float disc = 1.0f;
        for (int k = 0; k < a.T; ++k) {
            wait_or_abort(st_full + (k & 1), (uint32_t)(k >> 1) & 1u, abort_flag, a.err);
            __syncwarp();
            // the variance partials of step k (2 CS per scored sample) arrive on
            // qbar[k & 3] while the next step's kernel rows are computed; one
            // local arrival carries the expected bytes
            if (ct == 0) tc::mbar_expect_tx(qbar + (k & 3), (uint32_t)(2 * MT * 4));
            const float* sstk = sst + (k & 1) * nown * SST;
#pragma unroll
            for (int js = 0; js < 2; ++js) {
                const int ci = ct / RC + js * spp;
                if (js * spp >= nown) break;            // warp-uniform
                const int mc = (int)rank + CS * ci;
                const int sc_me = tile * MT + mc;
                const bool cactive = sc_me < a.K;
                const float* o = sstk + ci * SST;
                const float px = o[0], py = o[1];
                // Eq. 10: Sigma' = A Sigma A^T + diag(0, 0, 0, s, s), A the Jacobian
                // of the unicycle step at the pre-step state (s is added below, once
                // the variance partials are in: the position block read by the
                // constraints does not depend on it)
                {
                    const float vp = o[5], sn = o[6], cs = o[7];
                    const float a02 = -a.dt * vp * sn, a03 = a.dt * cs;
                    const float a12 = a.dt * vp * cs, a13 = a.dt * sn;
                    float* S = Sg[js];
                    const float S00 = S[0], S01 = S[1], S02 = S[2], S03 = S[3], S04 = S[4], S11 = S[5],
                                S12 = S[6], S13 = S[7], S14 = S[8], S22 = S[9], S23 = S[10], S24 = S[11],
                                S33 = S[12], S34 = S[13], S44 = S[14];
                    const float B00 = S00 + a02 * S02 + a03 * S03, B01 = S01 + a02 * S12 + a03 * S13,
                                B02 = S02 + a02 * S22 + a03 * S23, B03 = S03 + a02 * S23 + a03 * S33,
                                B04 = S04 + a02 * S24 + a03 * S34;
                    const float B11 = S11 + a12 * S12 + a13 * S13, B12 = S12 + a12 * S22 + a13 * S23,
                                B13 = S13 + a12 * S23 + a13 * S33, B14 = S14 + a12 * S24 + a13 * S34;
                    const float B22 = S22 + a.dt * S24, B23 = S23 + a.dt * S34, B24 = S24 + a.dt * S44;
                    const float B33 = a.av * S33, B34 = a.av * S34;
                    const float B44 = a.aw * S44;
                    S[0] = B00 + a02 * B02 + a03 * B03;
                    S[1] = B01 + a12 * B02 + a13 * B03;
                    S[2] = B02 + a.dt * B04;
                    S[3] = a.av * B03;
                    S[4] = a.aw * B04;
                    S[5] = B11 + a12 * B12 + a13 * B13;
                    S[6] = B12 + a.dt * B14;
                    S[7] = a.av * B13;
                    S[8] = a.aw * B14;
                    S[9] = B22 + a.dt * B24;
                    S[10] = a.av * B23;
                    S[11] = a.aw * B24;
                    S[12] = a.av * B33;
                    S[13] = a.aw * B34;
                    S[14] = a.aw * B44;
                }
                float sxx = Sg[js][0], sxy = Sg[js][1], syy = Sg[js][5];
                if (a.nom_sxy) {
                    sxx = __ldg(a.nom_sxy + 3 * k);
                    sxy = __ldg(a.nom_sxy + 3 * k + 1);
                    syy = __ldg(a.nom_sxy + 3 * k + 2);
                }
                const int2 oc = lane_cands(a, px, py);     // candidate segments of this position
                const float lmax = fmaxf(0.0f, 0.5f * (sxx + syy) + hypotf(0.5f * (sxx - syy), sxy));
                float om = FLT_MAX;
                for (int ob = cpart; ob < a.O; ob += RC) {
                    const float cx = obsp[3 * ob], cy = obsp[3 * ob + 1], R = obsp[3 * ob + 2];
                    const float dx = px - cx, dy = py - cy;
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
                float best = FLT_MAX;
                // candidates in groups of four per lane, their indices fetched
                // together (one memory latency per group instead of one per candidate)
                for (int i0 = cpart; i0 < oc.y; i0 += 4 * RC) {
                    int gsg[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int i = i0 + j * RC;
                        gsg[j] = i < oc.y ? lane_seg(a, oc, i) : -1;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (gsg[j] < 0) continue;
                        const float4 sg = segp[gsg[j]];
                        const float il2 = il2p[gsg[j]];
                        const float qx0 = px - sg.x, qy0 = py - sg.y;
                        const float t = fminf(fmaxf((qx0 * sg.z + qy0 * sg.w) * il2, 0.0f), 1.0f);
                        const float qx = qx0 - t * sg.z, qy = qy0 - t * sg.w;
                        best = fminf(best, qx * qx + qy * qy);
                    }
                }
                for (int o2 = RC >> 1; o2 > 0; o2 >>= 1) {       // within the sample's lanes
                    om = fminf(om, __shfl_xor_sync(0xffffffffu, om, o2));
                    best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o2));
                }
                // GP variance s = sf2 - |V_m|^2, the partials summed in a fixed order
                wait_cluster_or_abort(qbar + (k & 3), (uint32_t)(k >> 2) & 1u, abort_flag, a.err);
                float qsum = 0.0f;
                for (int p = 0; p < 2 * CS; ++p) qsum += xq[((k & 3) * 2 * CS + p) * nown + ci];
                const float sv = fmaxf(0.0f, a.sf2 - qsum * cl.qscale);
                Sg[js][12] += sv;
                Sg[js][14] += sv;
                if (cpart == 0) {
                    const float omargin = om, e2min = best;
                    const float e_lane = sqrtf(e2min);
                    const float rbar = a.r - a.sq_chi2 * sqrtf(lmax);
                    const float vv = o[3];
                    float stage = a.c_var * (sv + sv) + a.c_speed * (a.v_des - vv) * (a.v_des - vv);
                    if (omargin <= 0.0f) stage += a.c_coll;
                    const float lmargin = e_lane - rbar;
                    stage += a.c_dev * e_lane;
                    if (lmargin > 0.0f) stage += a.c_lane * disc;
                    stage += goal_cost(a, k, px, py);                     // Eq. 12 goal terms
                    cost[js] += stage;
                    if (TRACE && cactive) {
                        const size_t sk = (size_t)sc_me * a.T + k;
                        if (a.tr_mu)
                            for (int i = 0; i < 5; ++i) a.tr_mu[sk * 5 + i] = o[i];
                        if (a.tr_sig)
                            for (int i = 0; i < 15; ++i) a.tr_sig[sk * 15 + i] = Sg[js][i];
                        if (a.tr_stage) a.tr_stage[sk] = stage;
                        if (a.tr_margin) {
                            a.tr_margin[sk * 2] = lmargin;
                            a.tr_margin[sk * 2 + 1] = (a.O > 0) ? omargin : __int_as_float(0x7f800000);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(st_empty + (k & 1));
            disc *= 0.9f;
        }
#pragma unroll
        for (int js = 0; js < 2; ++js) {
            const int ci = ct / RC + js * spp;
            if (js * spp >= nown) break;
            const int sc_me = tile * MT + (int)rank + CS * ci;
            if (cpart == 0 && sc_me < a.K && a.costs) a.costs[sc_me] = cost[js];
        }
    }
    // no CTA leaves while a peer may still write into its shared memory
    tc::fence_before_sync();
    __syncthreads();
    cluster_sync_all();
    if (warp == 0) tc::tmem_dealloc(taddr, TM_COLS);
}

}  // namespace

int cl_smem_bytes(const ClArgs& cl, int S, int O) {
    return cl_layout(cl.npc, cl.scene_smem ? S : 0, cl.scene_smem ? O : 0).total;
}

// whether at least one cluster of this shape fits on the device
bool cl_schedulable(const ClArgs& cl, int S, int O, int device) {
    (void)device;
    const int smem = cl_smem_bytes(cl, S, O);
    if (cudaFuncSetAttribute(k_rollout_cl<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl.cs);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_rollout_cl<0, false>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters > 0;
}

int launch_rollout_cl(const RolloutArgs& a, const ClArgs& cl, int fmt, bool trace, cudaStream_t st) {
    const int smem = cl_smem_bytes(cl, a.S, a.O);
    const int ntile = (a.K + MT - 1) / MT;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntile * cl.cs));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (fmt == 0) {
        if (trace) {
            GPM_CUDA(cudaFuncSetAttribute(k_rollout_cl<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            e = cudaLaunchKernelEx(&cfg, k_rollout_cl<0, true>, a, cl);
        } else {
            GPM_CUDA(cudaFuncSetAttribute(k_rollout_cl<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            e = cudaLaunchKernelEx(&cfg, k_rollout_cl<0, false>, a, cl);
        }
    } else {
        if (trace) {
            GPM_CUDA(cudaFuncSetAttribute(k_rollout_cl<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            e = cudaLaunchKernelEx(&cfg, k_rollout_cl<1, true>, a, cl);
        } else {
            GPM_CUDA(cudaFuncSetAttribute(k_rollout_cl<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            e = cudaLaunchKernelEx(&cfg, k_rollout_cl<1, false>, a, cl);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "launch_rollout_cl");
    GPM_CUDA(cudaGetLastError());
    return 0;
}

}  // namespace gpm
