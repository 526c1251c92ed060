// Fused MPPI rollout with the GP variance contraction on the tensor cores
// (tcgen05, split 16-bit operands, FP32 accumulation in TMEM).
//
// Same method as the FP32 rollout (Alg. 1 Step 1: noise, clamp, GP mean and
// variance, Eq. 10 mean/covariance, Eq. 11-16 costs); only the dense part
// of the variance, V = K* L^-T with |V_m|^2 = |L^-1 k*_m|^2, moves to the
// tensor cores.  Operands are split into a high and a low 16-bit part
// (x = hi + lo, both FP16 or both BF16) and the three products hi*hi, hi*lo,
// lo*hi are accumulated in FP32 (or, for the three-term BF16 split, x = hi +
// mid + lo and six products); the queries are scaled to a_j = k*_j / sf2 in
// [0, 1] and L^-T by a power of two cB so that both fit the 16-bit range.
// A terrain ensemble (Eq. 3) runs the same body over its GPs' factors stacked
// block-diagonally (MmaTerrains): each GP's passes use its own query scaling
// and stages, and the step mixes the GPs' means and variances.
// The tensor core's FP32 accumulation rounds at every MMA relative to the
// accumulator's magnitude, so its error grows with the number of MMAs that
// add into one accumulator.  For large training sets (mm.lo_set) hi*hi goes
// to one TMEM column set and the two small products to a second one, added
// only at the pass end: the large accumulator then sees one addition per
// chunk instead of three, which keeps the variance near FP32 accuracy at
// N = 2048, at the price of output passes half as wide.
//
// CTA = 128 samples (the MMA M), 256 producer threads: thread t serves
// sample t % 128 and half h = t / 128 of every shared loop.  The output
// columns of V are processed in passes of up to 512 columns (one TMEM
// allocation), or of 256 with the low column set in the other half.  The
// factor's 128-column blocks go to the tensor cores in pairs (MMA N = 256;
// a pair whose lower block has passed its last stage, the diagonal of the
// triangle, runs its upper block alone, N = 128).  The reduction dimension streams in stages of 32
// training points (two MMA K-steps) through a ring of shared-memory stages:
// per stage the producers compute the kernel-row tile (exp2 on the SFU), one
// thread fetches the pre-arranged L^-T pieces of the active pairs with one
// bulk copy per part, and one warp issues 3 MMAs per pair and K-step and
// commits them to the stage's mbarrier.  Stages of 32 points halve the
// handshakes per MMA against 16-point ones: the issuing warp's per-stage
// bookkeeping, not the tensor pipe, bounded the 16-point design.  At the end
// of a pass each thread reads its sample's TMEM row (both column sets, added,
// with mm.lo_set) and sums the squares.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cfloat>

#include "common.cuh"
#include "rollout_fp32_body.cuh"
#include "tc05.cuh"

namespace gpm {
namespace {

constexpr int MT = 128;               // samples per CTA (the MMA M)
constexpr int NPROD = 256;            // producer threads (warps 0-7): two per sample
constexpr int THREADS = NPROD + 64;   // + warp 8 (MMA issuer) + warp 9 (tile loader)
constexpr int KCS = 32;               // training points per stage (two MMA K-steps of 16)
constexpr int BLK = 128;              // output columns per block of L^-T
constexpr int PAIR = 2 * BLK;         // output columns per MMA (a pair of blocks, MMA N = 256)
constexpr int LO_COL = 256;           // first TMEM column of the low set
constexpr int NSTAGE = 6;             // maximum pipeline depth (fewer when the training set is large)
constexpr int A_PART = MT * KCS * 2;                        // 8 KiB: kernel-row tile, one part
constexpr int P_PART = PAIR * KCS * 2;                      // 16 KiB: factor pair piece, one part
// a stage: the A tile parts (hi, lo[, mid]), then up to ppp pair pieces hi,
// then ppp lo[, then ppp mid] (ppp = pairs per pass: a pass fills the 512
// TMEM columns, two pairs, or one pair per column set with mm.lo_set; parts =
// 2, or 3 for the three-term BF16 split)
__host__ __device__ constexpr int stage_bytes(int ppp, int parts) { return parts * (A_PART + ppp * P_PART); }
__host__ __device__ constexpr int pairs_per_pass(int lo_set) { return lo_set ? 1 : 2; }
constexpr uint64_t kWaitNs = 2000000000ull;

// Shared-memory layout for a given pipeline depth and padded training-set size.
struct MLayout {
    int bars, tslot, abort_flag, qh, mh, ep, om, xs, al, seg, il2, obs, total;
};

__host__ __device__ inline MLayout mma_layout(int nstage, int NpM, int S, int O, int ppp, int parts, int M) {
    MLayout L;
    L.bars = nstage * stage_bytes(ppp, parts);                     // a_full, b_full, empty [NSTAGE] + pass_done, tmem_free, x_res
    L.tslot = L.bars + 8 * (3 * NSTAGE + 3);
    L.abort_flag = L.tslot + 4;
    L.qh = ((L.abort_flag + 4 + 15) / 16) * 16;  // M x 2 x 128 floats: |V|^2 halves per GP
    L.mh = L.qh + M * 2 * MT * 4;                // M x 2 x 128 float2: mean partials per GP
    L.ep = L.mh + M * 2 * MT * 8;                // 2 x 128 floats
    L.om = L.ep + 2 * MT * 4;                    // 2 x 128 floats
    L.xs = ((L.om + 2 * MT * 4 + 127) / 128) * 128;   // NpM x 4 floats: scaled inputs, pair layout
    L.al = L.xs + NpM * 16;                      // NpM x 2 floats: alpha, pair layout
    L.seg = L.al + NpM * 8;                      // S float4: lane segments
    L.il2 = L.seg + S * 16;                      // S floats
    L.obs = L.il2 + ((S + 3) / 4) * 16;          // O x 3 floats: obstacles
    L.total = L.obs + O * 12;
    return L;
}

// deepest pipeline that fits (0 if none)
inline int mma_stages(int NpM, int S, int O, int optin, int ppp, int parts, int M) {
    for (int s = NSTAGE; s >= 2; --s)
        if (mma_layout(s, NpM, S, O, ppp, parts, M).total <= optin) return s;
    return 0;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_addr(bar))
        : "memory");
}

// hi/lo split of two values into packed 16-bit pairs (element a in the low half)
template <int FMT>
__device__ __forceinline__ void split2(float a, float b, uint32_t* hi, uint32_t* lo) {
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

// Three-term BF16 split of two values: hi = rn(a), mid = rn(a - hi), lo =
// rn(a - hi - mid), 8 + 8 + 8 significant bits; each residual is exact (one
// mixed-precision fma with the BF16 part taken as is).
__device__ __forceinline__ void split3(float a, float b, uint32_t* hi, uint32_t* mid, uint32_t* lo) {
    float ra, rb, sa, sb;
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    tc::split_resid<1>(*hi, a, b, ra, rb);
    const __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
    *mid = *reinterpret_cast<const uint32_t*>(&m);
    tc::split_resid<1>(*mid, ra, rb, sa, sb);
    const __nv_bfloat162 l = __floats2bfloat162_rn(sa, sb);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Bounded wait that gives up at once when another role has aborted.  The
// flag is read only once the phase is found incomplete: a phase that did
// complete is safe to use, and the fast path stays one instruction.
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

__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

// 2^x (the hardware approximation; results below the normal range flush to 0,
// far below what a 16-bit split operand can carry)
__device__ __forceinline__ float ex2_ftz(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

// R producer threads per sample: a CTA owns MTC = 256 / R samples (rows
// m >= MTC of the 128-row MMA tile are never written; their TMEM lanes are
// not read) and each thread makes KPT = 32 / R points of every stage.
// tmem_given: kTmemAlloc to allocate the 512 TMEM columns here (and free them
// at the end), else the base of columns the caller holds (the persistent
// batched kernel allocates once per CTA).
constexpr uint32_t kTmemAlloc = 0xFFFFFFFFu;

template <int FMT, int R, bool TRACE>
__device__ __forceinline__ void rollout_mma_body(const RolloutArgs& a, const MmaArgs& mm, int tile,
                                                 unsigned char* sm, uint32_t tmem_given) {
    constexpr int MTC = NPROD / R;
    constexpr int KPT = KCS / R;
    constexpr int NPARTS = FMT == 2 ? 3 : 2;    // operand parts: hi, lo (, mid)
    const int nstage = mm.stages;
    const int Ssm = mm.scene_smem ? a.S : 0, Osm = mm.scene_smem ? a.O : 0;
    const int ppp = pairs_per_pass(mm.lo_set);  // block pairs per pass
    const int bpp = 2 * ppp;                    // output blocks per pass
    const int STAGE = stage_bytes(ppp, NPARTS);
    const MLayout L = mma_layout(nstage, mm.nblocks * BLK, Ssm, Osm, ppp, NPARTS, mm.tr.M);
    uint64_t* a_full = reinterpret_cast<uint64_t*>(sm + L.bars);
    uint64_t* b_full = a_full + NSTAGE;
    uint64_t* empty = b_full + NSTAGE;
    uint64_t* pass_done = empty + NSTAGE;
    uint64_t* tmem_free = pass_done + 1;
    uint64_t* x_res = tmem_free + 1;            // the training set copied in
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tslot);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + L.abort_flag);
    float4* xs_s = reinterpret_cast<float4*>(sm + L.xs);
    float2* al_s = reinterpret_cast<float2*>(sm + L.al);
    float4* seg_s = reinterpret_cast<float4*>(sm + L.seg);
    float* il2_s = reinterpret_cast<float*>(sm + L.il2);
    float* obs_s = reinterpret_cast<float*>(sm + L.obs);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NB = mm.nblocks;                 // 128-column blocks of L^-T
    const int NP = (NB + 1) / 2;               // block pairs (the last one half empty for odd NB)
    const MmaTerrains& TR = mm.tr;             // the GPs' block ranges (one range for a single GP)

    if (tid == 0) {
        for (int i = 0; i < nstage; ++i) {
            tc::mbar_init(a_full + i, NPROD / 32);
            tc::mbar_init(b_full + i, 1);
            tc::mbar_init(empty + i, 1);
        }
        tc::mbar_init(pass_done, 1);
        tc::mbar_init(tmem_free, NPROD / 32);
        tc::mbar_init(x_res, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
        // scaled training inputs and alpha in pair layout (two points per
        // 16-byte line; rows past N hold a far point and alpha 0) by two bulk
        // copies (TMA engine)
        const uint32_t xb = (uint32_t)(NB * BLK) * 16u, ab = (uint32_t)(NB * BLK) * 8u;
        tc::mbar_expect_tx(x_res, xb + ab);
        if (xb) {
            bulk_copy(xs_s, mm.xa, xb, x_res);
            bulk_copy(al_s, mm.xa + 4 * NB * BLK, ab, x_res);
        }
    }
    // lane segments and obstacles too: the cost phase reads them every step
    for (int i = tid; i < Ssm; i += THREADS) {
        seg_s[i] = __ldg(a.seg + i);
        il2_s[i] = __ldg(a.seg_il2 + i);
    }
    for (int i = tid; i < 3 * Osm; i += THREADS) obs_s[i] = __ldg(a.obst + i);
    // a scene too large for shared memory is read from global memory instead
    const float4* segp = mm.scene_smem ? seg_s : a.seg;
    const float* il2p = mm.scene_smem ? il2_s : a.seg_il2;
    const float* obsp = mm.scene_smem ? obs_s : a.obst;
    if (tmem_given == kTmemAlloc) {
        if (warp == 0 && NB > 0) tc::tmem_alloc(tslot, 512);
    } else if (tid == 0) {
        *tslot = tmem_given;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;

    if (warp >= NPROD / 32) {
        // ======================= control warps ===============================
        if (NB == 0) return;
        const bool issuer = (warp == NPROD / 32);
        // one loader thread; the issuer is a converged warp whose elected lane
        // issues the MMAs (its operand arithmetic stays warp-uniform)
        if (!issuer && lane != 0) return;
        constexpr int TYPE = FMT == 0 ? 0 : 1;                  // FP16 or BF16 operands
        const uint32_t idesc2 = tc::idesc_f16(TYPE, MT, PAIR);  // a block pair
        const uint32_t idesc1 = tc::idesc_f16(TYPE, MT, BLK);   // one block of a pair
        // base descriptors of stage 0's A tile (128 rows, slabs MT * 16 bytes
        // apart) and pair pieces (256 rows, slabs PAIR * 16 bytes apart); stage,
        // K-step and pair offsets are multiples of 16 bytes inside shared memory
        const uint64_t dA0 = tc::smem_desc(tc::smem_addr(sm), MT * 16, 128);
        const uint64_t dB0 = tc::smem_desc(tc::smem_addr(sm), PAIR * 16, 128);
        int st = 0;                  // ring position: stage and the parity of its current use
        uint32_t ph = 0;
        bool wrapped = false;
        uint32_t pc = 0;
        for (int k = 0; k < a.T; ++k) {
          for (int t = 0; t < TR.M; ++t) {
            // GP t: its blocks [tb0, tb1) in passes of bpp blocks; its stages
            // start at c0 (its first training point), block b needs stages
            // c0 .. 4b+3 (the factor is block-diagonal)
            const int tb0 = TR.blk0[t], tb1 = TR.blk0[t + 1];
            const int c0 = 4 * tb0;
            for (int b0 = tb0; b0 < tb1; b0 += bpp, ++pc) {
                const int b1 = min(tb1, b0 + bpp);
                const int p0 = b0 >> 1, p1 = (b1 + 1) >> 1;
                const int nchunk = 4 * b1;
                if (issuer && pc > 0) {
                    wait_or_abort(tmem_free, (pc - 1) & 1u, abort_flag, a.err);
                    __syncwarp();
                    tc::fence_after_sync();
                }
                for (int c = c0; c < nchunk; ++c) {
                    unsigned char* stage = sm + st * STAGE;
                    // blocks active at stage c: [ba, b1), ba = max(b0, c / 4)
                    const int ba = max(b0, c >> 2);
                    const int pa = ba >> 1;
                    if (!issuer) {
                        // tile loader: wait until the stage's previous MMAs are done;
                        // the active pairs' pieces are contiguous in the tile
                        // arrays, one copy per part
                        if (wrapped && !wait_or_abort(empty + st, ph ^ 1u, abort_flag, a.err)) {
                            if (++st == nstage) { st = 0; ph ^= 1u; wrapped = true; }
                            continue;
                        }
                        const uint32_t bytes = (uint32_t)((p1 - pa) * P_PART);
                        tc::mbar_expect_tx(b_full + st, (uint32_t)NPARTS * bytes);
                        const size_t off = ((size_t)c * NP + pa) * (P_PART / 2);
                        unsigned char* dst = stage + NPARTS * A_PART + (pa - p0) * P_PART;
                        bulk_copy(dst, mm.Bhi + off, bytes, b_full + st);
                        bulk_copy(dst + ppp * P_PART, mm.Blo + off, bytes, b_full + st);
                        if (NPARTS == 3) bulk_copy(dst + 2 * ppp * P_PART, mm.Bmid + off, bytes, b_full + st);
                    } else {
                        bool ok = wait_or_abort(a_full + st, ph, abort_flag, a.err);
                        ok = ok && wait_or_abort(b_full + st, ph, abort_flag, a.err);
                        if (__all_sync(0xffffffffu, ok)) {
                            tc::fence_after_sync();
                            // descriptors by adds on precomputed bases: rebuilding them per
                            // MMA makes the single issuing thread the bottleneck
                            const uint64_t dAh = dA0 + (uint64_t)((st * STAGE) >> 4);
                            const uint64_t dAl = dAh + (uint64_t)(A_PART >> 4);
                            for (int p = pa; p < p1; ++p) {
                                // both blocks of the pair (N = 256), else the upper one
                                // (its lower block is done) or the lower one (no upper
                                // block: odd NB) with N = 128
                                const bool lower = 2 * p >= ba, upper = 2 * p + 1 < b1;
                                const int row0 = lower ? 0 : BLK;
                                const uint32_t id = (lower && upper) ? idesc2 : idesc1;
                                const uint64_t dBh = dB0 + (uint64_t)((st * STAGE + NPARTS * A_PART + (p - p0) * P_PART +
                                                                       row0 * 16) >> 4);
                                const uint64_t dBl = dBh + (uint64_t)((ppp * P_PART) >> 4);
                                const uint32_t d = taddr + (uint32_t)(2 * (p - p0) * BLK + row0);
#pragma unroll
                                for (int j = 0; j < 2; ++j) {
                                    // K-step j: A slabs 2j, 2j+1 (MT * 32 bytes on), pair slabs
                                    // 2j, 2j+1 (PAIR * 32 bytes on)
                                    const uint64_t ja = (uint64_t)((j * MT * 32) >> 4);
                                    const uint64_t jb = (uint64_t)((j * PAIR * 32) >> 4);
                                    const uint32_t acc = (c > c0 || j > 0) ? 1u : 0u;
                                    if (NPARTS == 3)
                                        tc::mma6_split3_elect(d, d + (uint32_t)LO_COL, dAh + ja,
                                                              dAh + ja + (uint64_t)((2 * A_PART) >> 4), dAl + ja,
                                                              dBh + jb, dBh + jb + (uint64_t)((2 * ppp * P_PART) >> 4),
                                                              dBl + jb, id, acc);
                                    else if (mm.lo_set)
                                        tc::mma3_split2_elect(d, d + (uint32_t)LO_COL, dAh + ja, dAl + ja, dBh + jb,
                                                              dBl + jb, id, acc);
                                    else
                                        tc::mma3_split_elect(d, dAh + ja, dAl + ja, dBh + jb, dBl + jb, id, acc);
                                }
                            }
                            tc::mma_commit_elect(empty + st);
                            if (c == nchunk - 1) tc::mma_commit_elect(pass_done);
                        }
                    }
                    if (++st == nstage) { st = 0; ph ^= 1u; wrapped = true; }
                }
            }
          }
        }
        return;
    }

    // ========================== producer warps =================================
    wait_or_abort(x_res, 0u, abort_flag, a.err);     // the training set in shared memory
    const int m = tid % MTC;           // sample within the CTA
    const int u = tid / MTC;           // which of its R threads
    const int mr = tid & (MT - 1);     // TMEM lane this thread reads at a pass end
    const int hr = tid >> 7;           // which half of the pass's columns
    const int s0 = tile * MTC;
    const int mvalid = min(MTC, a.K - s0);
    const bool active = m < mvalid;
    const int s_me = s0 + (active ? m : 0);
    const ulonglong2* xs2 = reinterpret_cast<const ulonglong2*>(xs_s);   // pair layout
    const ulonglong2* al2 = reinterpret_cast<const ulonglong2*>(al_s);
    float* qh = reinterpret_cast<float*>(sm + L.qh);
    float2* mh = reinterpret_cast<float2*>(sm + L.mh);
    float* ep = reinterpret_cast<float*>(sm + L.ep);
    float* omh = reinterpret_cast<float*>(sm + L.om);

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
    float S00 = 0, S01 = 0, S02 = 0, S03 = 0, S04 = 0, S11 = 0, S12 = 0, S13 = 0, S14 = 0,
          S22 = 0, S23 = 0, S24 = 0, S33 = 0, S34 = 0, S44 = 0;
    float cost = 0.0f, disc = 1.0f;
    uint32_t n = 0, pc = 0;          // stages produced, passes done
    int st = 0;                      // ring position: stage and the parity of its current use
    uint32_t ph = 0;
    bool wrapped = false;

    for (int k = 0; k < a.T; ++k) {
        // ---------------- P1: noise, clamp, query (both halves) ------------
        const float2 e = control_eps((uint32_t)k, (uint32_t)s_me, it0, it1, a.key0, a.key1,
                                     a.sig_v, a.sig_w);
        float2 ut;
        ut.x = fminf(fmaxf(__ldg(a.U + 2 * k) + e.x, a.umin0), a.umax0);
        ut.y = fminf(fmaxf(__ldg(a.U + 2 * k + 1) + e.y, a.umin1), a.umax1);
        if (u == 0 && active) a.u_tilde[(size_t)k * a.K + s_me] = ut;
        // ---------------- P2/P3: kernel-row tiles for the tensor cores ------
        for (int t = 0; t < TR.M; ++t) {
          // GP t: the query scaled by its inverse lengthscales, its blocks
          // [tb0, tb1) and stages from c0 on
          const float z0 = mu3 * TR.zscale[t][0], z1 = mu4 * TR.zscale[t][1];
          const float z2 = ut.x * TR.zscale[t][2], z3 = ut.y * TR.zscale[t][3];
          const uint64_t zz0 = tc::f2pack(z0, z0), zz1 = tc::f2pack(z1, z1);
          const uint64_t zz2 = tc::f2pack(z2, z2), zz3 = tc::f2pack(z3, z3);
          const int tb0 = TR.blk0[t], tb1 = TR.blk0[t + 1];
          const int c0 = 4 * tb0;
          float qpart = 0.0f, mv = 0.0f, mw = 0.0f, cv = 0.0f, cw = 0.0f;
          for (int b0 = tb0; b0 < tb1; b0 += bpp, ++pc) {
            const int b1 = min(tb1, b0 + bpp);
            const int nchunk = 4 * b1;
            const bool last_pass = (b1 == tb1);
            for (int c = c0; c < nchunk; ++c, ++n) {
                unsigned char* stage = sm + st * STAGE;
                // this thread's KPT training points of the stage, two at a time
                // (packed f32x2 arithmetic on the pair layout)
                const int pb = (c * KCS + u * KPT) / 2;
                float av[KPT];
#pragma unroll
                for (int q = 0; q < KPT / 2; ++q) {
                    const ulonglong2 xa = xs2[2 * (pb + q)], xb = xs2[2 * (pb + q) + 1];
                    const uint64_t d0 = tc::f2sub(zz0, xa.x), d1 = tc::f2sub(zz1, xa.y);
                    const uint64_t d2 = tc::f2sub(zz2, xb.x), d3 = tc::f2sub(zz3, xb.y);
                    uint64_t t = tc::f2mul(d0, d0);
                    t = tc::f2fma(d1, d1, t);
                    t = tc::f2fma(d2, d2, t);
                    t = tc::f2fma(d3, d3, t);
                    float t0, t1;
                    tc::f2unpack(t, t0, t1);
                    av[2 * q] = ex2_ftz(-t0);
                    av[2 * q + 1] = ex2_ftz(-t1);
                }
                if (last_pass) {
                    // the stage's mean terms as packed partial sums, then one
                    // compensated addition per output
                    uint64_t pv = 0ull, pw = 0ull;
#pragma unroll
                    for (int q = 0; q < KPT / 2; ++q) {
                        const ulonglong2 al = al2[pb + q];
                        const uint64_t k2 = tc::f2pack(av[2 * q], av[2 * q + 1]);
                        pv = tc::f2fma(k2, al.x, pv);
                        pw = tc::f2fma(k2, al.y, pw);
                    }
                    float pv0, pv1, pw0, pw1;
                    tc::f2unpack(pv, pv0, pv1);
                    tc::f2unpack(pw, pw0, pw1);
                    kahan_add(mv, cv, pv0 + pv1);
                    kahan_add(mw, cw, pw0 + pw1);
                }
                uint32_t hw[KPT / 2], lw[KPT / 2], mw[NPARTS == 3 ? KPT / 2 : 1];
#pragma unroll
                for (int q = 0; q < KPT / 2; ++q) {
                    if constexpr (NPARTS == 3)
                        split3(av[2 * q], av[2 * q + 1], &hw[q], &mw[q], &lw[q]);
                    else
                        split2<FMT>(av[2 * q], av[2 * q + 1], &hw[q], &lw[q]);
                }
                // the stage is free once the MMAs that last read it completed
                if (wrapped) wait_or_abort(empty + st, ph ^ 1u, abort_flag, a.err);
                {
                    // points u KPT .. u KPT + KPT - 1 of the stage: slab (u KPT) / 8
                    // on, byte offset ((u KPT) % 8) * 2 within the sample's row
                    const int sl = (u * KPT) / 8, off = ((u * KPT) % 8) * 2;
                    unsigned char* ph_ = stage + sl * MT * 16 + m * 16 + off;
                    unsigned char* pl_ = ph_ + A_PART;
                    if (KPT >= 8) {
#pragma unroll
                        for (int gq = 0; gq < KPT / 8; ++gq) {
                            *reinterpret_cast<uint4*>(ph_ + gq * MT * 16) =
                                make_uint4(hw[4 * gq], hw[4 * gq + 1], hw[4 * gq + 2], hw[4 * gq + 3]);
                            *reinterpret_cast<uint4*>(pl_ + gq * MT * 16) =
                                make_uint4(lw[4 * gq], lw[4 * gq + 1], lw[4 * gq + 2], lw[4 * gq + 3]);
                            if constexpr (NPARTS == 3)
                                *reinterpret_cast<uint4*>(ph_ + 2 * A_PART + gq * MT * 16) =
                                    make_uint4(mw[4 * gq], mw[4 * gq + 1], mw[4 * gq + 2], mw[4 * gq + 3]);
                        }
                    } else {
                        *reinterpret_cast<uint2*>(ph_) = make_uint2(hw[0], hw[1 % (KPT / 2)]);
                        *reinterpret_cast<uint2*>(pl_) = make_uint2(lw[0], lw[1 % (KPT / 2)]);
                        if constexpr (NPARTS == 3)
                            *reinterpret_cast<uint2*>(ph_ + 2 * A_PART) = make_uint2(mw[0], mw[1 % (KPT / 2)]);
                    }
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(a_full + st);
                if (++st == nstage) { st = 0; ph ^= 1u; wrapped = true; }
            }
            // pass end: every MMA of the pass has landed in TMEM
            bool ok = wait_or_abort(pass_done, pc & 1u, abort_flag, a.err);
            ok = __all_sync(0xffffffffu, ok);        // tcgen05.ld below is warp-collective
            tc::fence_after_sync();
            if (ok && 32 * (warp & 3) < MTC) {
                const int half_cols = (b1 - b0) * BLK / 2;
                const uint32_t row = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
                // with the low set: V = main + low column sets (32 columns per
                // load pair); without: 64 columns of V per load pair
                const int step = mm.lo_set ? 32 : 64;
                const uint32_t second = mm.lo_set ? (uint32_t)LO_COL : 32u;
#pragma unroll 1
                for (int cc = 0; cc < half_cols; cc += step) {
                    float v[32], w[32];
                    const uint32_t col = row + (uint32_t)(hr * half_cols + cc);
                    tc::tmem_ld32x2(col, col + second, v, w);
                    float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
                    if (mm.lo_set) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float x0 = v[i] + w[i], x1 = v[8 + i] + w[8 + i];
                            const float x2 = v[16 + i] + w[16 + i], x3 = v[24 + i] + w[24 + i];
                            p0 = fmaf(x0, x0, p0);
                            p1 = fmaf(x1, x1, p1);
                            p2 = fmaf(x2, x2, p2);
                            p3 = fmaf(x3, x3, p3);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            p0 = fmaf(v[i], v[i], p0);
                            p1 = fmaf(v[16 + i], v[16 + i], p1);
                            p2 = fmaf(w[i], w[i], p2);
                            p3 = fmaf(w[16 + i], w[16 + i], p3);
                        }
                    }
                    qpart += (p0 + p1) + (p2 + p3);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_free);
          }
          qh[(2 * t + hr) * MT + mr] = qpart;
          mh[(t * R + u) * MTC + m] = make_float2(mv + cv, mw + cw);
        }
        producers_sync();
        // Eq. 3: mean sum_t w_t m_t and variance sum_t w_t^2 var_t (a single
        // GP has w = 1: the same arithmetic as without the sums)
        float mean_v = 0.0f, mean_w = 0.0f, s = 0.0f;
        for (int t = 0; t < TR.M; ++t) {
            const float q = (qh[2 * t * MT + m] + qh[(2 * t + 1) * MT + m]) * TR.qscale[t];
            float2 msum = mh[t * R * MTC + m];
#pragma unroll
            for (int i = 1; i < R; ++i) {
                const float2 mi = mh[(t * R + i) * MTC + m];
                msum.x += mi.x;
                msum.y += mi.y;
            }
            const float wsf = TR.w[t] * TR.sf2[t];
            mean_v += wsf * msum.x;
            mean_w += wsf * msum.y;
            s += TR.w[t] * TR.w[t] * fmaxf(0.0f, TR.sf2[t] - q);
        }
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
        for (int o = u; o < a.O; o += R) {
            const float cx = obsp[3 * o], cy = obsp[3 * o + 1], rad = obsp[3 * o + 2];
            const float dx = mu0 - cx, dy = mu1 - cy;
            const float rho = sqrtf(dx * dx + dy * dy);
            float spread;
            if (rho > 1e-9f) {
                const float nx = dx / rho, ny = dy / rho;
                spread = sqrtf(fmaxf(0.0f, nx * nx * sxx + 2.0f * nx * ny * sxy + ny * ny * syy));
            } else {
                spread = sqrtf(lmax);
            }
            om = fminf(om, (rho - rad) - a.phi_inv * spread);
        }
        // ---------------- P5: lane distance (segments split by half) -------
        float best = FLT_MAX;
        const int2 oc = lane_cands(a, mu0, mu1);           // candidate segments of this position
        for (int i = u; i < oc.y; i += R) {
            const int gsg = lane_seg(a, oc, i);
            const float4 sg = segp[gsg];
            const float il2 = il2p[gsg];
            const float px = mu0 - sg.x, py = mu1 - sg.y;
            const float t = fminf(fmaxf((px * sg.z + py * sg.w) * il2, 0.0f), 1.0f);
            const float qx = px - t * sg.z, qy = py - t * sg.w;
            best = fminf(best, qx * qx + qy * qy);
        }
        omh[u * MTC + m] = om;
        ep[u * MTC + m] = best;
        producers_sync();
        float omargin = omh[m], e2min = ep[m];
#pragma unroll
        for (int i = 1; i < R; ++i) {
            omargin = fminf(omargin, omh[i * MTC + m]);
            e2min = fminf(e2min, ep[i * MTC + m]);
        }
        const float e_lane = sqrtf(e2min);
        // ---------------- P6: stage cost ------------------------------------
        float stage = a.c_var * (s + s) + a.c_speed * (a.v_des - mu3) * (a.v_des - mu3);
        if (omargin <= 0.0f) stage += a.c_coll;
        const float lmargin = e_lane - rbar;
        stage += a.c_dev * e_lane;
        if (lmargin > 0.0f) stage += a.c_lane * disc;
        stage += goal_cost(a, k, mu0, mu1);                           // Eq. 12 goal terms
        cost += stage;
        disc *= 0.9f;
        if (TRACE && active && u == 0) {
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
    if (active && u == 0 && a.costs) a.costs[s_me] = cost;
    // after an abort, give copies and MMAs in flight a bounded time to land
    // before the shared memory and TMEM are released
    if (*abort_flag && tid == 0 && n > 0) {
        const uint64_t t0 = tc::global_ns();
        for (uint32_t i = (n >= (uint32_t)nstage ? n - (uint32_t)nstage : 0); i < n; ++i)
            while (!tc::mbar_try_wait(empty + (i % (uint32_t)nstage), (i / (uint32_t)nstage) & 1u) &&
                   tc::global_ns() - t0 < 200000000ull) {
            }
    }
    tc::fence_before_sync();
    producers_sync();
    if (tmem_given == kTmemAlloc && warp == 0 && NB > 0) tc::tmem_dealloc(taddr, 512);
}

template <int FMT, int R, bool TRACE>
__global__ void __launch_bounds__(THREADS, 1) k_rollout_mma(const RolloutArgs a, const MmaArgs mm) {
    extern __shared__ __align__(1024) unsigned char sm[];
    rollout_mma_body<FMT, R, TRACE>(a, mm, blockIdx.x, sm, kTmemAlloc);
}

// ---------------------------------------------------------------------------
// Batched step of many controllers as ONE persistent launch: one CTA per SM
// takes items from an atomic work queue until it is empty.  An item is
// (controller, sample tile, kind, producer threads per sample); kind 0 runs the
// FP32 CUDA-core rollout body on warps 0-7 (warps 8-9 wait), kinds 1 and 2 the
// tensor-core body with FP16 or BF16 split operands.  The queue holds the
// items in decreasing order of their estimated time (longest first).  The CTA
// holds its 512 TMEM columns for the whole launch; between items every role of
// the CTA meets at a barrier and the previous item's mbarriers are
// invalidated before their shared memory is reused.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

__device__ __forceinline__ int fp32_mtp(int Np) { return Np <= 1024 ? 32 : (Np <= 2048 ? 16 : 8); }

// invalidate the mbarriers an item initialised (thread 0, after every role is done)
__device__ void inval_item_barriers(const RolloutArgs& a, const MmaArgs& mm, int kind, unsigned char* sm) {
    if (kind == 0) {
        const int mtp = fp32_mtp(a.Np);
        const int off = mtp == 32 ? f32r::Smem<32>::bars(a.Np, a.stages)
                                  : (mtp == 16 ? f32r::Smem<16>::bars(a.Np, a.stages) : f32r::Smem<8>::bars(a.Np, a.stages));
        uint64_t* bars = reinterpret_cast<uint64_t*>(sm + off);
        for (int i = 0; i < f32r::WARPS * a.stages; ++i) mbar_inval(bars + i);
        return;
    }
    const MLayout L = mma_layout(mm.stages, mm.nblocks * BLK, mm.scene_smem ? a.S : 0, mm.scene_smem ? a.O : 0,
                                 pairs_per_pass(mm.lo_set), mm.parts, mm.tr.M);
    uint64_t* a_full = reinterpret_cast<uint64_t*>(sm + L.bars);
    for (int i = 0; i < mm.stages; ++i) {
        mbar_inval(a_full + i);
        mbar_inval(a_full + NSTAGE + i);
        mbar_inval(a_full + 2 * NSTAGE + i);
    }
    for (int i = 0; i < 3; ++i) mbar_inval(a_full + 3 * NSTAGE + i);
}

// The item bodies as separate (not inlined) functions: the persistent kernel's
// register budget (168 per thread at 320 threads: ten warps on four schedulers)
// is then met by each body on its own instead of by their union.
template <int FMT, int R>
__device__ __noinline__ void persistent_mma_item(const RolloutArgs& a, const MmaArgs& mm, int tile,
                                                 unsigned char* sm, uint32_t taddr) {
    rollout_mma_body<FMT, R, false>(a, mm, tile, sm, taddr);
}
template <int MTP>
__device__ __noinline__ void persistent_fp32_item(const RolloutArgs& a, const CUtensorMap* tm, int tile,
                                                  unsigned char* sm) {
    f32r::rollout_fp32_body<MTP, false>(a, tm, tile, sm);
}

__global__ void __launch_bounds__(THREADS, 1)
    k_rollout_persistent(const RolloutArgs* __restrict__ args, const MmaArgs* __restrict__ mms,
                         const CUtensorMap* __restrict__ tmaps, const int4* __restrict__ items, int nitems,
                         unsigned int* __restrict__ head, int ctl_off) {
    // no static shared memory (it would move the dynamic region off the
    // alignment the bulk and tensor copies need): the CTA's own words (TMEM
    // base, current and previous item) sit past the largest item layout
    extern __shared__ __align__(1024) unsigned char sm[];
    uint32_t& tbase = *reinterpret_cast<uint32_t*>(sm + ctl_off);
    int& cur = *reinterpret_cast<int*>(sm + ctl_off + 4);
    int& prev = *reinterpret_cast<int*>(sm + ctl_off + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        // held for the whole launch (one CTA per SM), so the permit is not relinquished
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         tc::smem_addr(&tbase))
                     : "memory");
    }
    if (tid == 0) prev = -1;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    for (;;) {
        if (tid == 0) {
            if (prev >= 0) {
                const int4 pi = items[prev];
                inval_item_barriers(args[pi.x], mms[pi.x], pi.z, sm);
            }
            cur = (int)atomicAdd(head, 1u);
        }
        __syncthreads();
        const int item = cur;
        if (item >= nitems) break;
        const int4 it = items[item];
        const RolloutArgs& a = args[it.x];
        if (it.z == 0) {
            if (warp < f32r::WARPS) {
                const int mtp = fp32_mtp(a.Np);
                if (mtp == 32) persistent_fp32_item<32>(a, tmaps + it.x, it.y, sm);
                else if (mtp == 16) persistent_fp32_item<16>(a, tmaps + it.x, it.y, sm);
                else persistent_fp32_item<8>(a, tmaps + it.x, it.y, sm);
            }
        } else {
            const MmaArgs& mm = mms[it.x];
            if (it.z == 1) {
                if (it.w == 2) persistent_mma_item<0, 2>(a, mm, it.y, sm, taddr);
                else if (it.w == 4) persistent_mma_item<0, 4>(a, mm, it.y, sm, taddr);
                else persistent_mma_item<0, 8>(a, mm, it.y, sm, taddr);
            } else if (it.z == 2) {
                if (it.w == 2) persistent_mma_item<1, 2>(a, mm, it.y, sm, taddr);
                else if (it.w == 4) persistent_mma_item<1, 4>(a, mm, it.y, sm, taddr);
                else persistent_mma_item<1, 8>(a, mm, it.y, sm, taddr);
            } else {
                if (it.w == 2) persistent_mma_item<2, 2>(a, mm, it.y, sm, taddr);
                else if (it.w == 4) persistent_mma_item<2, 4>(a, mm, it.y, sm, taddr);
                else persistent_mma_item<2, 8>(a, mm, it.y, sm, taddr);
            }
        }
        // every role of this CTA is done with the item (TMEM reads included)
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) prev = item;
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

}  // namespace

int launch_rollout_persistent(const RolloutArgs* args, const MmaArgs* mms, const CUtensorMap* tmaps,
                              const int4* items, int nitems, unsigned int* head, int grid, int smem,
                              cudaStream_t st) {
    if (nitems == 0) return GPMPPI_OK;
    const int ctl_off = ((smem + 15) / 16) * 16;
    const int total = ctl_off + 16;
    GPM_CUDA(cudaFuncSetAttribute(k_rollout_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, total));
    k_rollout_persistent<<<grid, THREADS, total, st>>>(args, mms, tmaps, items, nitems, head, ctl_off);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

int rollout_mma_stages(int NpM, int S, int O, int smem_optin, int lo_set, int parts, int M) {
    return mma_stages(NpM, S, O, smem_optin, pairs_per_pass(lo_set), parts, M);
}

int launch_rollout_mma(const RolloutArgs& a, const MmaArgs& mm, int fmt, bool trace, cudaStream_t st) {
    const int nstage = mm.stages;
    if (nstage < 2 || nstage > NSTAGE) return fail(GPMPPI_ERR_INVALID_ARG, "rollout: bad MMA pipeline depth");
    if (mm.rps != 2 && mm.rps != 4 && mm.rps != 8) return fail(GPMPPI_ERR_INVALID_ARG, "rollout: bad threads per sample");
    if ((fmt == 2) != (mm.parts == 3) || (fmt == 2 && !mm.lo_set))
        return fail(GPMPPI_ERR_INVALID_ARG, "rollout: operand parts do not match the format");
    if (mm.tr.M < 1 || mm.tr.M > kMaxTerrains || mm.tr.blk0[0] != 0 || mm.tr.blk0[mm.tr.M] != mm.nblocks)
        return fail(GPMPPI_ERR_INVALID_ARG, "rollout: bad GP block ranges");
    const int smem = mma_layout(nstage, mm.nblocks * BLK, mm.scene_smem ? a.S : 0, mm.scene_smem ? a.O : 0,
                                pairs_per_pass(mm.lo_set), mm.parts, mm.tr.M).total;
    const int mtc = NPROD / mm.rps;
    const int grid = (a.K + mtc - 1) / mtc;
#define GPM_LAUNCH_MMA(F, RR, TR)                                                                 \
    do {                                                                                          \
        auto kern = k_rollout_mma<F, RR, TR>;                                                     \
        GPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));  \
        kern<<<grid, THREADS, smem, st>>>(a, mm);                                                 \
    } while (0)
#define GPM_LAUNCH_MMA_R(F, TR)                          \
    do {                                                 \
        if (mm.rps == 2) GPM_LAUNCH_MMA(F, 2, TR);       \
        else if (mm.rps == 4) GPM_LAUNCH_MMA(F, 4, TR);  \
        else GPM_LAUNCH_MMA(F, 8, TR);                   \
    } while (0)
    if (fmt == 0) {
        if (trace) GPM_LAUNCH_MMA_R(0, true); else GPM_LAUNCH_MMA_R(0, false);
    } else if (fmt == 1) {
        if (trace) GPM_LAUNCH_MMA_R(1, true); else GPM_LAUNCH_MMA_R(1, false);
    } else {
        if (trace) GPM_LAUNCH_MMA_R(2, true); else GPM_LAUNCH_MMA_R(2, false);
    }
#undef GPM_LAUNCH_MMA_R
#undef GPM_LAUNCH_MMA
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

}  // namespace gpm

namespace gpm {

int rollout_mma_smem(const MmaArgs& mm, int S, int O) {
    return mma_layout(mm.stages, mm.nblocks * BLK, mm.scene_smem ? S : 0, mm.scene_smem ? O : 0,
                      pairs_per_pass(mm.lo_set), mm.parts, mm.tr.M).total;
}

}  // namespace gpm
