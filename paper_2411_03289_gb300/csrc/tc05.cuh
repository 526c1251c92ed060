// Blackwell (sm_100 family) tensor-core building blocks in inline PTX:
// shared-memory matrix descriptors, the tcgen05 instruction descriptor for
// kind::f16, tcgen05.mma / commit / ld, TMEM allocation, mbarriers and TMA.
//
// Operand layout used everywhere in this library ("slab-major", K-major,
// no swizzle): a tile of R rows x Kc elements (16-bit) is stored as Kc/8
// slabs; slab s holds, for every row r, the 16 bytes of elements
// [8s, 8s+8) at byte offset s * (R * 16) + r * 16.  In the descriptor's
// terms the 8 x 16-byte core matrices are 128 bytes apart along M/N
// (stride byte offset = 128) and R * 16 bytes apart along K (leading byte
// offset).  One MMA consumes K = 16 = two slabs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpm {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;          // descriptor version for tcgen05
    // base offset 0, LBO mode 0, layout type 0 (no swizzle)
    return d;
}

// Instruction descriptor for kind::f16 with FP32 accumulation, both operands
// K-major.  fmt: 0 = F16, 1 = BF16 (A and B always share it).
__host__ __device__ constexpr uint32_t idesc_f16(int fmt, int M, int N) {
    return (1u << 4)                              // D format: F32
           | ((uint32_t)fmt << 7)                 // A format
           | ((uint32_t)fmt << 10)                // B format
           | ((uint32_t)(N >> 3) << 17)           // N / 8
           | ((uint32_t)(M >> 4) << 24);          // M / 16
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The same product with A read from tensor memory: row i of the 128 x 16 A
// tile is TMEM lane i, its 16 elements packed two per 32-bit column (even
// element in the low half) in the 8 columns starting at a_tmem.
__device__ __forceinline__ void mma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The three products of one 16-point chunk and one output block of the split
// contraction, A and B in shared memory: A_hi B_hi (accumulating only if
// acc0 != 0), A_hi B_lo, A_lo B_hi, all into d_tmem.  Warp-collective: one
// elect.sync picks the lane that issues them.
__device__ __forceinline__ void mma3_split_elect(uint32_t d_tmem, uint64_t a_hi, uint64_t a_lo, uint64_t b_hi,
                                                 uint64_t b_lo, uint32_t idesc, uint32_t acc0) {
    asm volatile(
        "{\n\t.reg .pred e, p0, p1;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p0, %6, 0;\n\t"
        "setp.ne.b32 p1, 1, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %5, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %5, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %5, p1;\n\t}" ::"r"(d_tmem),
        "l"(a_hi), "l"(a_lo), "l"(b_hi), "l"(b_lo), "r"(idesc), "r"(acc0)
        : "memory");
}

// The same three products with the two small ones kept apart from the main
// one: A_hi B_hi into d_main (accumulating only if acc0 != 0), A_hi B_lo and
// A_lo B_hi into d_lo (the first of them accumulating only if acc0 != 0).
// The FP32 accumulator of the large product then sees one addition per
// chunk instead of three; the small products' rounding is 2^-11 (FP16) of
// the main one's.
__device__ __forceinline__ void mma3_split2_elect(uint32_t d_main, uint32_t d_lo, uint64_t a_hi, uint64_t a_lo,
                                                  uint64_t b_hi, uint64_t b_lo, uint32_t idesc, uint32_t acc0) {
    asm volatile(
        "{\n\t.reg .pred e, p0, p1;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p0, %7, 0;\n\t"
        "setp.ne.b32 p1, 1, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %4, %6, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %5, %6, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %3, %4, %6, p1;\n\t}" ::"r"(d_main), "r"(d_lo),
        "l"(a_hi), "l"(a_lo), "l"(b_hi), "l"(b_lo), "r"(idesc), "r"(acc0)
        : "memory");
}

// The six products of the three-term split (hi + mid + lo, 8 bits each) that
// carry 24 bits: A_hi B_hi into d_main (accumulating only if acc0 != 0);
// A_hi B_mid, A_mid B_hi, A_hi B_lo, A_lo B_hi and A_mid B_mid into d_lo (the
// first accumulating only if acc0 != 0).  The dropped products are below
// 2^-24 of the main one.  Warp-collective, one elected lane issues them.
__device__ __forceinline__ void mma6_split3_elect(uint32_t d_main, uint32_t d_lo, uint64_t a_hi, uint64_t a_mid,
                                                  uint64_t a_lo, uint64_t b_hi, uint64_t b_mid, uint64_t b_lo,
                                                  uint32_t idesc, uint32_t acc0) {
    asm volatile(
        "{\n\t.reg .pred e, p0, p1;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p0, %9, 0;\n\t"
        "setp.ne.b32 p1, 1, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %5, %8, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %6, %8, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %3, %5, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %7, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %5, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%1], %3, %6, %8, p1;\n\t}" ::"r"(d_main), "r"(d_lo),
        "l"(a_hi), "l"(a_mid), "l"(a_lo), "l"(b_hi), "l"(b_mid), "l"(b_lo), "r"(idesc), "r"(acc0)
        : "memory");
}

// Warp-collective commit: the whole (converged) warp executes it and one lane,
// chosen by elect.sync, issues it.
__device__ __forceinline__ void mma_commit_elect(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
            smem_addr(bar))
        : "memory");
}

// The same commit arriving on the mbarrier at bar's offset in every CTA of
// the cluster whose bit is set in cta_mask (not in this CTA unless its bit is
// set): a peer learns that this CTA's earlier MMAs have completed.
__device__ __forceinline__ void mma_commit_mc_elect(uint64_t* bar, uint16_t cta_mask) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}" ::"r"(
            smem_addr(bar)),
        "h"(cta_mask)
        : "memory");
}

// One ring stage of four 16-point chunks, A from tensor memory: for chunk
// j = 0 .. 3 the products A_hi,j x B_j (instruction descriptor i_hi) and
// A_lo,j x B_j (i_lo), all into d_tmem, then the commit that arrives on bar
// once they completed.  A_hi,j and A_lo,j start at TMEM columns a + 16 j and
// a + 16 j + 8; B_j's descriptor is b0 + j * bstep.  The first product
// accumulates only if acc0 != 0.  Warp-collective: one elect.sync picks the
// lane that issues all nine instructions, which keeps the issue cost per MMA
// below the tensor pipe's time for these small shapes.
__device__ __forceinline__ void mma_stage4_elect(uint32_t d_tmem, uint32_t a, uint64_t b0, uint64_t bstep,
                                                 uint64_t* bar, uint32_t acc0, uint32_t i_hi, uint32_t i_lo) {
    asm volatile(
        "{\n\t.reg .pred e, p0, p1;\n\t"
        ".reg .b32 a1, a2, a3, a4, a5, a6, a7;\n\t"
        ".reg .b64 b1, b2, b3;\n\t"
        "add.u32 a1, %1, 8;\n\tadd.u32 a2, %1, 16;\n\tadd.u32 a3, %1, 24;\n\t"
        "add.u32 a4, %1, 32;\n\tadd.u32 a5, %1, 40;\n\tadd.u32 a6, %1, 48;\n\t"
        "add.u32 a7, %1, 56;\n\t"
        "add.u64 b1, %2, %3;\n\tadd.u64 b2, b1, %3;\n\tadd.u64 b3, b2, %3;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p0, %5, 0;\n\t"
        "setp.ne.b32 p1, 1, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %6, p0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], %2, %7, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b1, %6, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b1, %7, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a4], b2, %6, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a5], b2, %7, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a6], b3, %6, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [a7], b3, %7, p1;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%4];\n\t}" ::"r"(d_tmem),
        "r"(a), "l"(b0), "l"(bstep), "r"(smem_addr(bar)), "r"(acc0), "r"(i_hi), "r"(i_lo)
        : "memory");
}

// The same four chunks with A in shared memory: A_hi,j at descriptor a_j,
// A_lo,j at a_j + lo_off; every product accumulates; no commit.
__device__ __forceinline__ void mma_stage4_sa_elect(uint32_t d_tmem, uint64_t a0, uint64_t a1, uint64_t a2,
                                                    uint64_t a3, uint64_t lo_off, uint64_t b0, uint64_t bstep,
                                                    uint32_t i_hi, uint32_t i_lo) {
    asm volatile(
        "{\n\t.reg .pred e, p1;\n\t"
        ".reg .b64 l0, l1, l2, l3, b1, b2, b3;\n\t"
        "add.u64 l0, %1, %5;\n\tadd.u64 l1, %2, %5;\n\tadd.u64 l2, %3, %5;\n\tadd.u64 l3, %4, %5;\n\t"
        "add.u64 b1, %6, %7;\n\tadd.u64 b2, b1, %7;\n\tadd.u64 b3, b2, %7;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p1, 1, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %6, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], l0, %6, %9, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, b1, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], l1, b1, %9, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %3, b2, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], l2, b2, %9, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %4, b3, %8, p1;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], l3, b3, %9, p1;\n\t}" ::"r"(d_tmem),
        "l"(a0), "l"(a1), "l"(a2), "l"(a3), "l"(lo_off), "l"(b0), "l"(bstep), "r"(i_hi), "r"(i_lo)
        : "memory");
}

// Four consecutive 32-bit columns of this thread's TMEM lane (warp-collective;
// warp w writes lanes 32 (w % 4) .. 32 (w % 4) + 31, encoded in taddr).
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r0), "r"(r1),
                 "r"(r2), "r"(r3)
                 : "memory");
}
// Sixteen consecutive 32-bit columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
// Wait until this thread's tcgen05.st writes are complete.
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Arrive on an mbarrier once every tcgen05.mma issued so far by this thread completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM allocation (one warp, all lanes): the column base is written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31; the lane offset is encoded in taddr).  The
// wait is part of the same asm statement, so that no use of the registers
// can be scheduled before it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Two sets of 32 consecutive FP32 columns of this thread's TMEM lane (at taddr0
// and taddr1), both loads in flight before the one wait; a single asm statement
// so that no use of the registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t taddr0, uint32_t taddr1, float* v, float* w) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr0), "r"(taddr1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        v[i] = __uint_as_float(r[i]);
        w[i] = __uint_as_float(r[32 + i]);
    }
}

// ---- mbarrier / TMA ---------------------------------------------------------
// Residuals of a hi/lo split: (a - hi0, b - hi1) for the packed 16-bit pair
// hb = (hi0, hi1) (FP16 for FMT 0, BF16 for FMT 1), each from one
// mixed-precision fma hi * (-1) + a with the 16-bit operand taken as is (no
// conversion of hi back to FP32); exact when hi is a or a's rounding.
template <int FMT>
__device__ __forceinline__ void split_resid(uint32_t hb, float a, float b, float& ra, float& rb) {
    if (FMT == 0)
        asm("{\n\t.reg .b16 h0, h1;\n\tmov.b32 {h0, h1}, %2;\n\t"
            "fma.rn.f32.f16 %0, h0, %4, %3;\n\tfma.rn.f32.f16 %1, h1, %4, %5;\n\t}"
            : "=f"(ra), "=f"(rb)
            : "r"(hb), "f"(a), "h"((unsigned short)0xBC00u), "f"(b));
    else
        asm("{\n\t.reg .b16 h0, h1;\n\tmov.b32 {h0, h1}, %2;\n\t"
            "fma.rn.f32.bf16 %0, h0, %4, %3;\n\tfma.rn.f32.bf16 %1, h1, %4, %5;\n\t}"
            : "=f"(ra), "=f"(rb)
            : "r"(hb), "f"(a), "h"((unsigned short)0xBF80u), "f"(b));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false (and bit 0 of *err set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns, unsigned int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) {
            if (err) atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Packed FP32 pairs (f32x2: two lanes per 64-bit register, element 0 in the
// low half).  The kernel rows are computed two training points at a time, so
// one packed instruction does the work of two scalar ones.
__device__ __forceinline__ uint64_t f2pack(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(uint64_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

}  // namespace tc
}  // namespace gpm
