// Self-test of the tcgen05 building blocks (tc05.cuh): one CTA multiplies a
// 128 x K tile by an N x K tile (both K-major, 16-bit) on the tensor cores
// with the slab-major shared-memory layout, the matrix and instruction
// descriptors, TMEM allocation, tcgen05.commit on an mbarrier and tcgen05.ld,
// and writes D = A B^T (128 x N, FP32).  The rollout's variance contraction
// uses exactly these pieces, so this call lets a test pin them in isolation.
// Variant 2 writes A into tensor memory instead (tcgen05.st, one row per
// lane) and issues the products with A read from there.
#include "common.cuh"
#include "tc05.cuh"

namespace gpm {
namespace {

constexpr int ST_THREADS = 128;
constexpr int ST_REGION = 32 * 1024;   // bytes reserved per operand

__global__ void __launch_bounds__(ST_THREADS, 1)
    k_mma_selftest(int fmt, int N, int K, int variant, const uint16_t* __restrict__ A,
                   const uint16_t* __restrict__ B, float* __restrict__ D, unsigned int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sA = sm;
    unsigned char* sB = sm + ST_REGION;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * ST_REGION);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * ST_REGION + 64);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int slabs = K / 8;
    // operands to shared memory, slab-major: slab s, row r at s * (rows * 16) + r * 16
    for (int i = tid; i < 128 * slabs; i += ST_THREADS) {
        const int r = i % 128, s = i / 128;
        *reinterpret_cast<uint4*>(sA + s * 128 * 16 + r * 16) =
            *reinterpret_cast<const uint4*>(A + (size_t)r * K + 8 * s);
    }
    for (int i = tid; i < N * slabs; i += ST_THREADS) {
        const int r = i % N, s = i / N;
        *reinterpret_cast<uint4*>(sB + s * N * 16 + r * 16) =
            *reinterpret_cast<const uint4*>(B + (size_t)r * K + 8 * s);
    }
    tc::fence_proxy_async();            // generic-proxy writes visible to the tensor core
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    constexpr uint32_t ACOL = 256;      // A in TMEM (variant 2): columns 256 .. 256 + K/2
    if (variant == 2) {
        // thread tid = row r of A (lane r); K/2 packed columns in steps of 4
        const uint32_t lane_addr = taddr + ((uint32_t)(32 * warp) << 16) + ACOL;
        const uint32_t* row = reinterpret_cast<const uint32_t*>(A + (size_t)tid * K);
        for (int c = 0; c < K / 2; c += 4)
            tc::tmem_st4(lane_addr + (uint32_t)c, row[c], row[c + 1], row[c + 2], row[c + 3]);
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16(fmt, 128, N);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint32_t a0 = tc::smem_addr(sA) + ks * 2 * 128 * 16;
            const uint32_t b0 = tc::smem_addr(sB) + ks * 2 * N * 16;
            uint64_t ad, bd;
            if (variant == 0 || variant == 2) {
                ad = tc::smem_desc(a0, 128 * 16, 128);
                bd = tc::smem_desc(b0, N * 16, 128);
            } else {
                ad = tc::smem_desc(a0, 128, 128 * 16);
                bd = tc::smem_desc(b0, 128, N * 16);
            }
            if (variant == 2)
                tc::mma_f16_ta(taddr, taddr + ACOL + 8u * ks, bd, idesc, ks > 0 ? 1u : 0u);
            else
                tc::mma_f16(taddr, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar);
    }
    tc::mbar_wait(bar, 0, 1000000000ull, err);
    tc::fence_after_sync();
    const uint32_t row_addr = taddr + ((uint32_t)(32 * warp) << 16);
    for (int c = 0; c < N / 32; ++c) {
        float v[32];
        tc::tmem_ld32(row_addr + 32 * c, v);
        for (int i = 0; i < 32; ++i) D[(size_t)(32 * warp + lane) * N + 32 * c + i] = v[i];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

}  // namespace

int launch_mma_selftest(int fmt, int N, int K, int variant, const uint16_t* A, const uint16_t* B,
                        float* D, unsigned int* err, cudaStream_t st) {
    // operands and barrier use the first 64 KiB; the rest is reserved so that
    // every address a descriptor can form from these offsets stays inside the
    // CTA's own shared memory
    const int smem = 200 * 1024;
    GPM_CUDA(cudaFuncSetAttribute(k_mma_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_mma_selftest<<<1, ST_THREADS, smem, st>>>(fmt, N, K, variant, A, B, D, err);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

}  // namespace gpm
