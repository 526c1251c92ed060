// Throughput probes of the two arithmetic units the CUDA-core rollouts are
// bound by: the FP32 FMA pipe (scalar fma.rn.f32 and packed fma.rn.f32x2)
// and the SFU's ex2.approx.  They are measurement tools for the roofline
// denominators, not part of the method: each thread runs 16 independent
// dependency chains of one instruction kind for `iters` iterations and
// writes one value (so that nothing is optimised away).  The caller times the
// launch with events on `stream`; the operation count is
// blocks * 256 * iters * 16 (FMAs for kinds 0 and 1, exponentials for kind 2).
#include "common.cuh"

namespace gpm {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 16;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(float* out, int iters, float a, float b) {
    float x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j];
    out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma2(float* out, int iters, float a, float b) {
    uint64_t x[CHAINS / 2];
    uint64_t av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int j = 0; j < CHAINS / 2; ++j) {
        const float v = (float)(threadIdx.x + j) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[j]) : "f"(v), "f"(v + 0.5f));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS / 2; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(av), "l"(bv));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < CHAINS / 2; ++j) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[j]));
        s += lo + hi;
    }
    out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ex2(float* out, int iters) {
    float x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) {
            // x <- 2^-x stays bounded (it converges to the root of x = 2^-x)
            const float nx = -x[j];
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[j]) : "f"(nx));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j];
    out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

}  // namespace
}  // namespace gpm

using namespace gpm;

extern "C" int gpmppi_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float* out, void* stream) {
    if (kind < 0 || kind > 2) return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_alu_probe: kind must be 0, 1 or 2");
    if (blocks < 1 || blocks > (1 << 20) || iters < 1)
        return fail(GPMPPI_ERR_INVALID_ARG, "gpmppi_alu_probe: blocks in [1, 2^20] and iters >= 1");
    int rc;
    if ((rc = check_dev_ptr(out, "gpmppi_alu_probe: out", false))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (kind == 0)
        k_probe_fma<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, 0.999f, 1e-4f);
    else if (kind == 1)
        k_probe_fma2<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, 0.999f, 1e-4f);
    else
        k_probe_ex2<<<blocks, PROBE_THREADS, 0, st>>>(out, iters);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}
