// MPPI weights and control update, Alg. 1 Step 2 (nominal tightening) and
// the raw-noise entry points.
//
// Update (Alg. 1, "weights" and "weighted sum"): every CTA reduces the K
// costs to rho = min S and Z = sum_s exp(-(S_s - rho)/lambda) in one fixed
// order (so all CTAs agree bit for bit), writes w_s for its own samples, and
// reduces sum_s w_s (u~_s,k - U_k) over them for every step k (one warp per
// step, coalesced reads of u~, warp shuffles).  The per-CTA partials go to a scratch array; the CTA that
// finishes last (atomic ticket) sums them in CTA order and writes U_new.
#include <cfloat>

#include "common.cuh"

namespace gpm {
namespace {

constexpr int UPD_THREADS = 256;
constexpr int UPD_WARPS = UPD_THREADS / 32;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// loads of the K costs in groups of eight per thread, all in flight together
template <typename F>
__device__ __forceinline__ void for_costs(const float* __restrict__ costs, int K, F&& f) {
    const int tid = threadIdx.x;
    for (int s0 = tid; s0 < K; s0 += 8 * UPD_THREADS) {
        float c[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int s = s0 + j * UPD_THREADS;
            c[j] = s < K ? __ldg(costs + s) : FLT_MAX;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (s0 + j * UPD_THREADS < K) f(c[j]);
    }
}

__device__ __forceinline__ void update_body(const UpdateArgs& a, int cta, int n_cta,
                                            unsigned long long* it_dev) {
    __shared__ float red[UPD_WARPS];
    __shared__ float bcast[2];
    __shared__ float wsh[UPD_THREADS];
    __shared__ unsigned int is_last;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = a.K, T = a.T;
    // rho = min_s S_s
    float mn = FLT_MAX;
    for_costs(a.costs, K, [&](float c) { mn = fminf(mn, c); });
    mn = warp_min(mn);
    if (lane == 0) red[warp] = mn;
    __syncthreads();
    if (tid == 0) {
        float r = red[0];
        for (int w = 1; w < UPD_WARPS; ++w) r = fminf(r, red[w]);
        bcast[0] = r;
    }
    __syncthreads();
    const float rho = bcast[0];
    // Z = sum_s exp(-(S_s - rho)/lambda), fixed summation order
    float z = 0.0f;
    for_costs(a.costs, K, [&](float c) { z += expf((rho - c) * a.inv_lambda); });
    z = warp_sum(z);
    if (lane == 0) red[warp] = z;
    __syncthreads();
    if (tid == 0) {
        float r = 0.0f;
        for (int w = 0; w < UPD_WARPS; ++w) r += red[w];
        bcast[1] = r;
    }
    __syncthreads();
    const float inv_z = 1.0f / bcast[1];
    // own samples' weights
    const int s_base = cta * a.per_cta;
    const int s = s_base + tid;
    const bool act = (tid < a.per_cta) && (s < K);
    const float w = act ? expf((rho - __ldg(a.costs + s)) * a.inv_lambda) * inv_z : 0.0f;
    if (act && a.weights) a.weights[s] = w;
    wsh[tid] = w;
    __syncthreads();
    // sum_s w_s (u~_s,k - U_k) over the CTA's samples: warp w takes the steps
    // k = w, w + 8, ..., lane l the samples l, l + 32, ... (coalesced reads of
    // u~, all of a lane's loads in flight together)
    const int ns = min(a.per_cta, K - s_base);
    for (int k = warp; k < T; k += UPD_WARPS) {
        const float uv = __ldg(a.U + 2 * k), uw = __ldg(a.U + 2 * k + 1);
        const float2* ut = a.u_tilde + (size_t)k * K + s_base;
        float dv = 0.0f, dw = 0.0f;
#pragma unroll 8
        for (int i = lane; i < ns; i += 32) {
            const float2 u = __ldg(ut + i);
            dv = fmaf(wsh[i], u.x - uv, dv);
            dw = fmaf(wsh[i], u.y - uw, dw);
        }
        dv = warp_sum(dv);
        dw = warp_sum(dw);
        if (lane == 0) {
            a.partial[((size_t)cta * T + k) * 2] = dv;
            a.partial[((size_t)cta * T + k) * 2 + 1] = dw;
        }
    }
    // last CTA combines the partials in CTA order
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(a.counter, 1u) == (unsigned int)n_cta - 1u) ? 1u : 0u;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int i = tid; i < 2 * T; i += UPD_THREADS) {
        float acc = 0.0f;
        for (int c = 0; c < n_cta; ++c) acc += __ldcg(a.partial + (size_t)c * 2 * T + i);
        a.U_new[i] = __ldg(a.U + i) + acc;
    }
    if (tid == 0) {
        *a.counter = 0u;
        if (it_dev) *it_dev += 1ull;     // the next iteration's Philox counter
    }
}

__global__ void __launch_bounds__(UPD_THREADS) k_update(const UpdateArgs a) {
    update_body(a, blockIdx.x, gridDim.x, nullptr);
}

// Many controllers: CTA i serves CTA items[i].y of controller items[i].x,
// whose update needs ncta[items[i].x] CTAs; the last one advances its
// iteration counter.
__global__ void __launch_bounds__(UPD_THREADS)
    k_update_batched(const UpdateArgs* __restrict__ args, const int2* __restrict__ items,
                     const int* __restrict__ ncta, unsigned long long* __restrict__ iters) {
    const int2 it = items[blockIdx.x];
    update_body(args[it.x], it.y, ncta[it.x], iters + it.x);
}

__global__ void k_philox(uint32_t key0, uint32_t key1, const uint4* __restrict__ ctr, int M,
                         uint4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) out[i] = philox4x32_10(ctr[i], key0, key1);
}

__global__ void k_noise(uint32_t key0, uint32_t key1, uint32_t it0, uint32_t it1, int K, int T,
                        float sv, float sw, float2* __restrict__ eps) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)K * T) return;
    const int s = (int)(i / T), k = (int)(i % T);
    eps[i] = control_eps((uint32_t)k, (uint32_t)s, it0, it1, key0, key1, sv, sw);
}

// ---------------------------------------------------------------------------
// Alg. 1 Step 2: mean and covariance along the updated controls (no noise),
// one CTA; records Sigma_XY(k+1) for the next iteration's tightening.
// ---------------------------------------------------------------------------
constexpr int NOM_THREADS = 256;

__device__ float nom_block_sum(float v, float* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float s = 0.0f;
    for (int i = 0; i < NOM_THREADS / 32; ++i) s += red[i];
    return s;
}

__global__ void __launch_bounds__(NOM_THREADS) k_nominal(const RolloutArgs a, const float* __restrict__ Uc,
                                                         float* __restrict__ sxy_out) {
    extern __shared__ __align__(16) float ks[];   // N floats
    __shared__ float red[NOM_THREADS / 32];
    __shared__ float4 zsh;
    float mu[5] = {a.x0[0], a.x0[1], a.x0[2], a.x0[3], a.x0[4]};
    float S[5][5] = {};
    const int tid = threadIdx.x;
    for (int k = 0; k < a.T; ++k) {
        const float ux = fminf(fmaxf(Uc[2 * k], a.umin0), a.umax0);
        const float uy = fminf(fmaxf(Uc[2 * k + 1], a.umin1), a.umax1);
        if (tid == 0)
            zsh = make_float4(mu[3] * a.zscale[0], mu[4] * a.zscale[1], ux * a.zscale[2],
                              uy * a.zscale[3]);
        __syncthreads();
        const float4 z = zsh;
        float mv = 0.0f, mw = 0.0f;
        for (int j = tid; j < a.N; j += NOM_THREADS) {
            const float4 x = reinterpret_cast<const float4*>(a.Xs)[j];
            const float e0 = z.x - x.x, e1 = z.y - x.y, e2 = z.z - x.z, e3 = z.w - x.w;
            const float kv = a.sf2 * exp2f(-(e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3));
            ks[j] = kv;
            mv = fmaf(kv, a.alpha[2 * j], mv);
            mw = fmaf(kv, a.alpha[2 * j + 1], mw);
        }
        mv = nom_block_sum(mv, red);
        mw = nom_block_sum(mw, red);
        float q = 0.0f;
        for (int i = tid; i < a.N; i += NOM_THREADS) {
            float v = 0.0f;
            for (int j = 0; j <= i; ++j) v = fmaf(a.W[(size_t)j * a.Np + i], ks[j], v);
            q = fmaf(v, v, q);
        }
        q = nom_block_sum(q, red);
        const float s = fmaxf(0.0f, a.sf2 - q);
        // every thread carries the (identical) single-trajectory state
        float sn, cs;
        sincosf(mu[2], &sn, &cs);
        float A[5][5] = {};
        for (int i = 0; i < 5; ++i) A[i][i] = 1.0f;
        A[0][2] = -a.dt * mu[3] * sn;
        A[0][3] = a.dt * cs;
        A[1][2] = a.dt * mu[3] * cs;
        A[1][3] = a.dt * sn;
        A[2][4] = a.dt;
        A[3][3] = a.av;
        A[4][4] = a.aw;
        float B[5][5];
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                float acc = 0.0f;
                for (int l = 0; l < 5; ++l) acc = fmaf(A[i][l], S[l][j], acc);
                B[i][j] = acc;
            }
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                float acc = 0.0f;
                for (int l = 0; l < 5; ++l) acc = fmaf(B[i][l], A[j][l], acc);
                S[i][j] = acc;
            }
        S[3][3] += s;
        S[4][4] += s;
        const float nX = mu[0] + a.dt * mu[3] * cs, nY = mu[1] + a.dt * mu[3] * sn;
        const float nT = mu[2] + a.dt * mu[4];
        const float nV = mu[3] + a.kv * (ux - mu[3]) + mv;
        const float nW = mu[4] + a.kw * (uy - mu[4]) + mw;
        mu[0] = nX; mu[1] = nY; mu[2] = nT; mu[3] = nV; mu[4] = nW;
        if (tid == 0) {
            sxy_out[3 * k] = S[0][0];
            sxy_out[3 * k + 1] = S[0][1];
            sxy_out[3 * k + 2] = S[1][1];
        }
        __syncthreads();
    }
}

}  // namespace

int launch_update(const UpdateArgs& a, int n_cta, cudaStream_t st) {
    k_update<<<n_cta, UPD_THREADS, 0, st>>>(a);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

int launch_update_batched(const UpdateArgs* args, const int2* items, const int* ncta,
                          unsigned long long* iters, int nitems, int maxT, cudaStream_t st) {
    if (nitems == 0) return GPMPPI_OK;
    (void)maxT;
    k_update_batched<<<nitems, UPD_THREADS, 0, st>>>(args, items, ncta, iters);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

int launch_philox(uint64_t seed, const uint32_t* ctr, int M, uint32_t* out, cudaStream_t st) {
    if (M == 0) return GPMPPI_OK;
    k_philox<<<(M + 255) / 256, 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32),
                                              reinterpret_cast<const uint4*>(ctr), M,
                                              reinterpret_cast<uint4*>(out));
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

int launch_noise(uint64_t seed, int K, int T, uint64_t it, float sv, float sw, float* eps,
                 cudaStream_t st) {
    const size_t n = (size_t)K * T;
    if (n == 0) return GPMPPI_OK;
    k_noise<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32),
                                                         (uint32_t)it, (uint32_t)(it >> 32), K, T,
                                                         sv, sw, reinterpret_cast<float2*>(eps));
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

int launch_nominal(const RolloutArgs& a, float* sxy_out, cudaStream_t st) {
    const int smem = (a.N > 0 ? a.N : 1) * (int)sizeof(float);
    GPM_CUDA(cudaFuncSetAttribute(k_nominal, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // a.U holds the updated controls for this launch
    k_nominal<<<1, NOM_THREADS, smem, st>>>(a, a.U, sxy_out);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

}  // namespace gpm
