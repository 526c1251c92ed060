// MPPI weights and control update, Alg. 1 Step 2 (nominal tightening) and
// the raw-noise entry points.
//
// Update (Alg. 1, "weights" and "weighted sum"): CTA (b, j) of the grid
// takes sample block b (256 samples) and step block j (16 steps).  It
// reduces its own samples to the log-sum-exp tuple (rho_b = min S,
// Z_b = sum exp(-(S - rho_b)/lambda), V_b = sum exp(-(S - rho_b)/lambda)
// (u~ - U) for its steps; two steps per warp, all loads of a lane in flight
// together, coalesced reads of u~, warp shuffles).  The tuples go to a
// scratch array; the CTA that finishes last (atomic ticket) rescales them to
// the global minimum and combines them in sample-block order into U_new and
// the weights.
#include <cfloat>

#include "common.cuh"

namespace gpm {
namespace {

constexpr int UPD_THREADS = 256;
constexpr int UPD_WARPS = UPD_THREADS / 32;
constexpr int UPD_SPW = 2;                          // steps per warp
constexpr int UPD_STEPS = UPD_WARPS * UPD_SPW;      // steps per CTA

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

__device__ __forceinline__ float block_reduce(float v, float* red, bool is_min) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = is_min ? warp_min(v) : warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float r = red[0];
    for (int w = 1; w < UPD_WARPS; ++w) r = is_min ? fminf(r, red[w]) : r + red[w];
    return r;
}

// cta: sample block; [k_lo, k_hi): the CTA's steps; n_sb sample blocks and
// n_total CTAs in all (the ticket counts every CTA).
//
// Each CTA reduces only its own samples: rho_b = min S over the block,
// e_s = exp(-(S_s - rho_b)/lambda), Z_b = sum e_s and, for its steps,
// V_b,k = sum_s e_s (u~_s,k - U_k).  (rho_b, Z_b, V_b) is the associative
// log-sum-exp tuple: with rho = min_b rho_b and c_b = exp(-(rho_b - rho)/lambda),
// Z = sum_b c_b Z_b and U_new = U + sum_b c_b V_b / Z.  The last CTA forms
// that combination in sample-block order and writes the weights
// w_s = exp(-(S_s - rho)/lambda) / Z.  No CTA reads all K costs but the last.
//
// Scratch layout (a.partial): V at [(b T + k) 2 + {0,1}], then the block
// statistics (rho_b, Z_b) at [n_sb T 2 + 2 b + {0,1}].
__device__ __forceinline__ void update_body(const UpdateArgs& a, int cta, int n_sb, int k_lo, int k_hi,
                                            int n_total, unsigned long long* it_dev) {
    // launched as a programmatic dependent of the rollout (its launch overlaps
    // the rollout's tail): wait until the rollout grid has completed and its
    // costs and u~ are visible (a no-op for an ordinary launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __shared__ float red[UPD_WARPS];
    __shared__ float wsh[UPD_THREADS];
    __shared__ unsigned int is_last;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = a.K, T = a.T;
    const int s_base = cta * a.per_cta;
    const int s = s_base + tid;
    const bool act = (tid < a.per_cta) && (s < K);
    const float cs = act ? __ldg(a.costs + s) : FLT_MAX;
    const float rho_b = block_reduce(cs, red, true);
    const float e = act ? expf((rho_b - cs) * a.inv_lambda) : 0.0f;
    const float z_b = block_reduce(e, red, false);
    float* stats = a.partial + (size_t)n_sb * T * 2;
    if (k_lo == 0 && tid == 0) {
        stats[2 * cta] = rho_b;
        stats[2 * cta + 1] = z_b;
    }
    wsh[tid] = e;
    __syncthreads();
    // sum_s e_s (u~_s,k - U_k) over the CTA's samples: warp w takes steps
    // k_lo + 2 w and k_lo + 2 w + 1 (then + 16 ...), lane l the samples l,
    // l + 32, ... (coalesced reads of u~, all of a lane's loads in flight)
    const int ns = min(a.per_cta, K - s_base);
    for (int k0 = k_lo + warp * UPD_SPW; k0 < k_hi; k0 += UPD_STEPS) {
        float2 uu[UPD_SPW][8];
        float uv[UPD_SPW], uw[UPD_SPW];
#pragma unroll
        for (int j = 0; j < UPD_SPW; ++j) {
            const int k = k0 + j;
            const bool kin = k < k_hi;
            uv[j] = kin ? __ldg(a.U + 2 * k) : 0.0f;
            uw[j] = kin ? __ldg(a.U + 2 * k + 1) : 0.0f;
            const float2* ut = a.u_tilde + (size_t)(kin ? k : k_lo) * K + s_base;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = lane + 32 * q;
                uu[j][q] = (kin && i < ns) ? __ldg(ut + i) : make_float2(0.0f, 0.0f);
            }
        }
#pragma unroll
        for (int j = 0; j < UPD_SPW; ++j) {
            float dv = 0.0f, dw = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = lane + 32 * q;
                if (i < ns) {
                    dv = fmaf(wsh[i], uu[j][q].x - uv[j], dv);
                    dw = fmaf(wsh[i], uu[j][q].y - uw[j], dw);
                }
            }
            dv = warp_sum(dv);
            dw = warp_sum(dw);
            const int k = k0 + j;
            if (lane == 0 && k < k_hi) {
                a.partial[((size_t)cta * T + k) * 2] = dv;
                a.partial[((size_t)cta * T + k) * 2 + 1] = dw;
            }
        }
    }
    // the last CTA combines the blocks' tuples in sample-block order
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(a.counter, 1u) == (unsigned int)n_total - 1u) ? 1u : 0u;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    float mn = FLT_MAX;
    for (int b = tid; b < n_sb; b += UPD_THREADS) mn = fminf(mn, __ldcg(stats + 2 * b));
    const float rho = block_reduce(mn, red, true);
    // c_b replaces rho_b in the scratch; Z = sum_b c_b Z_b
    float zp = 0.0f;
    for (int b = tid; b < n_sb; b += UPD_THREADS) {
        const float cb = expf((rho - __ldcg(stats + 2 * b)) * a.inv_lambda);
        zp = fmaf(cb, __ldcg(stats + 2 * b + 1), zp);
        __stcg(stats + 2 * b, cb);
    }
    const float inv_z = 1.0f / block_reduce(zp, red, false);   // its barriers publish the c_b
    for (int i = tid; i < 2 * T; i += UPD_THREADS) {
        // sample-block order; sixteen loads in flight at a time
        float acc = 0.0f;
        for (int c0 = 0; c0 < n_sb; c0 += 16) {
            float p[16], cb[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const bool in = c0 + j < n_sb;
                p[j] = in ? __ldcg(a.partial + (size_t)(c0 + j) * 2 * T + i) : 0.0f;
                cb[j] = in ? __ldcg(stats + 2 * (c0 + j)) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (c0 + j < n_sb) acc = fmaf(cb[j], p[j], acc);
        }
        a.U_new[i] = fmaf(acc, inv_z, __ldg(a.U + i));
    }
    if (a.weights) {
        // w_s = exp(-(S_s - rho)/lambda) / Z, eight loads in flight per thread
        for (int s0 = tid; s0 < K; s0 += 8 * UPD_THREADS) {
            float c[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int q = s0 + j * UPD_THREADS;
                c[j] = q < K ? __ldg(a.costs + q) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int q = s0 + j * UPD_THREADS;
                if (q < K) a.weights[q] = expf((rho - c[j]) * a.inv_lambda) * inv_z;
            }
        }
    }
    if (tid == 0) {
        *a.counter = 0u;
        if (it_dev) *it_dev += 1ull;     // the next iteration's Philox counter
    }
}

// gridDim.y step blocks of UPD_STEPS steps (one block of all T steps when
// gridDim.y == 1)
__global__ void __launch_bounds__(UPD_THREADS) k_update(const UpdateArgs a) {
    const int tb = gridDim.y == 1 ? a.T : UPD_STEPS;
    const int k_lo = blockIdx.y * tb;
    update_body(a, blockIdx.x, gridDim.x, k_lo, min(a.T, k_lo + tb), gridDim.x * gridDim.y, nullptr);
}

// Many controllers: CTA i serves CTA items[i].y of controller items[i].x,
// whose update needs ncta[items[i].x] CTAs; the last one advances its
// iteration counter.
__global__ void __launch_bounds__(UPD_THREADS)
    k_update_batched(const UpdateArgs* __restrict__ args, const int2* __restrict__ items,
                     const int* __restrict__ ncta, unsigned long long* __restrict__ iters) {
    const int2 it = items[blockIdx.x];
    update_body(args[it.x], it.y, ncta[it.x], 0, args[it.x].T, ncta[it.x], iters + it.x);
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

int launch_update(const UpdateArgs& a, int n_cta, cudaStream_t st, bool after_rollout) {
    // sample blocks x step blocks of UPD_STEPS steps (a CTA reads only its own
    // samples' costs, so the step blocks add no reduction work)
    const int nstep = a.T > 0 ? (a.T + UPD_STEPS - 1) / UPD_STEPS : 1;
    // after_rollout: programmatic stream serialisation, so that the launch may
    // begin while the previous kernel on the stream (the rollout) finishes;
    // the kernel's griddepcontrol.wait holds every CTA until that kernel has
    // completed.  Otherwise (say a memset precedes it) an ordinary launch.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_cta, (unsigned)nstep);
    cfg.blockDim = dim3(UPD_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_rollout ? 1 : 0;
    GPM_CUDA(cudaLaunchKernelEx(&cfg, k_update, a));
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
