// GP fit in FP64 on the GPU and the FP32 GP posterior.
//
// Sec. III-A fits two GPs (delta_v, delta_omega) on 4-D inputs; the rollout
// needs, per output, alpha = K^-1 y and L^-1 with L = chol(K_XX + sn2 I)
// (Rasmussen & Williams, Alg. 2.1).  The factorisation runs once per fit in
// FP64 as a right-looking blocked Cholesky (32 x 32 blocks: diagonal factor,
// panel solve, trailing update), followed by a column-block triangular
// inverse and two matrix-vector products for alpha.  Results are then
// converted to the FP32 layouts the rollout reads.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include <cstring>

#include "common.cuh"

namespace gpm {
namespace {

constexpr int NB = 32;

__global__ void k_build_kxx(const double* __restrict__ X, int N, double il0, double il1,
                            double il2, double il3, double sf2, double sn2, double* __restrict__ A) {
    const int i = blockIdx.y * 16 + threadIdx.y;
    const int j = blockIdx.x * 16 + threadIdx.x;
    if (i >= N || j >= N) return;
    const double d0 = (X[i * 4 + 0] - X[j * 4 + 0]) * il0;
    const double d1 = (X[i * 4 + 1] - X[j * 4 + 1]) * il1;
    const double d2 = (X[i * 4 + 2] - X[j * 4 + 2]) * il2;
    const double d3 = (X[i * 4 + 3] - X[j * 4 + 3]) * il3;
    double v = sf2 * exp(-0.5 * (d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3));
    if (i == j) v += sn2;
    A[(size_t)i * N + j] = v;
}

// Unblocked Cholesky of the diagonal block at (kb, kb), size n <= 32.
__global__ void k_potrf_diag(double* __restrict__ A, int N, int kb, int n, int* __restrict__ flag) {
    __shared__ double a[NB][NB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (ty < n && tx < n) a[ty][tx] = A[(size_t)(kb + ty) * N + kb + tx];
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        if (tx == 0 && ty == 0) {
            const double d = a[c][c];
            if (!(d > 0.0)) {
                atomicExch(flag, 1);
                a[c][c] = 1.0;   // keep going with finite values; the host reports NOT_PD
            } else {
                a[c][c] = sqrt(d);
            }
        }
        __syncthreads();
        if (tx == 0 && ty > c && ty < n) a[ty][c] /= a[c][c];
        __syncthreads();
        if (ty > c && ty < n && tx > c && tx <= ty) a[ty][tx] -= a[ty][c] * a[tx][c];
        __syncthreads();
    }
    if (ty < n && tx <= ty) A[(size_t)(kb + ty) * N + kb + tx] = a[ty][tx];
}

// Panel solve: rows below the diagonal block, X L_kk^T = B.
__global__ void k_trsm_panel(double* __restrict__ A, int N, int kb, int n) {
    __shared__ double l[NB][NB + 1];
    __shared__ double b[NB][NB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int r0 = kb + n + blockIdx.x * NB;
    const int rows = min(NB, N - r0);
    if (ty < n && tx < n) l[ty][tx] = A[(size_t)(kb + ty) * N + kb + tx];
    if (ty < rows && tx < n) b[ty][tx] = A[(size_t)(r0 + ty) * N + kb + tx];
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        if (tx == c && ty < rows) {
            double s = b[ty][c];
            for (int q = 0; q < c; ++q) s -= b[ty][q] * l[c][q];
            b[ty][c] = s / l[c][c];
        }
        __syncthreads();
    }
    if (ty < rows && tx < n) A[(size_t)(r0 + ty) * N + kb + tx] = b[ty][tx];
}

// Trailing update A[ib][jb] -= P[ib] P[jb]^T for trailing blocks jb <= ib.
__global__ void k_syrk(double* __restrict__ A, int N, int kb, int n) {
    const int ib = blockIdx.y, jb = blockIdx.x;
    if (jb > ib) return;
    __shared__ double pi[NB][NB + 1];
    __shared__ double pj[NB][NB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int t0 = kb + n;
    const int ri = t0 + ib * NB + ty, rj = t0 + jb * NB + ty;
    pi[ty][tx] = (ri < N && tx < n) ? A[(size_t)ri * N + kb + tx] : 0.0;
    pj[ty][tx] = (rj < N && tx < n) ? A[(size_t)rj * N + kb + tx] : 0.0;
    __syncthreads();
    const int row = t0 + ib * NB + ty, col = t0 + jb * NB + tx;
    if (row >= N || col >= N || col > row) return;
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < NB; ++q) s += pi[ty][q] * pj[tx][q];
    A[(size_t)row * N + col] -= s;
}

// L entry with an identity extension beyond N (used by the inverse).
__device__ __forceinline__ double lval(const double* L, int N, int r, int c) {
    if (r < N && c < N) return c <= r ? L[(size_t)r * N + c] : 0.0;
    return r == c ? 1.0 : 0.0;
}

// X = L^-1, one CTA per 32-column block cb: blocked forward substitution
// X[ib][cb] = L[ib][ib]^-1 (I[ib][cb] - sum_{cb<=jb<ib} L[ib][jb] X[jb][cb]).
__global__ void k_trtri(const double* __restrict__ L, int N, double* __restrict__ Xo) {
    __shared__ double lb[NB][NB + 1];
    __shared__ double xb[NB][NB + 1];
    __shared__ double r[NB][NB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cb = blockIdx.x;
    const int nblk = (N + NB - 1) / NB;
    const int col = cb * NB + tx;
    for (int ib = cb; ib < nblk; ++ib) {
        double acc = (ib == cb && ty == tx) ? 1.0 : 0.0;
        for (int jb = cb; jb < ib; ++jb) {
            __syncthreads();
            lb[ty][tx] = lval(L, N, ib * NB + ty, jb * NB + tx);
            const int xr = jb * NB + ty;
            xb[ty][tx] = (xr < N && col < N) ? Xo[(size_t)xr * N + col] : 0.0;
            __syncthreads();
#pragma unroll 8
            for (int q = 0; q < NB; ++q) acc -= lb[ty][q] * xb[q][tx];
        }
        __syncthreads();
        lb[ty][tx] = lval(L, N, ib * NB + ty, ib * NB + tx);
        r[ty][tx] = acc;
        __syncthreads();
        // forward substitution down the rows, one thread per column
        if (ty == 0) {
            for (int rr = 0; rr < NB; ++rr) {
                double s = r[rr][tx];
                for (int q = 0; q < rr; ++q) s -= lb[rr][q] * r[q][tx];
                r[rr][tx] = s / lb[rr][rr];
            }
        }
        __syncthreads();
        const int row = ib * NB + ty;
        if (row < N && col < N) Xo[(size_t)row * N + col] = r[ty][tx];
    }
}

// t = X y   (one thread per row)
__global__ void k_matvec(const double* __restrict__ Xm, const double* __restrict__ y, int N,
                         int ystride, double* __restrict__ t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s += Xm[(size_t)i * N + j] * y[(size_t)j * ystride];
    t[i] = s;
}

// a = X^T t   (one thread per column)
__global__ void k_matvec_t(const double* __restrict__ Xm, const double* __restrict__ t, int N,
                           double* __restrict__ a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s = 0.0;
    for (int i = j; i < N; ++i) s += Xm[(size_t)i * N + j] * t[i];
    a[j] = s;
}

// FP32 layouts for the rollout.
__global__ void k_pack_w(const double* __restrict__ Xm, int N, int Np, float* __restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // column of W (row of L^-1)
    const int j = blockIdx.y;                              // row of W
    if (i >= Np) return;
    float v = 0.0f;
    if (i < N && j < N && i >= j) v = (float)Xm[(size_t)i * N + j];
    W[(size_t)j * Np + i] = v;
}

__global__ void k_pack_x(const double* __restrict__ X, int N, double s0, double s1, double s2,
                         double s3, float* __restrict__ Xs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    Xs[j * 4 + 0] = (float)(X[j * 4 + 0] * s0);
    Xs[j * 4 + 1] = (float)(X[j * 4 + 1] * s1);
    Xs[j * 4 + 2] = (float)(X[j * 4 + 2] * s2);
    Xs[j * 4 + 3] = (float)(X[j * 4 + 3] * s3);
}

__global__ void k_pack_alpha(const double* __restrict__ a0, const double* __restrict__ a1, int N,
                             float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    out[j * 2 + 0] = (float)a0[j];
    out[j * 2 + 1] = (float)a1[j];
}

// ---------------------------------------------------------------------------
// GP posterior at M queries, one CTA per query (FP32).
// ---------------------------------------------------------------------------
constexpr int PRED_THREADS = 128;

__device__ float block_sum(float v, float* red) {
    // deterministic: fixed shuffle tree, then warp partials summed in order
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float s = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

struct PredArgs {
    const float* Xs[2];
    const float* W[2];
    const float* alpha;
    float sf2[2];
    float zscale[2][4];
    int N, Np;
    bool shared;
};

__global__ void k_gp_predict(PredArgs p, const float* __restrict__ Z, int M, float* __restrict__ mean,
                             float* __restrict__ var) {
    extern __shared__ float ks[];   // N floats
    __shared__ float red[PRED_THREADS / 32];
    const int q = blockIdx.x;
    if (q >= M) return;
    const int N = p.N;
    float zq[4];
    for (int o = 0; o < 2; ++o) {
        if (o == 1 && p.shared) {
            // identical kernel row: only the mean weights differ
            float m = 0.0f;
            for (int j = threadIdx.x; j < N; j += blockDim.x) m += ks[j] * p.alpha[j * 2 + 1];
            m = block_sum(m, red);
            if (threadIdx.x == 0) {
                mean[q * 2 + 1] = m;
                var[q * 2 + 1] = var[q * 2 + 0];
            }
            break;
        }
        for (int d = 0; d < 4; ++d) zq[d] = Z[q * 4 + d] * p.zscale[o][d];
        const float* Xs = p.Xs[o];
        __syncthreads();
        float m = 0.0f;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            const float4 x = reinterpret_cast<const float4*>(Xs)[j];
            const float e0 = zq[0] - x.x, e1 = zq[1] - x.y, e2 = zq[2] - x.z, e3 = zq[3] - x.w;
            const float k = p.sf2[o] * exp2f(-(e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3));
            ks[j] = k;
            m += k * p.alpha[j * 2 + o];
        }
        m = block_sum(m, red);   // contains the barrier that publishes ks
        float qf = 0.0f;
        const float* W = p.W[o];
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            float v = 0.0f;
            for (int j = 0; j <= i; ++j) v += W[(size_t)j * p.Np + i] * ks[j];
            qf += v * v;
        }
        qf = block_sum(qf, red);
        if (threadIdx.x == 0) {
            mean[q * 2 + o] = m;
            var[q * 2 + o] = fmaxf(0.0f, p.sf2[o] - qf);
        }
    }
}

// max |L^-1| over the lower triangle (positive doubles order like their bits)
__global__ void k_absmax(const double* __restrict__ Xm, size_t n, unsigned long long* out) {
    double m = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(Xm[i]));
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Tensor-core tiles of the streaming rollout.  The factor's rows (output
// columns of V) are grouped in pairs of 128-row blocks (NP = ceil(NB / 2)
// pairs of 256 rows; the rows past NpM of an odd NB's last pair are zero) and
// its columns (training points) in stages of 32.  Piece (c, p) holds element
// (i = 256 p + r, j = 32 c + 8 sl + e) of cB L^-1 at
// ((c * NP + p) * 4 + sl) * 2048 + r * 8 + e, so one stage holds the 16 KiB
// pieces of all pairs contiguously, each as four 8-point slabs of 256 rows.
// Formats 0 (FP16) and 1 (BF16): hi = round(v), lo = round(v - hi); format 2
// (BF16, three parts): hi = round(v), mid = round(v - hi), lo = round(v - hi -
// mid), the residuals exact in double.  A GP of a terrain ensemble goes to the
// diagonal block of a stacked factor: its piece (c, p) lands at (c + c_off,
// p + p_off) of a grid NP_out pairs wide (a single GP: 0, 0, its own NP).
__global__ void k_pack_mma(const double* __restrict__ Xm, int N, int NpM, int fmt, double cB, int c_off,
                           int p_off, int NP_out, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                           uint16_t* __restrict__ mid) {
    const size_t idx0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int NP = (NpM / 128 + 1) / 2;
    const size_t total = (size_t)(NpM / 32) * NP * 8192;
    if (idx0 >= total) return;
    const size_t piece = idx0 / 8192;
    const int w = (int)(idx0 % 8192);
    const int c = (int)(piece / NP), p = (int)(piece % NP);
    const size_t idx = ((size_t)(c + c_off) * NP_out + (p + p_off)) * 8192 + w;
    const int sl = w / 2048, r = (w / 8) % 256, e = w % 8;
    const int i = 256 * p + r, j = 32 * c + 8 * sl + e;
    double v = 0.0;
    if (i < N && j < N && j <= i) v = cB * Xm[(size_t)i * N + j];
    if (fmt == 0) {
        const __half h = __double2half(v);
        hi[idx] = __half_as_ushort(h);
        lo[idx] = __half_as_ushort(__double2half(v - (double)__half2float(h)));
    } else if (fmt == 1) {
        const __nv_bfloat16 h = __double2bfloat16(v);
        hi[idx] = __bfloat16_as_ushort(h);
        lo[idx] = __bfloat16_as_ushort(__double2bfloat16(v - (double)__bfloat162float(h)));
    } else {
        const __nv_bfloat16 h = __double2bfloat16(v);
        const double r1 = v - (double)__bfloat162float(h);
        const __nv_bfloat16 m = __double2bfloat16(r1);
        hi[idx] = __bfloat16_as_ushort(h);
        mid[idx] = __bfloat16_as_ushort(m);
        lo[idx] = __bfloat16_as_ushort(__double2bfloat16(r1 - (double)__bfloat162float(m)));
    }
}

// Resident tiles of the cluster rollout.  Cluster rank r owns the 64-column
// slices r and NS - 1 - r of cB L^-1 (NS = NpC / 64); chunk c (training points
// 16c .. 16c + 15) of rank r is one piece: 128 rows (slice r then slice
// NS - 1 - r) while both slices need it (c < 4 (r + 1)), else 64 rows (slice
// NS - 1 - r alone, needed while c < 4 (NS - r)).  A piece is its hi part then
// its lo part, each slab-major: slab sl (points 8 sl .. 8 sl + 7), row rr at
// element sl * rows * 8 + rr * 8.  Pieces follow each other in chunk order;
// rank r's pieces start at element offset base[r].
__global__ void k_pack_cl(const double* __restrict__ Xm, int N, int NS, int fmt, double cB,
                          const int4* __restrict__ pieces, int npieces, uint16_t* __restrict__ out) {
    const int p = blockIdx.y;
    if (p >= npieces) return;
    const int4 d = pieces[p];            // (element offset, chunk, rank, rows per part)
    const int rows = d.w, R2 = 2 * rows; // the piece holds the hi and the lo rows
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R2 * 16) return;
    const int sl = idx / (R2 * 8), rr = (idx / 8) % R2, e = idx % 8;
    const int c = d.y, r = d.z;
    const int j = 16 * c + 8 * sl + e;
    const int lo_row = 64 * r, up_row = 64 * (NS - 1 - r);
    // row order: [hi lower | hi upper | lo upper | lo lower] while both slices
    // need the chunk (rows = 128), [hi upper | lo upper] after (rows = 64)
    int i;
    bool lo;
    if (rows == 128) {
        const int q = rr >> 6, o = rr & 63;
        i = (q == 0 || q == 3) ? lo_row + o : up_row + o;
        lo = q >= 2;
    } else {
        i = up_row + (rr & 63);
        lo = rr >= 64;
    }
    double v = 0.0;
    if (i < N && j < N && j <= i) v = cB * Xm[(size_t)i * N + j];
    uint16_t h;
    if (fmt == 0) {
        const __half hh = __double2half(v);
        h = lo ? __half_as_ushort(__double2half(v - (double)__half2float(hh))) : __half_as_ushort(hh);
    } else {
        const __nv_bfloat16 hh = __double2bfloat16(v);
        h = lo ? __bfloat16_as_ushort(__double2bfloat16(v - (double)__bfloat162float(hh)))
               : __bfloat16_as_ushort(hh);
    }
    out[(size_t)d.x + idx] = h;
}

}  // namespace

// training inputs and alpha of the cluster rollout in pair layout: for points
// 2p and 2p + 1, x[2p] = (x0, x0', x1, x1'), x[2p + 1] = (x2, x2', x3, x3') and
// a[p] = (a_v, a_v', a_w, a_w') (primes: point 2p + 1); rows j >= N get a far
// point (exp2 underflows to exactly 0) and alpha 0
// Training inputs and alpha of one GP in pair layout: point j (j < npc; far
// away with alpha 0 past N) at position J0 + j of an array of NpT points (a
// single GP: J0 = 0, NpT = npc; J0 even).
__global__ void k_pack_xa(const float* __restrict__ Xs, const float* __restrict__ alpha, int N, int npc,
                          int J0, int NpT, float* __restrict__ out) {
    const int j0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (j0 >= npc) return;
    const int j = j0;
    float4 x = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 1.0e4f);
    float2 al = make_float2(0.0f, 0.0f);
    if (j < N) {
        x = reinterpret_cast<const float4*>(Xs)[j];
        al = reinterpret_cast<const float2*>(alpha)[j];
    }
    const int J = J0 + j;
    float* xp = out + 8 * (J >> 1) + (J & 1);
    xp[0] = x.x;
    xp[2] = x.y;
    xp[4] = x.z;
    xp[6] = x.w;
    float* ap = out + 4 * NpT + 4 * (J >> 1) + (J & 1);
    ap[0] = al.x;
    ap[2] = al.y;
}

int build_cl_tiles(GpDevice& g, int fmt) {
    if (g.cl_tiles[fmt] || g.N == 0) return GPMPPI_OK;
    int rc = build_mma_tiles(g, fmt);      // sets cB (and the streaming tiles)
    if (rc) return rc;
    const int NpC = g.N <= 128 ? 128 : (g.N <= 256 ? 256 : 512);
    if (g.N > 512) return fail(GPMPPI_ERR_UNSUPPORTED, "cluster tiles: N > 512");
    const int NS = NpC / 64, CS = NS / 2;
    std::vector<int4> pieces;
    size_t off = 0;
    for (int r = 0; r < CS; ++r) {
        g.cl_base[r] = (int)off;
        for (int c = 0; c < 4 * (NS - r); ++c) {
            const int rows = (c < 4 * (r + 1)) ? 128 : 64;
            pieces.push_back(make_int4((int)off, c, r, rows));
            off += (size_t)rows * 16 * 2;
        }
        g.cl_bytes[r] = (int)((off - (size_t)g.cl_base[r]) * sizeof(uint16_t));
    }
    g.cl_npc = NpC;
    int4* dp = nullptr;
    GPM_CUDA(cudaMalloc(&dp, pieces.size() * sizeof(int4)));
    cudaError_t e = cudaMemcpy(dp, pieces.data(), pieces.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g.cl_tiles[fmt], off * sizeof(uint16_t));
    if (e == cudaSuccess) {
        k_pack_cl<<<dim3(16, (unsigned)pieces.size()), 256>>>(g.Linv64[0], g.N, NS, fmt, (double)g.mma_cB, dp,
                                                           (int)pieces.size(), g.cl_tiles[fmt]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dp);
    if (e != cudaSuccess) return cuda_fail(e, "build_cl_tiles");
    if (!g.cl_xa) {
        e = cudaMalloc(&g.cl_xa, sizeof(float) * 6 * (size_t)NpC);
        if (e == cudaSuccess) {
            k_pack_xa<<<(NpC + 127) / 128, 128>>>(g.Xs[0], g.alpha, g.N, NpC, 0, NpC, g.cl_xa);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "build_cl_tiles: training-set layout");
    }
    return GPMPPI_OK;
}

int build_mma_tiles(GpDevice& g, int fmt) {
    if (g.mma_hi[fmt] || g.N == 0) return GPMPPI_OK;
    const int N = g.N;
    g.NpM = ((N + 127) / 128) * 128;
    if (g.mma_cB == 0.0f) {
        unsigned long long* d = nullptr;
        GPM_CUDA(cudaMalloc(&d, sizeof(unsigned long long)));
        cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
        if (e == cudaSuccess) {
            k_absmax<<<256, 256>>>(g.Linv64[0], (size_t)N * N, d);
            e = cudaGetLastError();
        }
        unsigned long long bits = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost);
        cudaFree(d);
        if (e != cudaSuccess) return cuda_fail(e, "build_mma_tiles: absmax");
        double mx = 0.0;
        std::memcpy(&mx, &bits, sizeof(mx));
        // largest power of two with cB * max|L^-1| <= 2^14 (16-bit range, room for the sums)
        g.mma_cB = (float)std::ldexp(1.0, (int)std::floor(std::log2(16384.0 / (mx > 0 ? mx : 1.0))));
    }
    // 32-point stages x pairs of 128-row blocks x 256 rows x 32 points
    const size_t n = (size_t)(g.NpM / 32) * (size_t)((g.NpM / 128 + 1) / 2) * 8192;
    GPM_CUDA(cudaMalloc(&g.mma_hi[fmt], n * sizeof(uint16_t)));
    GPM_CUDA(cudaMalloc(&g.mma_lo[fmt], n * sizeof(uint16_t)));
    if (fmt == 2) GPM_CUDA(cudaMalloc(&g.mma_mid, n * sizeof(uint16_t)));
    k_pack_mma<<<(unsigned)((n + 255) / 256), 256>>>(g.Linv64[0], N, g.NpM, fmt, (double)g.mma_cB, 0, 0,
                                                      (g.NpM / 128 + 1) / 2, g.mma_hi[fmt], g.mma_lo[fmt],
                                                      g.mma_mid);
    GPM_CUDA(cudaGetLastError());
    if (!g.mma_xa) {
        // the streaming rollout's training inputs and alpha in pair layout
        GPM_CUDA(cudaMalloc(&g.mma_xa, sizeof(float) * 6 * (size_t)g.NpM));
        k_pack_xa<<<(g.NpM + 127) / 128, 128>>>(g.Xs[0], g.alpha, g.N, g.NpM, 0, g.NpM, g.mma_xa);
        GPM_CUDA(cudaGetLastError());
    }
    GPM_CUDA(cudaDeviceSynchronize());
    return GPMPPI_OK;
}

int build_mma_ensemble(GpDevice* const* gs, int M, int fmt, MmaTerrains& tr, uint16_t** hi, uint16_t** lo,
                       uint16_t** mid, float** xa) {
    *hi = *lo = *mid = nullptr;
    *xa = nullptr;
    tr = MmaTerrains{};
    tr.M = M;
    int nb = 0;
    for (int t = 0; t < M; ++t) {
        GpDevice& g = *gs[t];
        int rc = build_mma_tiles(g, fmt);             // the GP's cB (and its own tiles)
        if (rc) return rc;
        // an even number of blocks per GP: no block pair straddles two GPs
        const int nbt = g.N == 0 ? 0 : 2 * ((g.NpM / 128 + 1) / 2);
        tr.blk0[t] = nb;
        nb += nbt;
        const double r = (double)g.sf2[0] / (g.mma_cB > 0.0f ? (double)g.mma_cB : 1.0);
        tr.qscale[t] = (float)(r * r);
        tr.sf2[t] = g.sf2[0];
        tr.w[t] = 1.0f;
        for (int d = 0; d < 4; ++d) tr.zscale[t][d] = g.zscale[0][d];
    }
    tr.blk0[M] = nb;
    if (nb == 0) return GPMPPI_OK;
    const int NpT = nb * 128, NP = nb / 2;
    const size_t n = (size_t)(NpT / 32) * NP * 8192;
    GPM_CUDA(cudaMalloc(hi, n * sizeof(uint16_t)));
    GPM_CUDA(cudaMalloc(lo, n * sizeof(uint16_t)));
    GPM_CUDA(cudaMemset(*hi, 0, n * sizeof(uint16_t)));
    GPM_CUDA(cudaMemset(*lo, 0, n * sizeof(uint16_t)));
    if (fmt == 2) {
        GPM_CUDA(cudaMalloc(mid, n * sizeof(uint16_t)));
        GPM_CUDA(cudaMemset(*mid, 0, n * sizeof(uint16_t)));
    }
    GPM_CUDA(cudaMalloc(xa, sizeof(float) * 6 * (size_t)NpT));
    for (int t = 0; t < M; ++t) {
        const GpDevice& g = *gs[t];
        const int nbt = tr.blk0[t + 1] - tr.blk0[t];
        if (nbt == 0) continue;
        const size_t nt = (size_t)(nbt * 4) * (nbt / 2) * 8192;
        k_pack_mma<<<(unsigned)((nt + 255) / 256), 256>>>(g.Linv64[0], g.N, nbt * 128, fmt, (double)g.mma_cB,
                                                           4 * tr.blk0[t], tr.blk0[t] / 2, NP, *hi, *lo, *mid);
        GPM_CUDA(cudaGetLastError());
        k_pack_xa<<<(nbt * 128 + 127) / 128, 128>>>(g.Xs[0], g.alpha, g.N, nbt * 128, 128 * tr.blk0[t], NpT, *xa);
        GPM_CUDA(cudaGetLastError());
    }
    GPM_CUDA(cudaDeviceSynchronize());
    return GPMPPI_OK;
}

int launch_gp_predict(const GpDevice& g, const float* Z, int M, float* mean, float* var,
                      cudaStream_t st) {
    if (M == 0) return GPMPPI_OK;
    PredArgs p;
    for (int o = 0; o < 2; ++o) {
        p.Xs[o] = g.Xs[o];
        p.W[o] = g.W[o];
        p.sf2[o] = g.sf2[o];
        for (int d = 0; d < 4; ++d) p.zscale[o][d] = g.zscale[o][d];
    }
    p.alpha = g.alpha;
    p.N = g.N;
    p.Np = g.Np;
    p.shared = g.shared;
    const size_t smem = (size_t)(g.N > 0 ? g.N : 1) * sizeof(float);
    GPM_CUDA(cudaFuncSetAttribute(k_gp_predict, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    k_gp_predict<<<M, PRED_THREADS, smem, st>>>(p, Z, M, mean, var);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

// Fit both outputs.  X (N x 4) and Y (N x 2) are host arrays; g.hyper is set.
int gp_fit_device(GpDevice& g, const double* X, const double* Y, int N, cudaStream_t st) {
    g.N = N;
    // rows of W padded to a multiple of 16, at least 64 so that every TMA box
    // of the rollout fits inside the tensor; N = 0 has no W at all
    g.Np = (N > 0) ? ((N + 15) / 16) * 16 : 0;
    if (g.Np > 0 && g.Np < 64) g.Np = 64;
    const double log2e = 1.4426950408889634;
    for (int o = 0; o < 2; ++o) {
        g.sf2[o] = (float)g.hyper[o].signal_var;
        for (int d = 0; d < 4; ++d)
            g.zscale[o][d] = (float)(std::sqrt(0.5 * log2e) / g.hyper[o].lengthscale[d]);
    }
    const int nout = g.shared ? 1 : 2;
    const size_t nn = (size_t)N * N;
    // device allocations owned by g (freed by the caller on any failure)
    GPM_CUDA(cudaMalloc(&g.alpha, sizeof(float) * 2 * (N > 0 ? N : 1)));
    for (int o = 0; o < nout; ++o) {
        GPM_CUDA(cudaMalloc(&g.Xs[o], sizeof(float) * 4 * (N > 0 ? N : 1)));
        GPM_CUDA(cudaMalloc(&g.W[o], sizeof(float) * (g.Np > 0 ? (size_t)g.Np * g.Np : 1)));
        GPM_CUDA(cudaMalloc(&g.Linv64[o], sizeof(double) * (nn > 0 ? nn : 1)));
        GPM_CUDA(cudaMalloc(&g.alpha64[o], sizeof(double) * (N > 0 ? N : 1)));
    }
    if (g.shared) {
        g.Xs[1] = g.Xs[0];
        g.W[1] = g.W[0];
        g.Linv64[1] = g.Linv64[0];
        GPM_CUDA(cudaMalloc(&g.alpha64[1], sizeof(double) * (N > 0 ? N : 1)));
    }
    if (N == 0) return GPMPPI_OK;

    double *dX = nullptr, *dY = nullptr, *dA = nullptr, *dt = nullptr;
    int* dflag = nullptr;
    auto cleanup = [&]() {
        cudaFree(dX);
        cudaFree(dY);
        cudaFree(dA);
        cudaFree(dt);
        cudaFree(dflag);
    };
    auto check = [&](cudaError_t e, const char* what) -> int {
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, what);
        }
        return GPMPPI_OK;
    };
    int rc;
    if ((rc = check(cudaMalloc(&dX, sizeof(double) * 4 * N), "cudaMalloc X"))) return rc;
    if ((rc = check(cudaMalloc(&dY, sizeof(double) * 2 * N), "cudaMalloc Y"))) return rc;
    if ((rc = check(cudaMalloc(&dA, sizeof(double) * nn), "cudaMalloc K"))) return rc;
    if ((rc = check(cudaMalloc(&dt, sizeof(double) * N), "cudaMalloc t"))) return rc;
    if ((rc = check(cudaMalloc(&dflag, sizeof(int)), "cudaMalloc flag"))) return rc;
    if ((rc = check(cudaMemcpyAsync(dX, X, sizeof(double) * 4 * N, cudaMemcpyHostToDevice, st),
                    "copy X")))
        return rc;
    if ((rc = check(cudaMemcpyAsync(dY, Y, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, st),
                    "copy Y")))
        return rc;
    const int nblk = (N + NB - 1) / NB;
    for (int o = 0; o < nout; ++o) {
        const gpmppi_hyper& h = g.hyper[o];
        if ((rc = check(cudaMemsetAsync(dflag, 0, sizeof(int), st), "memset flag"))) return rc;
        dim3 b16(16, 16), gK((N + 15) / 16, (N + 15) / 16);
        k_build_kxx<<<gK, b16, 0, st>>>(dX, N, 1.0 / h.lengthscale[0], 1.0 / h.lengthscale[1],
                                        1.0 / h.lengthscale[2], 1.0 / h.lengthscale[3],
                                        h.signal_var, h.noise_var, dA);
        for (int kb = 0; kb < N; kb += NB) {
            const int n = (N - kb < NB) ? (N - kb) : NB;
            k_potrf_diag<<<1, dim3(NB, NB), 0, st>>>(dA, N, kb, n, dflag);
            const int rest = N - kb - n;
            if (rest > 0) {
                const int nb_rest = (rest + NB - 1) / NB;
                k_trsm_panel<<<nb_rest, dim3(NB, NB), 0, st>>>(dA, N, kb, n);
                k_syrk<<<dim3(nb_rest, nb_rest), dim3(NB, NB), 0, st>>>(dA, N, kb, n);
            }
        }
        if ((rc = check(cudaGetLastError(), "cholesky kernels"))) return rc;
        int hflag = 0;
        if ((rc = check(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st),
                        "copy flag")))
            return rc;
        if ((rc = check(cudaStreamSynchronize(st), "cholesky sync"))) return rc;
        if (hflag) {
            cleanup();
            return fail(GPMPPI_ERR_NOT_PD, "gp_fit: K_XX + noise_var I is not positive definite");
        }
        if ((rc = check(cudaMemsetAsync(g.Linv64[o], 0, sizeof(double) * nn, st), "memset Linv")))
            return rc;
        k_trtri<<<nblk, dim3(NB, NB), 0, st>>>(dA, N, g.Linv64[o]);
        const int tb = 128, gb = (N + tb - 1) / tb;
        const int outs[2] = {o, g.shared ? 1 : -1};
        for (int oo : outs) {
            if (oo < 0) continue;
            k_matvec<<<gb, tb, 0, st>>>(g.Linv64[o], dY + oo, N, 2, dt);
            k_matvec_t<<<gb, tb, 0, st>>>(g.Linv64[o], dt, N, g.alpha64[oo]);
        }
        const double s = std::sqrt(0.5 * log2e);
        k_pack_x<<<gb, tb, 0, st>>>(dX, N, s / h.lengthscale[0], s / h.lengthscale[1],
                                    s / h.lengthscale[2], s / h.lengthscale[3], g.Xs[o]);
        k_pack_w<<<dim3((g.Np + 127) / 128, g.Np), 128, 0, st>>>(g.Linv64[o], N, g.Np, g.W[o]);
        if ((rc = check(cudaGetLastError(), "inverse kernels"))) return rc;
    }
    k_pack_alpha<<<(N + 127) / 128, 128, 0, st>>>(g.alpha64[0], g.alpha64[1], N, g.alpha);
    if ((rc = check(cudaGetLastError(), "pack alpha"))) return rc;
    if ((rc = check(cudaStreamSynchronize(st), "gp_fit sync"))) return rc;
    cleanup();
    return GPMPPI_OK;
}

}  // namespace gpm
