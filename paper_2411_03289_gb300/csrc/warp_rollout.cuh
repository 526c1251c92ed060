// Building blocks of the warp-per-sample rollout kernels (the adjoint
// rollout and the terrain-ensemble rollout): a CTA of GMT warps carries GMT
// samples, one warp each, so that a sample's scalar work (dynamics,
// covariance, costs) stays in one warp while the triangular products with the
// GP factor are shared by the whole CTA.
#pragma once

#include <cfloat>

#include "common.cuh"

namespace gpm {
namespace wr {
namespace {

constexpr int GMT = 8;              // samples per CTA (one warp each)
constexpr int GT = GMT * 32;        // threads per CTA
constexpr int REC = 20;             // mu (5) + Sigma upper triangle (15)

// upper-triangle position of Sigma[i][j], i <= j: rows hold 5, 4, 3, 2, 1 entries
__host__ __device__ constexpr int sidx(int i, int j) { return i * 5 - (i * (i - 1)) / 2 + (j - i); }

__device__ __forceinline__ float wsum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// warp-wide minimum with the smallest index among equal values
__device__ __forceinline__ void wargmin(float& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov < v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
}

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ float2 ldg2(const float* p) {
    return __ldg(reinterpret_cast<const float2*>(p));
}

template <int CPL>
struct Cols;
template <>
struct Cols<1> {
    using V = float;
    static __device__ __forceinline__ V load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float at(const V& v, int) { return v; }
};
template <>
struct Cols<2> {
    using V = float2;
    static __device__ __forceinline__ V load(const float* p) { return ldg2(p); }
    static __device__ __forceinline__ float at(const V& v, int c) { return c ? v.y : v.x; }
};

// Rows [r0, r1) of the product for the thread's two column groups of CPL
// columns each: LO / HI say which of the groups (at pl / ph) take part.  r0
// and r1 are multiples of 16.
template <int CPL, bool LO, bool HI>
__device__ __forceinline__ void tri_rows(int Np, const float* in, int r0, int r1, const float* pl,
                                         const float* ph, bool okl, bool okh, float (&al)[GMT][CPL],
                                         float (&ah)[GMT][CPL]) {
    using C = Cols<CPL>;
    typename C::V zero;
    if constexpr (CPL == 1) zero = 0.0f; else zero = make_float2(0.f, 0.f);
    for (int r = r0; r < r1; r += 8) {
        typename C::V ml[8], mh[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (LO) ml[u] = okl ? C::load(pl + (size_t)(r + u) * Np) : zero;
            if (HI) mh[u] = okh ? C::load(ph + (size_t)(r + u) * Np) : zero;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 x0 = *reinterpret_cast<const float4*>(in + (r + u) * GMT);
            const float4 x1 = *reinterpret_cast<const float4*>(in + (r + u) * GMT + 4);
            const float xs[GMT] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int s = 0; s < GMT; ++s)
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    if (LO) al[s][c] = fmaf(xs[s], C::at(ml[u], c), al[s][c]);
                    if (HI) ah[s][c] = fmaf(xs[s], C::at(mh[u], c), ah[s][c]);
                }
        }
    }
}

// The product below with column blocks of 32 CPL columns.
template <bool LOWER, int CPL>
__device__ void tri_product_cols(const float* __restrict__ M, int Np, const float* in, float* out) {
    constexpr int NBLK = 2 * (GT / 32);
    constexpr int BW = 32 * CPL;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < Np; c0 += NBLK * BW) {
        const int blo = c0 + BW * warp, bhi = c0 + BW * (NBLK - 1 - warp);
        if (blo >= Np) continue;                  // then bhi >= Np too (warp-uniform)
        const int clo = blo + CPL * lane, chi = bhi + CPL * lane;
        const bool okl = clo < Np, okh = chi < Np;
        const bool hi_any = bhi < Np;              // warp-uniform
        float al[GMT][CPL], ah[GMT][CPL];
#pragma unroll
        for (int s = 0; s < GMT; ++s)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                al[s][c] = 0.0f;
                ah[s][c] = 0.0f;
            }
        const float* pl = M + (okl ? clo : 0);
        const float* ph = M + (okh ? chi : 0);
        // block edges are multiples of 32 and Np of 16: every row range below
        // starts and ends on a multiple of 16
        if (!LOWER) {
            const int el = min(Np, blo + BW);
            if (hi_any) {
                tri_rows<CPL, true, true>(Np, in, 0, el, pl, ph, okl, okh, al, ah);
                tri_rows<CPL, false, true>(Np, in, el, min(Np, bhi + BW), pl, ph, okl, okh, al, ah);
            } else {
                tri_rows<CPL, true, false>(Np, in, 0, el, pl, ph, okl, okh, al, ah);
            }
        } else {
            if (hi_any) {
                tri_rows<CPL, true, false>(Np, in, blo, bhi, pl, ph, okl, okh, al, ah);
                tri_rows<CPL, true, true>(Np, in, bhi, Np, pl, ph, okl, okh, al, ah);
            } else {
                tri_rows<CPL, true, false>(Np, in, blo, Np, pl, ph, okl, okh, al, ah);
            }
        }
        if (okl) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                float4* o = reinterpret_cast<float4*>(out + (clo + c) * GMT);
                o[0] = make_float4(al[0][c], al[1][c], al[2][c], al[3][c]);
                o[1] = make_float4(al[4][c], al[5][c], al[6][c], al[7][c]);
            }
        }
        if (okh) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                float4* o = reinterpret_cast<float4*>(out + (chi + c) * GMT);
                o[0] = make_float4(ah[0][c], ah[1][c], ah[2][c], ah[3][c]);
                o[1] = make_float4(ah[4][c], ah[5][c], ah[6][c], ah[7][c]);
            }
        }
    }
}

// out[i * GMT + s] = sum_r in[r * GMT + s] * M[r * Np + i] for every column i < Np.
// LOWER = false: M holds rows of L^-T (M[r][i] = 0 for i < r), so a column
// block [b, b + BW) needs rows [0, b + BW); LOWER = true: M holds rows of L^-1
// (M[r][i] = 0 for i > r), so it needs rows [b, Np).  Both matrices are
// zero-padded to Np x Np.  Each pass covers 16 column blocks; warp w takes
// blocks w and 15 - w (lane l their columns l CPL .. l CPL + CPL - 1), so that
// every warp visits the same number of rows of either triangle.  Blocks are 64
// columns wide (CPL = 2, float2 loads) where that keeps the warps balanced
// (768 < Np <= 1024 or Np >= 2048) and 32 wide elsewhere.  Called by all
// threads; no barrier inside.
template <bool LOWER>
__device__ void tri_product(const float* __restrict__ M, int Np, const float* in, float* out) {
    if ((Np > 768 && Np <= 1024) || Np >= 2048)
        tri_product_cols<LOWER, 2>(M, Np, in, out);
    else
        tri_product_cols<LOWER, 1>(M, Np, in, out);
}

struct Lam {
    float lmax, sq;          // clamped eigenvalue and its square root
    float dxx, dxy, dyy;     // d sqrt(lmax) / d (Sxx, Sxy, Syy)
};

__device__ __forceinline__ Lam lam_max(float sxx, float sxy, float syy) {
    Lam L;
    const float d = 0.5f * (sxx - syy);
    const float h = hypotf(d, sxy);
    const float raw = 0.5f * (sxx + syy) + h;
    L.lmax = fmaxf(0.0f, raw);
    L.sq = sqrtf(L.lmax);
    // derivative of the square root: zero where it is undefined (Sigma_XY = 0)
    const float ds = (raw > 0.0f && L.sq > 0.0f) ? 0.5f / L.sq : 0.0f;
    const float gx = (h > 0.0f) ? 0.5f + 0.5f * d / h : 0.5f;
    const float gy = (h > 0.0f) ? 0.5f - 0.5f * d / h : 0.5f;
    const float gxy = (h > 0.0f) ? sxy / h : 0.0f;
    L.dxx = ds * gx;
    L.dxy = ds * gxy;
    L.dyy = ds * gy;
    return L;
}

// nearest lane segment of point (px, py): squared distance and index (warp-wide)
__device__ __forceinline__ void lane_nearest(const RolloutArgs& a, float px, float py, float& best,
                                             int& bi) {
    const int lane = threadIdx.x & 31;
    best = FLT_MAX;
    bi = 0x7fffffff;
    const int2 oc = lane_cands(a, px, py);                 // candidate segments of this position
    for (int i = lane; i < oc.y; i += 32) {
        const int gI = lane_seg(a, oc, i);
        const float4 sg = __ldg(a.seg + gI);
        const float il2 = __ldg(a.seg_il2 + gI);
        const float qx0 = px - sg.x, qy0 = py - sg.y;
        const float t = fminf(fmaxf((qx0 * sg.z + qy0 * sg.w) * il2, 0.0f), 1.0f);
        const float qx = qx0 - t * sg.z, qy = qy0 - t * sg.w;
        const float d2 = qx * qx + qy * qy;
        if (d2 < best) {
            best = d2;
            bi = gI;
        }
    }
    wargmin(best, bi);
}

// obstacle margin d_bar (Eq. 15-16) of obstacle o at (px, py)
__device__ __forceinline__ float obstacle_margin(const RolloutArgs& a, int o, float px, float py,
                                                 float sxx, float sxy, float syy, float sqlam) {
    const float cx = __ldg(a.obst + 3 * o), cy = __ldg(a.obst + 3 * o + 1), R = __ldg(a.obst + 3 * o + 2);
    const float dx = px - cx, dy = py - cy;
    const float rho = sqrtf(dx * dx + dy * dy);
    float spread;
    if (rho > 1e-9f) {
        const float nx = dx / rho, ny = dy / rho;
        spread = sqrtf(fmaxf(0.0f, nx * nx * sxx + 2.0f * nx * ny * sxy + ny * ny * syy));
    } else {
        spread = sqrtf(fmaxf(0.0f, sqlam * sqlam));
    }
    return (rho - R) - a.phi_inv * spread;
}

__device__ __forceinline__ void obstacle_nearest(const RolloutArgs& a, float px, float py, float sxx,
                                                 float sxy, float syy, float sqlam, float& best,
                                                 int& bi) {
    const int lane = threadIdx.x & 31;
    best = FLT_MAX;
    bi = 0x7fffffff;
    for (int o = lane; o < a.O; o += 32) {
        const float m = obstacle_margin(a, o, px, py, sxx, sxy, syy, sqlam);
        if (m < best) {
            best = m;
            bi = o;
        }
    }
    wargmin(best, bi);
}

}  // namespace
}  // namespace wr
}  // namespace gpm
