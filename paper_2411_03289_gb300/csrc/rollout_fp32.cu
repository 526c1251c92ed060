// Fused MPPI rollout, FP32 on the CUDA cores (Alg. 1 Step 1).
//
// One CTA owns `mt` samples and carries them through all T steps of the
// horizon (the recurrence of Eq. 10 is sequential in k).  Per step k:
//   P1  (warp 0, lane = sample) Philox noise, clamp (Eq. 8), GP query z
//   P2  (all)  k*_j = sf2 exp(-|z - x_j|^2 / 2l^2) into shared memory, and the
//              mean partials k* . alpha (Eq. 3)
//   P3  (all)  V = K* L^-T as a register-tiled triangular product; each thread
//              squares and sums its tile, giving partial |L^-1 k*|^2.  Every
//              warp streams the two column tiles of L^-T it needs through its
//              own ring of shared-memory stages filled by TMA tensor copies
//              (cp.async.bulk.tensor, completion on an mbarrier), so the FMA
//              loop reads shared memory while later rows are in flight
//   P4  (warp 0) GP mean / variance, mean dynamics (Eq. 6, 10), covariance
//              A Sigma A^T + diag(0,0,0,s,s) (Eq. 10), obstacle chance
//              constraint (Eq. 15-16), variance and speed terms (Eq. 11-12)
//   P5  (all)  distance to the lane polyline, split over segments
//   P6  (warp 0) lane deviation and tightened lane indicator (Eq. 11, 13-14)
// The triangular product dominates: N(N+1)/2 FMAs per sample-step.
#include "rollout_fp32_body.cuh"

namespace gpm {
namespace {

using namespace f32r;

template <int MTP, bool TRACE>
__global__ void __launch_bounds__(THREADS, 1)
    k_rollout_fp32(const RolloutArgs a, const __grid_constant__ CUtensorMap tmW) {
    // no static shared memory in this kernel: the dynamic region starts at the
    // base of the CTA's shared memory, aligned as the tensor copies need
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    rollout_fp32_body<MTP, TRACE>(a, &tmW, blockIdx.x, smem_raw);
}

template <int MTP, bool TRACE>
int launch_t(const RolloutArgs& a, const CUtensorMap* tm, cudaStream_t st) {
    const int smem = Smem<MTP>::total(a.Np, a.stages);
    auto kern = k_rollout_fp32<MTP, TRACE>;
    GPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int grid = (a.K + a.mt - 1) / a.mt;
    kern<<<grid, THREADS, smem, st>>>(a, *tm);
    GPM_CUDA(cudaGetLastError());
    return GPMPPI_OK;
}

template <int MTP>
int tile_box(int* w, int* h) {
    *w = Tile<MTP>::TW;
    *h = Tile<MTP>::R;
    return GPMPPI_OK;
}

}  // namespace

int rollout_fp32_mtp(int Np) {
    if (Np <= 1024) return 32;
    if (Np <= 2048) return 16;
    return 8;
}

int rollout_fp32_smem_bytes(int Np, int mtp, int stages) {
    switch (mtp) {
        case 32: return Smem<32>::total(Np, stages);
        case 16: return Smem<16>::total(Np, stages);
        default: return Smem<8>::total(Np, stages);
    }
}

int rollout_fp32_stages(int Np, int smem_optin) {
    const int mtp = rollout_fp32_mtp(Np);
    for (int s = 4; s >= 2; --s)
        if (rollout_fp32_smem_bytes(Np, mtp, s) <= smem_optin) return s;
    return 0;
}

int make_w_tensor_map(CUtensorMap* out, const float* W, int Np) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        GPM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                  cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn)
            return fail(GPMPPI_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    int bw = 0, bh = 0;
    switch (rollout_fp32_mtp(Np)) {
        case 32: tile_box<32>(&bw, &bh); break;
        case 16: tile_box<16>(&bw, &bh); break;
        default: tile_box<8>(&bw, &bh); break;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)Np, (cuuint64_t)Np};
    const cuuint64_t strides[1] = {(cuuint64_t)Np * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(W), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GPMPPI_ERR_CUDA, "cuTensorMapEncodeTiled failed for L^-T");
    return GPMPPI_OK;
}

int launch_rollout_fp32(const RolloutArgs& a, const CUtensorMap* tm, bool trace, cudaStream_t st) {
    const int mtp = rollout_fp32_mtp(a.Np);
    if (a.mt < 1 || a.mt > mtp) return fail(GPMPPI_ERR_INVALID_ARG, "rollout: bad samples per CTA");
    if (a.stages < 2 || a.stages > 4) return fail(GPMPPI_ERR_INVALID_ARG, "rollout: bad pipeline depth");
    if (trace) {
        switch (mtp) {
            case 32: return launch_t<32, true>(a, tm, st);
            case 16: return launch_t<16, true>(a, tm, st);
            default: return launch_t<8, true>(a, tm, st);
        }
    }
    switch (mtp) {
        case 32: return launch_t<32, false>(a, tm, st);
        case 16: return launch_t<16, false>(a, tm, st);
        default: return launch_t<8, false>(a, tm, st);
    }
}

}  // namespace gpm
