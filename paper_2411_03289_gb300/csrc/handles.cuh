// Internal layout of the opaque handles of the C ABI (gpmppi_gp, gpmppi_ctrl),
// shared by the translation units that implement the ABI.
#pragma once


#include "common.cuh"

constexpr uint32_t kGpMagicValue = 0x47504d31u;     // "GPM1"
constexpr uint32_t kCtrlMagicValue = 0x4d505031u;   // "MPP1"

struct gpmppi_gp_s {
    uint32_t magic = kGpMagicValue;
    gpm::GpDevice g;
};

struct gpmppi_ctrl_s {
    uint32_t magic = kCtrlMagicValue;
    gpmppi_params p{};
    gpmppi_gp gp = nullptr;
    int device = 0;
    int O = 0, P = 0, S = 0;
    int mt = 1, n_upd = 1;
    uint64_t it = 0;
    uint64_t wait_ns = 2000000000ull;   // FP32 rollout: limit of each tile-copy wait
    int expire_first = 0;               // FP32 rollout: failure-detection hook
    double sq_chi2 = 0.0, phi_inv = 0.0;
    float* obst = nullptr;
    float4* seg = nullptr;
    float* seg_il2 = nullptr;
    float* costs = nullptr;       // K, used when the caller passes no costs array
    float* hs_U = nullptr;        // mppi_step_host staging: U_nom then U_new (2 x T x 2)
    float* hs_w = nullptr;        // mppi_step_host staging: weights (K)
    // a terrain ensemble on the tensor cores: the stacked factor tiles and
    // training set of its GPs (owned by the controller)
    uint16_t* ens_hi = nullptr;
    uint16_t* ens_lo = nullptr;
    uint16_t* ens_mid = nullptr;
    float* ens_xa = nullptr;
    float2* u_tilde = nullptr;    // T x K
    float* partial = nullptr;     // n_upd x T x 2 update partials, then n_upd x 2 block statistics
    unsigned int* counter = nullptr;
    float* nom_sxy = nullptr;     // T x 3
    int2* gcell = nullptr;        // lane-distance grid (null: scan every segment)
    int* gidx = nullptr;
    float gx0 = 0, gy0 = 0, ginv = 0;
    int gnx = 0, gny = 0;
    unsigned int* err = nullptr;  // device status word written by the rollout
    int stages = 2;               // per-warp TMA pipeline depth
    CUtensorMap tmW;              // TMA map over the GP's W
    gpm::MmaArgs mm{};              // tensor-core tiles (split precisions)
    int fmt = -1;                 // 0 = FP16, 1 = BF16 split, -1 = FP32 path
    bool cl = false;              // split precisions with N <= 512: the cluster rollout
    gpm::ClArgs cla{};
    // terrain ensemble (Eq. 3): M >= 2 GPs mixed with weights tw on the
    // ensemble rollout; M = 1 is the single GP `gp`
    int M = 1;
    bool ens = false;             // runs the ensemble rollout
    gpmppi_gp tgp[gpm::kMaxTerrains] = {};
    float tw[gpm::kMaxTerrains] = {};
    // adjoint-rollout scratch (allocated by the first mppi_grad call)
    void* grad_scr = nullptr;
    size_t grad_bytes = 0;
    bool profiling = false;
    bool profiled = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};


namespace gpm {
// Launch arguments of one rollout of controller c from state (host, 5) with
// nominal controls U (device, T x 2).
RolloutArgs make_rollout_args(gpmppi_ctrl c, const float* state, const float* U);
}  // namespace gpm
