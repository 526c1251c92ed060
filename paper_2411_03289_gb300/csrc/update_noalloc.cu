// Allocation-free entry point for the MPPI weights-and-update step.
//
// Some callers of this library cannot call cudaMalloc once they are running:
// a controller inside a real-time loop whose device memory is fixed at
// start-up (an allocation may synchronise the device and has no latency
// bound), or a host framework that owns all device memory and forbids its
// plug-ins from allocating.  mppi_update_noalloc serves them: it runs the same
// update kernel as mppi_step's second launch, but the kernel's scratch (the
// per-CTA partial sums and the completion ticket) lives in the fixed static
// device array below instead of in buffers a controller allocated.  The
// caller passes every input and output.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

// ceil(K / 256) * T * 2 partial sums at most, then two statistics per
// sample block (at most 2 * 65536 floats), then one ticket word.
constexpr int kNoallocPartials = 1 << 17;     // 512 KiB of floats
constexpr int kNoallocFloats = 2 * kNoallocPartials + 64;   // 1 MiB + 256 B in all
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[kNoallocFloats];

struct DeviceScratch {
    float* partial = nullptr;
    unsigned int* ticket = nullptr;
};

DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// The host-side name of a __device__ array is only a stand-in; the device
// address is looked up once per device, with that device current.
int scratch_for_current_device(DeviceScratch* out) {
    int dev = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return gpm::fail(GPMPPI_ERR_UNSUPPORTED, "mppi_update_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch[dev].partial) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return gpm::cuda_fail(e, "mppi_update_noalloc: cudaGetSymbolAddress");
        g_scratch[dev].partial = static_cast<float*>(p);
        g_scratch[dev].ticket = reinterpret_cast<unsigned int*>(static_cast<float*>(p) + 2 * kNoallocPartials);
    }
    *out = g_scratch[dev];
    return GPMPPI_OK;
}

}  // namespace

extern "C" int mppi_update_noalloc(const float* costs, const float* u_tilde, const float* U_nom,
                                   float* U_new, float* weights, int32_t K, int32_t T, float lambda,
                                   void* stream) {
    using namespace gpm;
    if (K < 1 || T < 1) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_update_noalloc: K and T must be >= 1");
    if (!(lambda > 0.0f) || !std::isfinite(lambda))
        return fail(GPMPPI_ERR_INVALID_ARG, "mppi_update_noalloc: lambda must be finite and > 0");
    const long long n_cta = ((long long)K + 255) / 256;
    if (n_cta * (long long)T * 2 > kNoallocPartials || T > GPMPPI_MAX_T)
        return fail(GPMPPI_ERR_INVALID_ARG,
                    "mppi_update_noalloc: ceil(K/256) * T must not exceed 65536 (and T <= GPMPPI_MAX_T)");
    int rc;
    // device (or managed) memory of the current device: a host pointer or an
    // array on another GPU is refused here instead of faulting in the kernel
    if ((rc = check_dev_ptr(costs, "mppi_update_noalloc: costs", false))) return rc;
    if ((rc = check_dev_ptr(u_tilde, "mppi_update_noalloc: u_tilde", false))) return rc;
    if ((rc = check_dev_ptr(U_nom, "mppi_update_noalloc: U_nom", false))) return rc;
    if ((rc = check_dev_ptr(U_new, "mppi_update_noalloc: U_new", false))) return rc;
    if ((rc = check_dev_ptr(weights, "mppi_update_noalloc: weights", true))) return rc;
    if (U_new == U_nom) return fail(GPMPPI_ERR_INVALID_ARG, "mppi_update_noalloc: U_new must not alias U_nom");
    if (reinterpret_cast<uintptr_t>(u_tilde) & 7u)
        return fail(GPMPPI_ERR_INVALID_ARG, "mppi_update_noalloc: u_tilde must be 8-byte aligned");
    DeviceScratch sc;
    if ((rc = scratch_for_current_device(&sc))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the ticket must start at zero; the partial sums and block statistics
    // (ceil(K/256) * (T + 1) * 2 floats, within the array since
    // ceil(K/256) * T <= 65536) are fully written by their CTAs before the
    // last one reads them
    GPM_CUDA(cudaMemsetAsync(sc.ticket, 0, sizeof(unsigned int), st));
    UpdateArgs a;
    a.costs = costs;
    a.u_tilde = reinterpret_cast<const float2*>(u_tilde);
    a.U = U_nom;
    a.U_new = U_new;
    a.weights = weights;
    a.partial = sc.partial;
    a.counter = sc.ticket;
    a.K = K;
    a.T = T;
    a.per_cta = 256;
    a.inv_lambda = 1.0f / lambda;
    return launch_update(a, (int)n_cta, st, false);
}
