// tc_nonlinear_noalloc: the nonlinear-term evaluation for callers that must not allocate
// device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a host loop with real-time
// deadlines (cudaMalloc can block and synchronise the device), a plug-in living inside a
// framework that owns every byte of device memory through its own pool, or a caller that
// simply has no way to hand us a workspace.  Such a caller passes only its input and output
// arrays; the staging lines between the three transform kernels live in one static device
// array of this library instead of a caller workspace.
//
// Costs and limits:
//  - kStaticScratchBytes (80 MiB) of device memory is reserved on every GPU that loads this
//    library, for as long as the process lives.  Plans whose staging needs more are rejected
//    with TC_ERR_ARG before anything is launched.  The staging is everything the workspace
//    holds before N^i: the z-pass lines H1 and H2 (12 line sets: complex128 lines of
//    stage_rows radial rows for TC_FP64 plans, complex64 lines of all rows for TC_MIXED
//    plans), and for TC_MIXED plans the FP32 split of u and d_r u, 6 * N_r * (M+1) * (2K+1)
//    complex64 values, each region rounded up to 256 bytes.
//  - All calls share the one array, which keeps whatever the last call left in it.  The
//    kernels overwrite every staging entry before reading it, so nothing has to start at
//    zero, but two calls whose work overlaps on the GPU (different streams, or different
//    plans without ordering between them) race on the array: order them on one stream.
//  - The first call on each device looks up the array's device address once with
//    cudaGetSymbolAddress (with that device current) and keeps it for the life of the
//    process.  Make that first call before any stream capture begins.  A device reset
//    (cudaDeviceReset, or a reset of the primary context) unloads the array, and the kept
//    address is then stale: do not call this entry point after resetting a device.
#include <mutex>

#include "tc_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)80 << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (set up once per device).
tc_status scratch_on_current_device(tc_plan* p, void** out) {
    int dev = -1;
    TC_CUDA(p, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(p->err, sizeof(p->err), "tc_nonlinear_noalloc: device index %d not supported", dev);
        return TC_ERR_STATE;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) return tc::cuda_fail(p, e, "cudaGetSymbolAddress(g_scratch)");
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return TC_OK;
}

}  // namespace

extern "C" tc_status tc_nonlinear_noalloc(tc_plan* plan, const void* u_hat, void* N_hat, void* stream) {
    if (!plan) return TC_ERR_ARG;
    if (plan->host_only) {
        snprintf(plan->err, sizeof(plan->err), "host-only plan");
        return TC_ERR_STATE;
    }
    // staging used by the transform kernels: H1 (9 line sets), H2 (3 line sets) and, for the
    // mixed form, the FP32 split of u and d_r u -- every workspace region before N^i
    const size_t need = plan->ws.Ncur;
    if (need > kStaticScratchBytes) {
        snprintf(plan->err, sizeof(plan->err),
                 "tc_nonlinear_noalloc: this plan needs %zu bytes of staging but the static scratch "
                 "holds %zu bytes (80 MiB); use tc_nonlinear with a workspace", need, kStaticScratchBytes);
        return TC_ERR_ARG;
    }
    int dev = -1;
    TC_CUDA(plan, cudaGetDevice(&dev));
    if (dev != plan->device) {
        snprintf(plan->err, sizeof(plan->err), "current device %d differs from the plan's device %d", dev, plan->device);
        return TC_ERR_STATE;
    }
    tc_status st = tc::check_device_ptr(plan, u_hat, "u_hat", 3 * plan->S * sizeof(double2));
    if (st != TC_OK) return st;
    st = tc::check_device_ptr(plan, N_hat, "N_hat", 3 * plan->S * sizeof(double2));
    if (st != TC_OK) return st;
    if (u_hat == N_hat) return TC_ERR_ARG;
    void* scratch = nullptr;
    st = scratch_on_current_device(plan, &scratch);
    if (st != TC_OK) return st;
    plan->used = true;   // a compute call: tc_plan_set is refused from here on
    return tc::launch_nonlinear(plan, static_cast<const double2*>(u_hat), static_cast<double2*>(N_hat),
                                static_cast<char*>(scratch), static_cast<cudaStream_t>(stream));
}
