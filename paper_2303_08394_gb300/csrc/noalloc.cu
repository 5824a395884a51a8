// fmm_evaluate_noalloc: the evaluation of fmm_evaluate, with its
// per-evaluation workspace taken from a fixed array in device global memory
// instead of memory the plan allocates.
//
// Who needs it: code that may not allocate device memory at evaluation
// time -- an application whose device memory budget is owned by another
// allocator (a framework's caching allocator), a latency-critical loop in
// which cudaMalloc/cudaFree would add their implicit device-wide
// synchronisation, or a long-running service that must not grow its device
// footprint after start-up.  fmm_evaluate allocates its workspace on the
// first call and whenever nrhs grows; this entry point never allocates.
//
// The array below is a file-scope __device__ variable of kNoAllocScratchBytes
// bytes: every GPU that loads this library holds it until the process exits.
// In host code its name is only a host-side stand-in, so its device address
// is looked up once per device with cudaGetSymbolAddress (on the first call
// on that device, with that device current) and passed to the kernels.
#include <mutex>
#include <string>

#include "device.cuh"
#include "kifmm.h"
#include "plan_impl.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

fmm_status fail(fmm_status s, const std::string &m) { return kifmm::plan_set_error(s, m); }

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

} // namespace

extern "C" fmm_status fmm_evaluate_noalloc(fmm_plan_t plan, const float *charges, int nrhs,
                                           double *potentials, void *stream) {
    if (!plan) return fail(FMM_ERR_INVALID_ARG, "plan is NULL");
    if (kifmm::plan_host_only(plan))
        return fail(FMM_ERR_INVALID_ARG, "host-only plan cannot evaluate");
    if (!charges || !potentials) return fail(FMM_ERR_INVALID_ARG, "NULL charges or potentials");
    if (nrhs < 1) return fail(FMM_ERR_INVALID_ARG, "nrhs must be >= 1");
    const int dev = kifmm::plan_device(plan);
    if (dev < 0 || dev >= kMaxDevices) return fail(FMM_ERR_UNSUPPORTED, "device ordinal too large");
    kifmm::DeviceGuard guard;  // the caller's device is current again on return
    cudaError_t e = guard.set(dev);
    if (e != cudaSuccess) return fail(FMM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    if (fmm_status err = kifmm::plan_check_device_error(plan)) return err;
    if (!is_device_pointer(charges) || !is_device_pointer(potentials))
        return fail(FMM_ERR_INVALID_ARG,
                    "fmm_evaluate_noalloc needs device pointers (host buffers would need staging)");

    kifmm::WorkspaceBytes wb;
    kifmm::plan_workspace_bytes(plan, nrhs, &wb);
    const size_t sizes[12] = {wb.qs, wb.up,  wb.down, wb.qhat, wb.chat, wb.xchk,
                              wb.qh, wb.qh,  wb.chk,  wb.ybuf, wb.yp,  wb.part};
    size_t total = 0;
    for (size_t s : sizes) total += align256(s);
    if (total > kNoAllocScratchBytes)
        return fail(FMM_ERR_INVALID_ARG,
                    "workspace of " + std::to_string(total) + " bytes for nrhs=" +
                        std::to_string(nrhs) + " exceeds the fixed scratch of " +
                        std::to_string(kNoAllocScratchBytes) + " bytes; use fmm_evaluate");

    void *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        // a reset of the device's primary context (cudaDeviceReset) frees the
        // array's old address: look it up again when the kept one is no
        // longer device memory of this context
        if (g_scratch_ptr[dev] && !is_device_pointer(g_scratch_ptr[dev])) g_scratch_ptr[dev] = nullptr;
        if (!g_scratch_ptr[dev]) {
            e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_scratch);
            if (e != cudaSuccess) {
                g_scratch_ptr[dev] = nullptr;
                return fail(FMM_ERR_CUDA,
                            std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        base = g_scratch_ptr[dev];
    }
    // Carve the buffers out of the array.  Every kernel writes each value it
    // later reads within the same call, so nothing has to start at zero and
    // the previous call's contents are harmless.
    unsigned char *p = static_cast<unsigned char *>(base);
    float *parts[12];
    for (int i = 0; i < 12; ++i) {
        parts[i] = reinterpret_cast<float *>(p);
        p += align256(sizes[i]);
    }
    kifmm::WorkBuffers b;
    b.qs = parts[0];
    b.up = parts[1];
    b.down = parts[2];
    b.qhat = parts[3];
    b.chat = parts[4];
    b.xchk = parts[5];
    b.qh_hi = wb.qh ? parts[6] : nullptr;
    b.qh_lo = wb.qh ? parts[7] : nullptr;
    b.chk = parts[8];
    b.ybuf = parts[9];
    b.yp = parts[10];
    b.part = wb.part ? parts[11] : nullptr;
    fmm_status s = kifmm::plan_enqueue(plan, charges, nrhs, potentials, nullptr, b,
                                       static_cast<cudaStream_t>(stream));
    return s;  // on failure plan_enqueue has set the message fmm_last_error() returns
}
