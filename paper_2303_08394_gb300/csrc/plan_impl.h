// Internal entry points shared by the C-ABI translation units.
#pragma once
#include <cstddef>
#include <string>
#include <cuda_runtime.h>

#include "kifmm.h"

namespace kifmm {

// Per-evaluation device buffers (see DevWork for their layouts).
struct WorkBuffers {
    float *qs = nullptr, *up = nullptr, *down = nullptr, *qhat = nullptr, *chat = nullptr,
          *xchk = nullptr;
    float *qh_hi = nullptr, *qh_lo = nullptr;  // tensor-core M2L operand splits
    float *chk = nullptr, *ybuf = nullptr, *yp = nullptr;  // level-product temporaries
    float *part = nullptr;  // split-K partial products (may be null: no split)
};

// Byte sizes of those buffers for one plan and nrhs.
struct WorkspaceBytes {
    size_t qs = 0, up = 0, down = 0, qhat = 0, chat = 0, xchk = 0;
    size_t qh = 0;  // each of the two operand splits (0 for the FP32 M2L)
    size_t chk = 0, ybuf = 0, yp = 0;
    size_t part = 0;  // split-K scratch of the M2M level products
};

void plan_workspace_bytes(const fmm_plan_s *P, int nrhs, WorkspaceBytes *out);
// grad (rows x nrhs x 3, may be null): also write the gradient of the
// potential at every target; pot may then be null.
fmm_status plan_enqueue(fmm_plan_s *P, const float *charges, int nrhs, double *pot,
                        double *grad, const WorkBuffers &b, cudaStream_t st);
int plan_device(const fmm_plan_s *P);
int plan_m2l_mode(const fmm_plan_s *P);
// FMM_ERR_TIMEOUT (once) if a device-side bounded wait expired, else FMM_OK.
fmm_status plan_check_device_error(fmm_plan_s *P);
// Record the message fmm_last_error() returns on this thread; returns s.
fmm_status plan_set_error(fmm_status s, const std::string &msg);
bool plan_host_only(const fmm_plan_s *P);

// Makes a plan's device current for the guard's lifetime and then makes the
// caller's device current again, so no entry point leaves it switched.
struct DeviceGuard {
    int prev = -1;
    cudaError_t set(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        return prev == device ? cudaSuccess : cudaSetDevice(device);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

} // namespace kifmm
