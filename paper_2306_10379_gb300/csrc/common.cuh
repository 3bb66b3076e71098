// Shared helpers of the gsi CUDA library: status plumbing and launch checks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/gsi.h"

namespace gsi {

void set_last_error(const char* msg);
gsi_status cuda_status(cudaError_t e);

inline gsi_status cuda_status_ok(cudaError_t e) {
  return e == cudaSuccess ? GSI_OK : cuda_status(e);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per process).
int sm_count();

// Count of kernels launched by this library in this process.
void note_launch();

// cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
// only when the limit set for this kernel on the current device is below
// bytes: the call costs microseconds of host time, which fall on the
// critical path after every readback of the iteration.
cudaError_t ensure_dyn_smem(const void* f, int bytes);

}  // namespace gsi

#define GSI_CUDA_TRY(expr)                                         \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return gsi::cuda_status(_e);            \
  } while (0)

#define GSI_LAUNCH_CHECK()  \
  do {                      \
    gsi::note_launch();     \
    GSI_CUDA_TRY(cudaGetLastError()); \
  } while (0)

#define GSI_TRY(expr)                                              \
  do {                                                             \
    gsi_status _s = (expr);                                        \
    if (_s != GSI_OK) return _s;                                   \
  } while (0)
