// Shared host/device helpers of the mpmrom library: status handling, error
// strings, small device utilities.  Everything here is implementation detail
// behind the C ABI declared in include/mpmrom.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/mpmrom.h"

namespace mpmrom {

// Records a message for mpm_last_error() and returns the status.
mpm_status set_error(mpm_status st, const std::string& msg);

#define MPM_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess)                                                              \
      return ::mpmrom::set_error(MPM_ECUDA, std::string(#expr) + ": " +                 \
                                                cudaGetErrorString(_e));                \
  } while (0)

#define MPM_CHECK_ARG(cond, msg)                                                        \
  do {                                                                                  \
    if (!(cond)) return ::mpmrom::set_error(MPM_EINVAL, msg);                           \
  } while (0)

// Device status word bits (OR-ed by kernels, read by mpm_sync_status and friends).
enum : uint32_t {
  STATUS_NONFINITE = 1u << 0,     // NaN / Inf in a particle quantity
  STATUS_INVERTED = 1u << 1,      // det F <= 0
  STATUS_OUT_OF_GRID = 1u << 2,   // a stencil left the grid (particle clamped, not scattered)
  STATUS_GN_NO_DECREASE = 1u << 3,// Gauss-Newton line search found no decrease
  STATUS_CHOLESKY = 1u << 4,      // normal equations not positive definite
  STATUS_TIMEOUT = 1u << 5,       // a bounded wait ran out
  STATUS_CAPACITY = 1u << 6,      // a fixed-capacity list overflowed
};

__device__ __forceinline__ void raise_status(uint32_t* status, uint32_t bits) {
  if (status) atomicOr(status, bits);
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace mpmrom
