// Split-precision chi0 on tcgen05 tensor cores (placeholder until the kernel
// lands: reports "not supported" so that callers fail loudly).
#include <cuda_runtime.h>

#include "rpa_internal.h"

namespace rpa {

bool mixed_supported() { return false; }

size_t mixed_workspace_bytes(const BatchGeom&, int) { return 0; }

cudaError_t launch_chi0_mixed(const BatchGeom&, int, const double* const*, const double*, double*, void*, size_t,
                              uint64_t*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace rpa
