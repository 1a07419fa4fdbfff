// Tensor-core (tcgen05) bf16 screen of the candidate Gram matrices.
#include "kernels.h"

namespace trstmi {

bool screen_supported(int, int) { return false; }
cudaError_t init_screen_attributes(int) { return cudaSuccess; }

cudaError_t launch_screen_bf16(int, int, uint64_t, const float2*, int, uint32_t, uint32_t, double,
                               const DevState*, unsigned int*, uint32_t*, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace trstmi
