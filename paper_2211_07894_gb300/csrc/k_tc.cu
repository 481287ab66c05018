// Tensor-core (tcgen05) forms of the two contractions.
#include "lrdm_internal.h"

namespace lrdm {

bool tc_supported() { return false; }

cudaError_t launch_gemm1_tc(int, const Channel&, const SysState&, int, int, const float*, void*,
                            int*, cudaStream_t) {
  return cudaErrorNotSupported;
}

cudaError_t launch_gemm2_tc(int, const Channel&, const SysState&, int, double, const void*,
                            long long, void*, long long, int, int, int*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace lrdm
