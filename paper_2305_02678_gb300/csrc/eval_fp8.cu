// FP8 tensor-core evaluation: the instantiations of the kernel in
// eval_tc.cuh whose hidden -> hidden layers run on E4M3 operands (the rest
// of the path as in FP16).  A translation unit of its own so that the build
// compiles the two sets in parallel.
#include "eval_tc.cuh"

namespace nam {

int launch_eval_fp8(const LaunchCommon& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!f16_supported(L.shape)) return (int)cudaErrorInvalidValue;
  if (L.shape.NH == 3) return f16_frame<64, 3, true>(L, s);
  if (L.shape.H == 16) return f16_frame<16, 2, true>(L, s);
  if (L.shape.H == 32) return f16_frame<32, 2, true>(L, s);
  return f16_frame<64, 2, true>(L, s);
}

}  // namespace nam
