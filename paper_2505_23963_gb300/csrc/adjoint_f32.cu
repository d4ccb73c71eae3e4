// adjoint_f32.cu -- FP32 instantiation of the reverse step (adjoint.cuh).
#include "adjoint.cuh"

namespace fdtdbath {

int launch_adjoint_f32(const AdjParams<float>& p, int nbmax, int te, void* stream) {
  return launch_adjoint_impl<float>(p, nbmax, te, stream);
}

int64_t adjoint_blocks(int64_t ncell) { return (ncell + kAdjThreads - 1) / kAdjThreads; }

}  // namespace fdtdbath
