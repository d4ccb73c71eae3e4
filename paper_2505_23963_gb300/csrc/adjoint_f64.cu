// adjoint_f64.cu -- FP64 instantiation of the reverse step (adjoint.cuh), built without FMA
// contraction like the FP64 forward kernels.
#include "adjoint.cuh"

namespace fdtdbath {

int launch_adjoint_f64(const AdjParams<double>& p, int nbmax, int te, void* stream) {
  return launch_adjoint_impl<double>(p, nbmax, te, stream);
}

}  // namespace fdtdbath
