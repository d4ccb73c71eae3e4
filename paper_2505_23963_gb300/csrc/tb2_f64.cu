// tb2_f64.cu -- double instantiation of the two-steps-per-pass kernel (built without contraction,
// so its fields agree bit for bit with two single steps of the other FP64 kernels).
#include "tb2.cuh"

namespace fdtdbath {

int launch_tb2_f64(const Tb2Params<double>& q, int nchunks, void* stream) { return tb2_launch<double>(q, nchunks, stream); }

}  // namespace fdtdbath
