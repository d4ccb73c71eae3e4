// tb2_f32.cu -- float instantiation of the two-steps-per-pass kernel.
#include "tb2.cuh"

namespace fdtdbath {

int launch_tb2_f32(const Tb2Params<float>& q, int nchunks, void* stream) { return tb2_launch<float>(q, nchunks, stream); }

}  // namespace fdtdbath
