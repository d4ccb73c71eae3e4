// te2d_f32.cu -- the FP32 TE-form step kernel for the z-chunks without bath modes (te2d.cuh).
#include <cuda_runtime.h>

#include "te2d.cuh"

namespace fdtdbath {

int launch_te2d_f32(const Step3DParams<float>& p, int nchunks, void* stream) {
  dim3 grid((unsigned)(p.nx / (te2d::SEG * te2d::WARPS)), (unsigned)nchunks), block(32 * te2d::WARPS);
  te2d_kernel<float><<<grid, block, 0, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

}  // namespace fdtdbath
