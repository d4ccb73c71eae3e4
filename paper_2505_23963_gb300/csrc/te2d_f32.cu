// te2d_f32.cu -- the FP32 TE-form step kernel (te2d.cuh): the z-chunks without bath modes, and
// those with at most 8 modes per material.
#include <cuda_runtime.h>

#include "te2d.cuh"

namespace fdtdbath {

int launch_te2d_f32(const Step3DParams<float>& p, int nchunks, int nb, void* stream) {
  if (nb == 0) {
    dim3 grid((unsigned)(p.nx / (32 * 4 * te2d::WARPS)), (unsigned)nchunks), block(32 * te2d::WARPS);
    te2d_kernel<float, 4, 0><<<grid, block, 0, (cudaStream_t)stream>>>(p);
  } else if (nb <= 8) {
    dim3 grid((unsigned)(p.nx / (32 * te2d::WARPS)), (unsigned)nchunks), block(32 * te2d::WARPS);
    te2d_kernel<float, 1, 8><<<grid, block, 0, (cudaStream_t)stream>>>(p);
  } else {
    return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_te2d_fused_f32(const Step3DParams<float>& p, int nplain, int nbath, int nb, void* stream) {
  if (nb > 8) return (int)cudaErrorInvalidValue;
  const unsigned nblk = (unsigned)(nbath * (p.nx / (32 * te2d::WARPS)) + nplain * (p.nx / (128 * te2d::WARPS)));
  te2d_fused_kernel<float, 8><<<nblk, 32 * te2d::WARPS, 0, (cudaStream_t)stream>>>(p, nplain, nbath);
  return (int)cudaGetLastError();
}

}  // namespace fdtdbath
