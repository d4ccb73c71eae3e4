// plain3d_f64.cu -- double instantiation of the plain-plane step kernel (built without FMA
// contraction).
#include <cuda_runtime.h>

#include "plain3d.cuh"

namespace fdtdbath {

int launch_plain3d_f64(const Step3DParams<double>& p, int nchunks, int, void* stream) {
  using L = Plain3DLayout<double, 2, 2>;
  auto kern = plain3d_kernel<double, false, 2, 2>;
  static bool attr_set = false;   // once per process: more than 48 KB, shared-memory carveout
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  dim3 grid((p.nx + L::TX - 1) / L::TX, (p.ny + L::TY - 1) / L::TY, nchunks), block(L::threads);
  kern<<<grid, block, L::bytes, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

}  // namespace fdtdbath
