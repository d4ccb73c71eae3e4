// plain3d_f32.cu -- float instantiations of the plain-plane step kernel.
#include <cuda_runtime.h>

#include "plain3d.cuh"

namespace fdtdbath {

template <int VX, int A>
static int launch_shape(const Step3DParams<float>& p, int nchunks, void* stream) {
  using L = Plain3DLayout<float, VX, A>;
  auto kern = plain3d_kernel<float, true, VX, A>;
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

// shape: 0 = four cells per thread, one plane ahead; 1 = four cells, two planes ahead;
// 2 = two cells, two planes ahead; 3 = two cells, three planes ahead
int launch_plain3d_f32(const Step3DParams<float>& p, int nchunks, int shape, void* stream) {
  switch (shape) {
    case 1: return launch_shape<4, 2>(p, nchunks, stream);
    case 2: return launch_shape<2, 2>(p, nchunks, stream);
    case 3: return launch_shape<2, 3>(p, nchunks, stream);
    default: return launch_shape<4, 1>(p, nchunks, stream);
  }
}

}  // namespace fdtdbath
