// plain3d_f32.cu -- float instantiation of the plain-plane step kernel (four cells per thread, two
// planes staged ahead, two CTAs per SM).
#include <cuda_runtime.h>

#include "plain3d.cuh"

namespace fdtdbath {

template <int VX, int A>
static int launch_shape(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                        void* stream) {
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
  dim3 grid(p.nx / L::TX, p.ny / L::TY, nchunks), block(L::threads);
  kern<<<grid, block, L::bytes, (cudaStream_t)stream>>>(p, maps, ebuf, hbuf);
  return (int)cudaGetLastError();
}

int launch_plain3d_f32(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                       void* stream) {
  return launch_shape<4, 2>(p, maps, ebuf, hbuf, nchunks, stream);
}

}  // namespace fdtdbath
