// plain3d_f64.cu -- double instantiations of the plain-plane step kernel (two cells per thread, two
// planes staged ahead; built without FMA contraction), without and with a per-cell sigma(r) map.
#include <cuda_runtime.h>

#include "plain3d.cuh"

namespace fdtdbath {

template <int VX, int A, bool SIG>
static int launch_shape(const Step3DParams<double>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                        void* stream) {
  using L = Plain3DLayout<double, VX, A>;
  auto kern = plain3d_kernel<double, false, VX, A, 0, false, SIG>;
  static bool attr_set = false;   // once per process: more than 48 KB, shared-memory carveout
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  dim3 grid(p.nx / L::TX, p.ny / L::TY, nchunks), block(L::threads);
  static const BathMaps none{};   // no bath planes in these chunks
  kern<<<grid, block, L::bytes, (cudaStream_t)stream>>>(p, maps, none, 0, ebuf, hbuf);
  return (int)cudaGetLastError();
}

int launch_plain3d_f64(const Step3DParams<double>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                       void* stream) {
  // with a per-cell sigma(r) map: the instantiation that reads it
  if (p.sig) return launch_shape<2, 2, true>(p, maps, ebuf, hbuf, nchunks, stream);
  return launch_shape<2, 2, false>(p, maps, ebuf, hbuf, nchunks, stream);
}

}  // namespace fdtdbath
