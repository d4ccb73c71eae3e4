// plain3d_f32.cu -- float instantiations of the plain-plane step kernel: four cells per thread for
// the chunks without bath planes, one cell per thread (bath state in registers, at most 4 or 8
// modes per material; two threads per cell with 16; up to 128 streamed through a shared-memory
// ring) for the Lorentz-Bath chunks; two planes staged ahead.
#include <cuda_runtime.h>

#include "plain3d.cuh"

namespace fdtdbath {

template <int VX, int A, int NB = 0, bool YB = false>
static int launch_shape(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur, int ebuf,
                        int hbuf, int nchunks, void* stream) {
  using L = Plain3DLayout<float, VX, A, NB>;
  auto kern = plain3d_kernel<float, true, VX, A, NB, YB>;
  static bool attr_set = false;   // once per process: more than 48 KB, shared-memory carveout
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  dim3 grid(p.nx / L::TX, p.ny / L::TY, nchunks), block(L::threads);
  kern<<<grid, block, L::bytes, (cudaStream_t)stream>>>(p, maps, bmaps, pcur, ebuf, hbuf);
  return (int)cudaGetLastError();
}

int launch_plain3d_f32(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                       void* stream) {
  static const BathMaps none{};   // no bath planes in these chunks
  return launch_shape<4, 2>(p, maps, none, 0, ebuf, hbuf, nchunks, stream);
}

int launch_bath3d_f32(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur, int ebuf,
                      int hbuf, int nchunks, int nb, int ybf, void* stream) {
  if (ybf) {
    if (nb <= 8) return launch_shape<1, 2, 8, true>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
    if (nb <= 16) return launch_shape<1, 2, 16, true>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
    return (int)cudaErrorInvalidValue;
  }
  if (nb <= 4) return launch_shape<1, 2, 4>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  if (nb <= 8) return launch_shape<1, 2, 8>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  if (nb <= 16) return launch_shape<1, 2, 16>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  if (nb <= 128) return launch_shape<1, 2, 128>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  return (int)cudaErrorInvalidValue;
}

}  // namespace fdtdbath
