// plain3d_launch.cuh -- the launch of one FP32 instantiation of the plain-plane step kernel (the
// shared-memory opt-in once per instantiation, the grid of its tiles), for the translation units
// that instantiate it with and without the per-cell sigma(r).
#pragma once

#include <cuda_runtime.h>

#include "plain3d.cuh"

namespace fdtdbath {

template <int VX, int A, int NB, bool YB, bool SIG>
int plain3d_launch_f32(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur,
                       int ebuf, int hbuf, int nchunks, void* stream) {
  using L = Plain3DLayout<float, VX, A, NB>;
  auto kern = plain3d_kernel<float, true, VX, A, NB, YB, SIG>;
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

// The bath-free form over the chunks without bath planes, and the Lorentz-Bath form for nb modes
// per material (ybf: bf16 bath storage) over those with them.
template <bool SIG>
int plain3d_plain_f32(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                      void* stream) {
  static const BathMaps none{};   // no bath planes in these chunks
  return plain3d_launch_f32<4, 2, 0, false, SIG>(p, maps, none, 0, ebuf, hbuf, nchunks, stream);
}

template <bool SIG>
int plain3d_bath_f32(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur, int ebuf,
                     int hbuf, int nchunks, int nb, int ybf, void* stream) {
  if (ybf) {
    if (nb <= 8) return plain3d_launch_f32<1, 2, 8, true, SIG>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
    if (nb <= 16) return plain3d_launch_f32<1, 2, 16, true, SIG>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
    return (int)cudaErrorInvalidValue;
  }
  if (nb <= 4) return plain3d_launch_f32<1, 2, 4, false, SIG>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  if (nb <= 8) return plain3d_launch_f32<1, 2, 8, false, SIG>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  if (nb <= 16) return plain3d_launch_f32<1, 2, 16, false, SIG>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  if (nb <= 128) return plain3d_launch_f32<1, 2, 128, false, SIG>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, stream);
  return (int)cudaErrorInvalidValue;
}

}  // namespace fdtdbath
