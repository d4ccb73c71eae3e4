// plain3d_f32.cu -- float instantiations of the plain-plane step kernel: four cells per thread for
// the chunks without bath planes, one cell per thread (bath state in registers, at most 4 or 8
// modes per material; two threads per cell with 16; up to 128 streamed through a shared-memory
// ring) for the Lorentz-Bath chunks; two planes staged ahead.  With a per-cell sigma(r) map the
// launches go to the instantiations of plain3d_sig_f32.cu.
#include <cuda_runtime.h>

#include "plain3d_launch.cuh"

namespace fdtdbath {

int launch_plain3d_f32(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                       void* stream) {
  if (p.sig) return launch_plain3d_sig_f32(p, maps, ebuf, hbuf, nchunks, stream);
  return plain3d_plain_f32<false>(p, maps, ebuf, hbuf, nchunks, stream);
}

int launch_bath3d_f32(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur, int ebuf,
                      int hbuf, int nchunks, int nb, int ybf, void* stream) {
  if (p.sig) return launch_bath3d_sig_f32(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, nb, ybf, stream);
  return plain3d_bath_f32<false>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, nb, ybf, stream);
}

}  // namespace fdtdbath
