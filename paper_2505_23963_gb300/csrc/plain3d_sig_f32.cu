// plain3d_sig_f32.cu -- the float instantiations of the plain-plane step kernel that read a
// per-cell sigma(r) map (Eq. EOM_Lorentz's sigma(r)); a translation unit of their own so that they
// compile beside the others.
#include <cuda_runtime.h>

#include "plain3d_launch.cuh"

namespace fdtdbath {

int launch_plain3d_sig_f32(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                           void* stream) {
  return plain3d_plain_f32<true>(p, maps, ebuf, hbuf, nchunks, stream);
}

int launch_bath3d_sig_f32(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur,
                          int ebuf, int hbuf, int nchunks, int nb, int ybf, void* stream) {
  return plain3d_bath_f32<true>(p, maps, bmaps, pcur, ebuf, hbuf, nchunks, nb, ybf, stream);
}

}  // namespace fdtdbath
