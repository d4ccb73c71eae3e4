// step3d_f32.cu -- float instantiations of the fused 3D step kernel (bath modes stored in FP32,
// or as bf16 value / increment pairs).
#include <cuda_runtime.h>

#include "step3d.cuh"

namespace fdtdbath {

template <int NB, int TY, bool YB, bool TE>
static int launch_nb(const Step3DParams<float>& p, int nbx, int nby, int nchunks, void* stream) {
  // the TE form runs 128-wide single-row tiles, every other form 32-wide tiles
  constexpr int TX = TE ? 4 * kTX : kTX;
  auto kern = step3d_kernel<float, true, NB, TY, YB, TE, TX>;
  const size_t smem = step3d_smem_bytes(TY, p.nmodes, sizeof(float), TX, TE);
  static size_t smem_set = 0;   // opt in once per instantiation for more than 48 KB
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    smem_set = smem;
  }
  dim3 grid(TX == kTX ? nbx : (p.nx + TX - 1) / TX, nby, nchunks), block(TX, TY);
  kern<<<grid, block, smem, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

template <int TY, bool YB, bool TE>
static int launch_ty(const Step3DParams<float>& p, int nbmax, int nbx, int nby, int nchunks, void* stream) {
  switch (nbmax) {
    case 0: return launch_nb<0, TY, false, TE>(p, nbx, nby, nchunks, stream);
    case 4: return launch_nb<4, TY, YB, TE>(p, nbx, nby, nchunks, stream);
    case 8: return launch_nb<8, TY, YB, TE>(p, nbx, nby, nchunks, stream);
    case 16: return launch_nb<16, TY, YB, TE>(p, nbx, nby, nchunks, stream);
    case 32: return launch_nb<32, TY, YB, TE>(p, nbx, nby, nchunks, stream);
    case 128: return launch_nb<128, TY, YB, TE>(p, nbx, nby, nchunks, stream);
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_step3d_f32(const Step3DParams<float>& p, int nbmax, int ty, int nbx, int nby, int nchunks,
                      int bath_bf16, int te, void* stream) {
  // te: the y-invariant TE form (ny = 1, single-row tiles only)
  if (bath_bf16) {
    if (ty == 8) return launch_ty<8, true, false>(p, nbmax, nbx, nby, nchunks, stream);
    if (ty == 1) return te ? launch_ty<1, true, true>(p, nbmax, nbx, nby, nchunks, stream)
                           : launch_ty<1, true, false>(p, nbmax, nbx, nby, nchunks, stream);
  } else {
    if (ty == 8) return launch_ty<8, false, false>(p, nbmax, nbx, nby, nchunks, stream);
    if (ty == 1) return te ? launch_ty<1, false, true>(p, nbmax, nbx, nby, nchunks, stream)
                           : launch_ty<1, false, false>(p, nbmax, nbx, nby, nchunks, stream);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace fdtdbath
