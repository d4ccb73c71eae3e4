// cavity1d_f64.cu -- double instantiations of the persistent 1D cavity kernel.
#include <cuda_runtime.h>

#include "cavity1d.cuh"

namespace fdtdbath {

template <int NB>
static int launch_nb(const Cav1DParams<double>& p, int cluster, void* stream) {
  auto kern = cavity1d_kernel<double, false, NB>;
  if (cluster > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(kCav1DThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, kern, p);
}

int launch_cavity1d_f64(const Cav1DParams<double>& p, int nbmax, int cluster, void* stream) {
  if (cluster < 1 || cluster > kCav1DMaxCluster) return (int)cudaErrorInvalidValue;
  switch (nbmax) {
    case 0: return launch_nb<0>(p, cluster, stream);
    case 4: return launch_nb<4>(p, cluster, stream);
    case 8: return launch_nb<8>(p, cluster, stream);
    case 16: return launch_nb<16>(p, cluster, stream);
    case 32: return launch_nb<32>(p, cluster, stream);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace fdtdbath
