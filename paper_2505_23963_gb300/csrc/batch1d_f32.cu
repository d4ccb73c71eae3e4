// batch1d_f32.cu -- FP32 instantiation of the batched 1D kernel (increment arithmetic on the
// two stored levels of P and of every bath mode).
#include "batch1d.cuh"

namespace fdtdbath {

int launch_batch1d_f32(const BatchParams<float>& p, int nctas, int cluster, int threads, int smem,
                       void* stream) {
  return launch_batch1d_impl<float, true>(p, nctas, cluster, threads, smem, stream);
}

int batch1d_occupancy_f32(int cluster, int threads, int smem, int* max_clusters, int* static_smem) {
  return batch1d_occupancy_impl<float, true>(cluster, threads, smem, max_clusters, static_smem);
}

}  // namespace fdtdbath
