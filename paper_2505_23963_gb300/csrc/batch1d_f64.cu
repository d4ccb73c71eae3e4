// batch1d_f64.cu -- FP64 instantiation of the batched 1D kernel (the updates exactly as the
// paper writes them, D stored; built without FMA contraction), the fixed-order reduction of its
// energy records into per-cavity traces and the step-counter advance.
#include "batch1d.cuh"

namespace fdtdbath {

int batch1d_occupancy_f32(int cluster, int threads, int smem, int* max_clusters, int* static_smem);

int launch_batch1d_f64(const BatchParams<double>& p, int nctas, int cluster, int threads, int smem,
                       void* stream) {
  return launch_batch1d_impl<double, false>(p, nctas, cluster, threads, smem, stream);
}

int batch1d_occupancy(int prec, int cluster, int threads, int smem, int* max_clusters,
                      int* static_smem) {
  if (prec == 32) return batch1d_occupancy_f32(cluster, threads, smem, max_clusters, static_smem);
  return batch1d_occupancy_impl<double, false>(cluster, threads, smem, max_clusters, static_smem);
}

// One block per cavity: every recorded step of the launch sums the cavity's record slots in
// CTA order and writes the trace entry (U_EM, U_P, U_bath, 0), U = dx/2 * sum.
__global__ void batch_reduce_kernel(const BatchReduceParams r) {
  const int cav = blockIdx.x;
  const int64_t step0 = *r.ctr;
  const int k0 = r.slot_ptr[cav], k1 = r.slot_ptr[cav + 1];
  for (int64_t s = step0 + threadIdx.x; s < step0 + r.nsteps; s += blockDim.x) {
    if (s % r.every) continue;
    const int64_t t = s / r.every;
    if (t >= r.trace_cap) continue;
    const double* rec = r.partial + (t % r.ring_cap) * r.ring_stride;
    double u[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = k0; k < k1; ++k) {
      const double* q = rec + 4 * (int64_t)r.slot_idx[k];
      u[0] += q[0];
      u[1] += q[1];
      u[2] += q[2];
      u[3] += q[3];
    }
    double* out = r.trace + ((int64_t)cav * r.trace_cap + t) * 4;
    out[0] = 0.5 * r.ew * (u[0] + u[3]);
    out[1] = 0.5 * r.ew * u[1];
    out[2] = 0.5 * r.ew * u[2];
    out[3] = 0.0;
  }
}

__global__ void batch_advance_kernel(long long* ctr, int nsteps) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *ctr += nsteps;
}

int launch_batch_reduce(const BatchReduceParams& r, void* stream) {
  if (r.ncav <= 0 || r.nsteps <= 0) return 0;
  batch_reduce_kernel<<<r.ncav, 128, 0, (cudaStream_t)stream>>>(r);
  return (int)cudaGetLastError();
}

int launch_batch_advance(long long* ctr, int nsteps, void* stream) {
  batch_advance_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(ctr, nsteps);
  return (int)cudaGetLastError();
}

}  // namespace fdtdbath
