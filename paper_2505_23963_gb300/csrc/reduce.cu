// reduce.cu -- deterministic reductions behind the monitors and energy traces.
//
// The step kernels leave one FP64 partial sum per block and quantity in a ring buffer
// (one ring entry per step).  reduce_series_kernel sums the blocks of each entry in a
// fixed order (strided per-thread sums, then a fixed shared-memory tree), so results do
// not depend on scheduling.  dft_kernel then advances the running DFT
//     F(nu) += f(t_n) exp(+i 2 pi nu t_n) dt
// of the plane means in FP64 (E at t = (n+1/2) dt, H = mean of planes z-1, z at
// t = (n+1) dt), step by step in order, and writes the energy trace entries.
#include <cuda_runtime.h>

#include "internal.h"

namespace fdtdbath {

__global__ void reduce_series_kernel(const ReduceParams r) {
  __shared__ double sh[256];
  const int64_t s = r.step_lo + blockIdx.x;
  const int q = blockIdx.y;
  const int ring = (int)(s % r.ring_cap);
  const double* base = r.partial + (int64_t)ring * r.ring_stride;
  const int nmE = 2 * r.nmon, nmH = 4 * r.nmon;
  const double* src;
  int count;
  if (q < nmE) {
    src = base + r.mon_E_off + (int64_t)q * r.nbxy;
    count = r.nbxy;
  } else if (q < nmE + nmH) {
    src = base + r.mon_H_off + (int64_t)(q - nmE) * r.nbxy;
    count = r.nbxy;
  } else if (q < nmE + nmH + 3) {
    if (!r.energy_on) return;
    src = base + r.en_E_off + (int64_t)(q - nmE - nmH) * r.nblocks;
    count = r.nblocks;
  } else {
    if (!r.energy_on) return;
    src = base + r.en_H_off;
    count = r.nblocks;
  }
  double v = 0.0;
  for (int b = threadIdx.x; b < count; b += blockDim.x) v += src[b];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) r.series[(int64_t)ring * (nmE + nmH + 4) + q] = sh[0];
}

int launch_reduce_series(const ReduceParams& r, void* stream) {
  const int64_t n = r.step_hi - r.step_lo;
  if (n <= 0) return 0;
  dim3 grid((unsigned)n, 6 * r.nmon + 4);
  reduce_series_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(r);
  return (int)cudaGetLastError();
}

__global__ void dft_kernel(const DftParams d, double inv_plane, double ew) {
  const int m = blockIdx.y;
  const int stride = d.series_stride;
  if (m < d.nmon) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < d.nfreq[m]) {
      const double nu = d.freqs[m][f];
      double* acc = d.acc[m] + (int64_t)f * 8;
      double a[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) a[c] = acc[c];
      const int nmE = 2 * d.nmon;
      for (int64_t s = d.step_lo; s < d.step_hi; ++s) {
        const double* row = d.series + (int64_t)(s % d.ring_cap) * stride;
        const double ex = row[2 * m] * inv_plane;
        const double ey = row[2 * m + 1] * inv_plane;
        const double hx = 0.5 * (row[nmE + 4 * m] + row[nmE + 4 * m + 1]) * inv_plane;
        const double hy = 0.5 * (row[nmE + 4 * m + 2] + row[nmE + 4 * m + 3]) * inv_plane;
        const double tE = ((double)s + 0.5) * d.dt, tH = ((double)s + 1.0) * d.dt;
        double sE, cE, sH, cH;
        sincos(2.0 * 3.14159265358979323846 * nu * tE, &sE, &cE);
        sincos(2.0 * 3.14159265358979323846 * nu * tH, &sH, &cH);
        a[0] += ex * cE * d.dt;
        a[1] += ex * sE * d.dt;
        a[2] += ey * cE * d.dt;
        a[3] += ey * sE * d.dt;
        a[4] += hx * cH * d.dt;
        a[5] += hx * sH * d.dt;
        a[6] += hy * cH * d.dt;
        a[7] += hy * sH * d.dt;
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = a[c];
    }
  } else if (d.energy_on && blockIdx.x == 0) {
    // energy trace entries: recorded step s (s % every == 0) goes to trace[s / every]
    const int nm = 6 * d.nmon;
    for (int64_t s = d.step_lo + threadIdx.x; s < d.step_hi; s += blockDim.x) {
      if (s % d.every) continue;
      const int64_t t = s / d.every;
      if (t >= d.trace_cap) continue;
      const double* row = d.series + (int64_t)(s % d.ring_cap) * stride;
      double* out = d.trace + 4 * t;
      out[0] = 0.5 * ew * (row[nm + 0] + row[nm + 3]);
      out[1] = 0.5 * ew * row[nm + 1];
      out[2] = 0.5 * ew * row[nm + 2];
      out[3] = 0.0;
    }
  }
}

int launch_dft_accumulate(const DftParams& d, void* stream) {
  if (d.step_hi <= d.step_lo) return 0;
  int maxf = 1;
  for (int m = 0; m < d.nmon; ++m) maxf = d.nfreq[m] > maxf ? d.nfreq[m] : maxf;
  dim3 grid((maxf + 127) / 128, d.nmon + 1);
  dft_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(d, d.inv_plane, d.ew);
  return (int)cudaGetLastError();
}

}  // namespace fdtdbath
