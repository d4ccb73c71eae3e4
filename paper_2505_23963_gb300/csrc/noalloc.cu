// noalloc.cu -- energy of a z-box of the current state, computed without allocating memory.
//
// Some callers may not allocate device memory at the moment they need a result: a real-time
// or latency-bound loop (an allocation can synchronize the device and take unbounded time), a
// host framework that owns the whole device memory pool and hands this library nothing beyond
// the simulation's own buffers, or a process held to a fixed device-memory budget.
// fdtdbath_box_energy_noalloc serves them: its scratch space is the file-scope device array
// below, not an allocation.  The call may launch the simulation's pending H half-step and waits
// for the simulation's stream.
//
// The array holds one FP64 partial sum per plane and quantity for at most
// kNoAllocMaxPlanes planes (about 96 KB), and every GPU that loads this library keeps it
// until the process exits.  All calls on a device share it and it keeps the last call's
// contents; every slot a call reads is written by that same call first, so nothing needs
// clearing between calls.  Calls that overlap on the GPU (e.g. from two streams) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/fdtdbath.h"
#include "internal.h"

namespace fdtdbath {
namespace {

constexpr int kNoAllocMaxPlanes = 4096;
constexpr int kNoAllocMaxDevices = 64;

// [kNoAllocMaxPlanes][3] per-plane partials, then the 3 final sums.
static __device__ __align__(256) double g_box_energy_scratch[3 * kNoAllocMaxPlanes + 4];

struct BoxEnergyParams {
  int64_t nx, ny, nz, plane, ncell, nmatcell;
  double dt, ew;
  int64_t z_lo, z_hi;
  int inc;
  const void *E, *H, *Pa, *Pb, *Ya, *Yb;
  int nmat;
  SimViewMat mat[kMaxMat];
  double* scratch;  // device address of g_box_energy_scratch
};

// One block per plane of the box: sum over its cells of eps E.E + H.H and of the P and bath
// energy densities (without their common factor 1/2), in FP64, reduced in a fixed order
// into the plane's scratch slots.
template <typename T>
__global__ void box_energy_planes_kernel(const BoxEnergyParams p) {
  __shared__ double sh[3][256];
  const int64_t k = p.z_lo + blockIdx.x;
  int mi = -1;
  for (int m = 0; m < p.nmat; ++m)
    if (k >= p.mat[m].zlo && k < p.mat[m].zhi) mi = m;
  const T* E = (const T*)p.E;
  const T* H = (const T*)p.H;
  const T* Pa = (const T*)p.Pa;
  const T* Pb = (const T*)p.Pb;
  const T* Ya = (const T*)p.Ya;
  const T* Yb = (const T*)p.Yb;
  double em = 0.0, up = 0.0, ub = 0.0;
  const double eps = mi >= 0 ? p.mat[mi].eps : 1.0;
  for (int64_t c0 = threadIdx.x; c0 < p.plane; c0 += blockDim.x) {
    const int64_t q = k * p.plane + c0;
    for (int c = 0; c < 3; ++c) {
      const double e = (double)E[c * p.ncell + q], h = (double)H[c * p.ncell + q];
      em += eps * e * e + h * h;
    }
    if (mi < 0) continue;
    const SimViewMat& M = p.mat[mi];
    if (M.kind == kVacuum || M.rho == 0.0) continue;
    const int64_t rl = (k - M.zlo) * p.plane + c0;
    const int64_t r = M.base + rl;
    for (int c = 0; c < 3; ++c) {
      const double P = (double)Pa[c * p.nmatcell + r];
      const double V = p.inc ? (double)Pb[c * p.nmatcell + r] : P - (double)Pb[c * p.nmatcell + r];
      up += M.rho * ((V / p.dt) * (V / p.dt) + M.w0r2 * P * P);
      for (int j = 0; j < M.nb; ++j) {
        const int64_t o = M.ybase + ((int64_t)c * M.nb + j) * M.ncell + rl;
        const double Y = (double)Ya[o];
        const double Vy = p.inc ? (double)Yb[o] : Y - (double)Yb[o];
        ub += M.rho * ((Vy / p.dt) * (Vy / p.dt) + M.wj2[j] * Y * Y);
      }
    }
  }
  sh[0][threadIdx.x] = em;
  sh[1][threadIdx.x] = up;
  sh[2][threadIdx.x] = ub;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) p.scratch[3 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// Sum the per-plane partials in plane order; (U_EM, U_P, U_bath) land after the partials.
__global__ void box_energy_sum_kernel(double* scratch, int nplanes, double ew) {
  if (threadIdx.x >= 3) return;
  double s = 0.0;
  for (int pl = 0; pl < nplanes; ++pl) s += scratch[3 * pl + threadIdx.x];
  scratch[3 * kNoAllocMaxPlanes + threadIdx.x] = 0.5 * ew * s;
}

// Device address of the scratch array on the current device, looked up once per device and
// cached for the life of the process (an address of the device's primary context: not valid
// after cudaDeviceReset).  The lookup is a host call (cudaGetSymbolAddress): the first call on a
// device should come before any stream capture on it.
double* scratch_address(int device, cudaError_t* err) {
  static std::mutex mu;
  static double* addr[kNoAllocMaxDevices] = {};
  *err = cudaSuccess;
  if (device < 0 || device >= kNoAllocMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* ptr = nullptr;
    *err = cudaGetSymbolAddress(&ptr, g_box_energy_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[device] = (double*)ptr;
  }
  return addr[device];
}

}  // namespace
}  // namespace fdtdbath

using namespace fdtdbath;

extern "C" int fdtdbath_box_energy_noalloc(fdtdbath_sim* sim, int64_t z_lo, int64_t z_hi, double* out,
                                           int32_t out_on_device) {
  if (!sim || !out) return FDTDBATH_ERR_ARG;
  SimView v;
  int rc = fdtdbath_internal_view(sim, &v);
  if (rc) return rc;
  if (z_lo < 0 || z_hi > v.nz || z_hi <= z_lo)
    return fdtdbath_internal_fail(sim, FDTDBATH_ERR_ARG, "box_energy_noalloc: box outside the grid or empty");
  if (z_hi - z_lo > kNoAllocMaxPlanes)
    return fdtdbath_internal_fail(sim, FDTDBATH_ERR_ARG,
                                  "box_energy_noalloc: box deeper than 4096 planes, the size of the static scratch");
  cudaError_t e = cudaSetDevice(v.device);
  double* scratch = e == cudaSuccess ? scratch_address(v.device, &e) : nullptr;
  if (!scratch) {
    std::string m = std::string("box_energy_noalloc: scratch address: ") + cudaGetErrorString(e);
    return fdtdbath_internal_fail(sim, FDTDBATH_ERR_CUDA, m.c_str());
  }
  BoxEnergyParams p{};
  p.nx = v.nx;
  p.ny = v.ny;
  p.nz = v.nz;
  p.plane = v.plane;
  p.ncell = v.ncell;
  p.nmatcell = v.nmatcell;
  p.dt = v.dt;
  p.ew = v.dx / (double)v.plane;
  p.z_lo = z_lo;
  p.z_hi = z_hi;
  p.inc = v.inc;
  p.E = v.E;
  p.H = v.H;
  p.Pa = v.Pa;
  p.Pb = v.Pb;
  p.Ya = v.Ya;
  p.Yb = v.Yb;
  p.nmat = v.nmat;
  for (int m = 0; m < v.nmat; ++m) p.mat[m] = v.mat[m];
  p.scratch = scratch;
  cudaStream_t st = (cudaStream_t)v.stream;
  const int nplanes = (int)(z_hi - z_lo);
  if (v.prec == 64) box_energy_planes_kernel<double><<<nplanes, 256, 0, st>>>(p);
  else box_energy_planes_kernel<float><<<nplanes, 256, 0, st>>>(p);
  box_energy_sum_kernel<<<1, 32, 0, st>>>(scratch, nplanes, p.ew);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + 3 * kNoAllocMaxPlanes, 3 * sizeof(double),
                        out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    std::string m = std::string("box_energy_noalloc: ") + cudaGetErrorString(e);
    return fdtdbath_internal_fail(sim, FDTDBATH_ERR_CUDA, m.c_str());
  }
  return FDTDBATH_OK;
}
