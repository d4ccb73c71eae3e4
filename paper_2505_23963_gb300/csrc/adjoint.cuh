// adjoint.cuh -- one reverse step of the discrete adjoint of the FDTD-Bath step.
//
// The forward step (Eq. FDTD-1D generalised to the 3D Yee grid, Eq. Pz_update-LB,
// Yzj_finite_difference, with the CPML of the d/dz terms) is, in exact arithmetic, the linear map
//   F1  psi_E <- b_E psi_E + c_E dz H                         (CPML planes)
//   F2  E <- E + (S [curl H with psi_E] + dt J - (P - P_m)) / eps_inf
//   F3  P_new = (1/A)[cE E - c1m P - c2 P_m - dt/2 sum_j k_j (a_j Y_j + b_j Y_m,j)]
//       Y_new,j = a_j Y_j + (b_j + 1) Y_m,j + c_j (P_new - P_m);  then P_m <- P, P <- P_new, likewise Y
//   F5  psi_H <- b_H psi_H + c_H dz E
//   F6  H <- H - S [curl E with psi_H]
// followed by the monitor observations (plane means of E after F2, of H after F6).  The D-free
// form of F2 is the same map as the stored-D form because D = eps_inf E + P_m holds at every
// step.  The adjoint step applies the transposes in reverse order to the adjoint state; every
// transpose of an update x <- alpha x + M y is  y_bar += M^T x_bar,  x_bar <- alpha x_bar.
//
//   kernel 1 (per cell):  F6^T (curl^T of H_bar into E_bar, H_bar into psi_H_bar), F5^T, F3^T
//            (P / bath adjoints, cE/A P_bar into E_bar, and the parameter gradient), the
//            E-monitor source, and the pointwise parts of F2^T (P_bar, P_m_bar, psi_E_bar).
//   kernel 2 (per cell):  the curl^T part of F2^T (E_bar / eps_inf into H_bar), F1^T, and the
//            H-monitor source.
// The H-monitor source of the step enters kernel 1 through its reads of H_bar (added on the fly)
// and kernel 2 through its update of H_bar.  CPML adjoint memories are double-buffered: a cell
// reads its neighbour's value of the previous buffer and writes the b-scaled value to the other.
//
// Parameter gradient of the differentiated material, with P_bar_new the total adjoint of P_new:
//   dL/dsigma  += P_bar_new (w0 dt)^2 E / A
//   dL/dgamma0 += P_bar_new (dt/2) (P_m - P_new) / A
//   dL/dk_j    += P_bar_new (dt/2)/A [dS/dk_j (P_m - P_new) - (a_j Y_j + b_j Y_m,j)] + Y_bar_new,j dc_j/dk_j (P_new - P_m)
// with S = sum_j k_j c_j, dS/dk_j = k_j dt/(1 + gamma_j dt/2), dc_j/dk_j = dt/(2 (1 + gamma_j dt/2)).
// These terms are summed in the state precision within a thread and a warp (FP64 arithmetic is
// slow on this part), then in FP64 across warps, blocks and steps.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace fdtdbath {

constexpr int kAdjThreads = 256;

__device__ __forceinline__ int adj_psiE_plane(int k, int nz, int npml) {
  if (k < npml) return k;
  if (k >= nz - npml) return npml + (k - (nz - npml));
  return -1;
}
__device__ __forceinline__ int adj_psiH_plane(int k, int nz, int npml) {
  if (npml <= 0) return -1;
  if (k < npml) return k;
  if (k >= nz - npml - 1) return npml + (k - (nz - npml - 1));
  return -1;
}

template <typename T>
__device__ __forceinline__ int adj_mat_of(const AdjParams<T>& p, int k) {
  return p.zmat[k];
}

// n / d for n < 2^31 (FastDiv, internal.h)
__device__ __forceinline__ uint32_t adj_div(uint32_t n, FastDiv f) { return (__umulhi(f.m, n) + n) >> f.l; }

// TE: the forward run was the y-invariant TE form (ny = 1, E_y sources) and the monitor sources
// of the adjoint sit on E_y and H_x only.  Then the adjoints of E_x, E_z, H_y and of the x / z
// polarization and bath modes stay exactly zero (their y-differences vanish on the single row);
// they are constants here, and the carried components are bit-identical to the general form's.
// The TE form carries one component's P / bath adjoints: up to N_b = 8 it runs three blocks per
// SM (80 registers; at four blocks' 64 registers it spilled and its reverse sweep took 2% longer).
//
// LIGHT: the launch over the planes outside [ra, rb) (no material there: field and CPML adjoints
// only), at eight blocks per SM; otherwise the launch over the cells [ra, rb).  The planes without
// material are most of a cavity's grid and do little work per cell, so at the heavy launch's
// occupancy they waited on memory latency.
template <typename T, int NBMAX, bool TE = false, bool LIGHT = false>
__global__ void __launch_bounds__(kAdjThreads, LIGHT ? 8 : ((TE && NBMAX <= 8) ? 3 : 0))
adjoint_k1(const AdjParams<T> p) {
  __shared__ double sg[kAdjThreads / 32][kAdjMaxGrad];
  constexpr int NBA = NBMAX > 0 ? NBMAX : 1;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q = LIGHT ? (idx < p.ra ? idx : idx + (p.rb - p.ra)) : p.ra + idx;
  const bool own = LIGHT ? q < p.ncell : q < p.rb;
  const int64_t N = p.ncell, plane = p.plane;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  // gradient terms: summed in the state precision over a thread's components and a warp's cells,
  // in FP64 from the warp partials on
  T gsig = T(0), ggam = T(0), gk[NBA];
#pragma unroll
  for (int j = 0; j < NBA; ++j) gk[j] = T(0);
  if (own) {
    // cell indices fit in 31 bits (checked when the simulation is created)
    const int k = (int)adj_div((uint32_t)q, p.fd_plane);
    const int r = (int)q - k * (int)plane;
    const int j = (int)adj_div((uint32_t)r, p.fd_nx), i = r - j * nx;
    const int im = i > 0 ? i - 1 : nx - 1, jm = j > 0 ? j - 1 : ny - 1;
    const T S = p.S;
    const T hsrc = T(0.5);
    // adjoint of H^{n+1}, with this step's H-monitor source added on the fly
    auto Hb = [&](int c, int ii, int jj, int kk) -> T {
      if (kk < 0 || kk >= nz || (TE && c == 1)) return T(0);
      T v = __ldg(p.Hb + c * N + (int64_t)kk * plane + (int64_t)jj * nx + ii);   // read-only here
      if (p.zm >= 0 && (kk == p.zm - 1 || kk == p.zm)) {
        if (c == 0) v += hsrc * p.gHx;
        if (c == 1) v += hsrc * p.gHy;
      }
      return v;
    };
    const T hx = Hb(0, i, j, k), hy = Hb(1, i, j, k), hz = Hb(2, i, j, k);
    // F6^T: curl^T of H_bar
    T ex = TE ? T(0) : p.Eb[q] + S * ((hy - Hb(1, i, j, k - 1)) - (hz - Hb(2, i, jm, k)));
    T ey = p.Eb[N + q] + S * ((hz - Hb(2, im, j, k)) - (hx - Hb(0, i, j, k - 1)));
    T ez = TE ? T(0) : p.Eb[2 * N + q] + S * ((hx - Hb(0, i, jm, k)) - (hy - Hb(1, im, j, k)));
    // F6^T into psi_H_bar, then F5^T
    const int kp = adj_psiH_plane(k, nz, p.npml);
    const int64_t nph = (int64_t)(2 * p.npml + 1) * plane;
    if (kp >= 0) {
      const int64_t o = (int64_t)kp * plane + r;
      const T px = __ldg(p.psiHb + o) + S * hx;
      const T py = TE ? T(0) : __ldg(p.psiHb + nph + o) - S * hy;
      const T bH = __ldg(p.pmlH + 2 * k), cH = __ldg(p.pmlH + 2 * k + 1);
      ey -= cH * px;
      if (!TE) ex -= cH * py;
      p.psiHb_out[o] = bH * px;
      if (!TE) p.psiHb_out[nph + o] = bH * py;
    }
    if (k > 0) {
      const int kpm = adj_psiH_plane(k - 1, nz, p.npml);
      if (kpm >= 0) {
        const int64_t o = (int64_t)kpm * plane + r;
        const T px = __ldg(p.psiHb + o) + S * Hb(0, i, j, k - 1);
        const T py = TE ? T(0) : __ldg(p.psiHb + nph + o) - S * Hb(1, i, j, k - 1);
        const T cH = __ldg(p.pmlH + 2 * (k - 1) + 1);
        ey += cH * px;
        if (!TE) ex += cH * py;
      }
    }
    // F3^T (polarization and bath), with the gradient of material gm
    const int mi = LIGHT ? -1 : adj_mat_of(p, k);
    T inv_eps = T(1);
    T Pold[3], Pmold[3];
    bool haveP = false;
    if (mi >= 0) {
      const MatK<T>& M = p.mat[mi];
      inv_eps = M.inv_eps;
      if (M.kind != kVacuum) {
        haveP = true;
        const int64_t rm = (int64_t)(k - M.zlo) * plane + r;
        const int nb = M.kind == kLorentzBath ? M.nb : 0;
        const T* __restrict__ cfm = p.coefLit + M.coef_off * kCoefStride;
        const bool grad = mi == p.gm;
        // each of these adjoint arrays is read and then written at the same index by this thread
        // only, and no two of them overlap
        T* __restrict__ Pb_ = p.Pb;
        T* __restrict__ Pmb_ = p.Pmb;
        T* __restrict__ Y0_ = p.Yb0;
        T* __restrict__ Y1_ = p.Yb1;
        T ec[3] = {ex, ey, ez};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (TE && c != 1) continue;
          const int64_t ip = c * p.nmatcell + M.base + rm;
          T pn = Pb_[ip];           // adjoint of P^{n+3/2}
          T pold = Pmb_[ip];        // adjoint of P^{n+1/2} (the shift P_m <- P)
          T pmold = T(0);
          T yold[NBA], ymold[NBA], ynb[NBA];
          const int64_t yc = M.ybase + (int64_t)c * nb * M.ncell + rm;
          // the TE form (one component, registers to spare) issues every load of the cell before
          // any arithmetic: the bath adjoints and, for the differentiated layer, the recorded
          // forward values; the arithmetic below is the same either way
          T y1v[NBA], fEv = T(0), fPnv = T(0), fPmv = T(0), fYv[NBA], fYmv[NBA];
          if constexpr (TE) {
            const int64_t ig = (int64_t)c * M.ncell + rm;
#pragma unroll
            for (int jj = 0; jj < NBA; ++jj) {
              if (jj < nb) {
                ynb[jj] = Y0_[yc + jj * M.ncell];
                y1v[jj] = Y1_[yc + jj * M.ncell];
              }
            }
            if (grad) {
              fEv = __ldg(p.fE + ig);
              fPnv = __ldg(p.fPn + ig);
              fPmv = __ldg(p.fPm + ig);
#pragma unroll
              for (int jj = 0; jj < NBA; ++jj) {
                if (jj < nb) {
                  const int64_t iy = ((int64_t)c * nb + jj) * M.ncell + rm;
                  fYv[jj] = __ldg(p.fY + iy);
                  fYmv[jj] = __ldg(p.fYm + iy);
                }
              }
            }
          }
#pragma unroll
          for (int jj = 0; jj < NBA; ++jj) {
            yold[jj] = T(0);
            ymold[jj] = T(0);
            if (!TE) ynb[jj] = T(0);
            if (jj < nb) {
              const T* cf = cfm + jj * kCoefStride;
              const T yn = TE ? ynb[jj] : Y0_[yc + jj * M.ncell];   // adjoint of Y^{n+3/2}
              ynb[jj] = yn;
              yold[jj] = (TE ? y1v[jj] : Y1_[yc + jj * M.ncell]) + __ldg(cf + 1) * yn;   // shift + a_j
              ymold[jj] = __ldg(cf + 3) * yn;                           // (b_j + 1)
              const T c4 = __ldg(cf + 4);
              pn += c4 * yn;                                            // c_j (P_new - P_m)
              pmold -= c4 * yn;
            }
          }
          const T f = pn * M.inv_A;
          ec[c] += M.cE * f;
          pold += -M.c1m * f;
          pmold += -M.c2 * f;
          // gradient terms first: they need pn and the incoming bath adjoints ynb
          if (grad) {
            const int64_t ig = (int64_t)c * M.ncell + rm;
            const T E = TE ? fEv : __ldg(p.fE + ig), Pn = TE ? fPnv : __ldg(p.fPn + ig);
            const T Pm = TE ? fPmv : __ldg(p.fPm + ig);
            const T hA = p.thA;
            gsig += pn * E * p.tsig;
            ggam += pn * hA * (Pm - Pn);
#pragma unroll
            for (int jj = 0; jj < NBA; ++jj) {
              if (jj < nb) {
                const int64_t iy = ((int64_t)c * nb + jj) * M.ncell + rm;
                const T Y = TE ? fYv[jj] : __ldg(p.fY + iy), Ym = TE ? fYmv[jj] : __ldg(p.fYm + iy);
                gk[jj] += pn * hA * (p.tds[jj] * (Pm - Pn) - (p.ta[jj] * Y + p.tb[jj] * Ym)) +
                          ynb[jj] * p.tdc[jj] * (Pn - Pm);
              }
            }
          }
#pragma unroll
          for (int jj = 0; jj < NBA; ++jj) {
            if (jj < nb) {
              const T* cf = cfm + jj * kCoefStride;
              const T w = T(-0.5) * p.dt * __ldg(cf) * f;   // -(dt/2) k_j / A * P_bar_new
              Y0_[yc + jj * M.ncell] = yold[jj] + w * __ldg(cf + 1);
              Y1_[yc + jj * M.ncell] = ymold[jj] + w * __ldg(cf + 2);
            }
          }
          Pold[c] = pold;
          Pmold[c] = pmold;
        }
        ex = ec[0];
        ey = ec[1];
        ez = ec[2];
      }
    }
    // E-monitor source (adjoint of the plane mean of E^{n+1/2})
    if (k == p.zm) {
      if (!TE) ex += p.gEx;
      ey += p.gEy;
    }
    // pointwise parts of F2^T
    if (haveP) {
      const MatK<T>& M = p.mat[mi];
      const int64_t rm = (int64_t)(k - M.zlo) * plane + r;
      const T e3[3] = {ex, ey, ez};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (TE && c != 1) continue;
        const int64_t ip = c * p.nmatcell + M.base + rm;
        p.Pb[ip] = Pold[c] - e3[c] * inv_eps;
        p.Pmb[ip] = Pmold[c] + e3[c] * inv_eps;
      }
    }
    const int kq = adj_psiE_plane(k, nz, p.npml);
    if (kq >= 0) {
      const int64_t npe = (int64_t)(2 * p.npml) * plane;
      const int64_t o = (int64_t)kq * plane + r;
      if (!TE) p.psiEb[o] += -S * inv_eps * ex;
      p.psiEb[npe + o] += S * inv_eps * ey;
    }
    if (!TE) p.Eb[q] = ex;
    p.Eb[N + q] = ey;
    if (!TE) p.Eb[2 * N + q] = ez;
  }
  // per-block gradient partials of material gm (blocks holding none of its cells skip)
  if (!LIGHT && p.gm >= 0) {
    const MatK<T>& G = p.mat[p.gm];
    const int64_t b0 = p.ra + (int64_t)blockIdx.x * blockDim.x, b1 = b0 + blockDim.x;
    const int64_t m0 = (int64_t)G.zlo * plane, m1 = (int64_t)G.zhi * plane;
    if (b1 > m0 && b0 < m1) {
      const int np = 2 + G.nb;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int t = 0; t < 2 + NBA; ++t) {
        if (t < np) {
          T v = t == 0 ? gsig : (t == 1 ? ggam : gk[t - 2 < NBA ? t - 2 : 0]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) sg[warp][t] = (double)v;
        }
      }
      __syncthreads();
      if ((int)threadIdx.x < np) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sg[w][threadIdx.x];
        p.gpart[(int64_t)blockIdx.x * kAdjMaxGrad + threadIdx.x] += v;
      }
    }
  }
}

template <typename T, bool TE = false>
__global__ void __launch_bounds__(kAdjThreads) adjoint_k2(const AdjParams<T> p) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.ncell) return;
  const int64_t N = p.ncell, plane = p.plane;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int k = (int)adj_div((uint32_t)q, p.fd_plane);
  const int r = (int)q - k * (int)plane;
  const int j = (int)adj_div((uint32_t)r, p.fd_nx), i = r - j * nx;
  const int ip = i + 1 < nx ? i + 1 : 0, jp = j + 1 < ny ? j + 1 : 0;
  const T S = p.S;
  const T inv0 = [&] {
    const int m = adj_mat_of(p, k);
    return m >= 0 ? p.mat[m].inv_eps : T(1);
  }();
  const T inv1 = [&] {
    if (k + 1 >= nz) return T(0);
    const int m = adj_mat_of(p, k + 1);
    return m >= 0 ? p.mat[m].inv_eps : T(1);
  }();
  // E_bar / eps_inf of a cell (zero outside the grid)
  auto Et = [&](int c, int ii, int jj, int kk, T inv) -> T {
    if (kk >= nz || (TE && c != 1)) return T(0);
    return p.Eb[c * N + (int64_t)kk * plane + (int64_t)jj * nx + ii] * inv;
  };
  const T ex = Et(0, i, j, k, inv0), ey = Et(1, i, j, k, inv0), ez = Et(2, i, j, k, inv0);
  T hx = p.Hb[q], hy = TE ? T(0) : p.Hb[N + q], hz = p.Hb[2 * N + q];
  // this step's H-monitor source
  if (p.zm >= 0 && (k == p.zm - 1 || k == p.zm)) {
    hx += T(0.5) * p.gHx;
    if (!TE) hy += T(0.5) * p.gHy;
  }
  // curl^T of F2
  hx += S * ((ey - Et(1, i, j, k + 1, inv1)) - (ez - Et(2, i, jp, k, inv0)));
  hy += S * ((ez - Et(2, ip, j, k, inv0)) - (ex - Et(0, i, j, k + 1, inv1)));
  hz += S * ((ex - Et(0, i, jp, k, inv0)) - (ey - Et(1, ip, j, k, inv0)));
  // F1^T
  const int64_t npe = (int64_t)(2 * p.npml) * plane;
  const int kq = adj_psiE_plane(k, nz, p.npml);
  if (kq >= 0) {
    const int64_t o = (int64_t)kq * plane + r;
    const T px = TE ? T(0) : p.psiEb[o], py = p.psiEb[npe + o];
    const T bE = p.pmlE[2 * k], cE = p.pmlE[2 * k + 1];
    if (!TE) hy += cE * px;
    hx += cE * py;
    if (!TE) p.psiEb_out[o] = bE * px;
    p.psiEb_out[npe + o] = bE * py;
  }
  if (k + 1 < nz) {
    const int kq1 = adj_psiE_plane(k + 1, nz, p.npml);
    if (kq1 >= 0) {
      const int64_t o = (int64_t)kq1 * plane + r;
      const T cE1 = p.pmlE[2 * (k + 1) + 1];
      if (!TE) hy -= cE1 * p.psiEb[o];
      hx -= cE1 * p.psiEb[npe + o];
    }
  }
  p.Hb[q] = hx;
  if (!TE) p.Hb[N + q] = hy;
  p.Hb[2 * N + q] = hz;
}

template <typename T, bool TE>
int launch_adjoint_form(const AdjParams<T>& p0, int nbmax, void* stream) {
  const int64_t nblk = (p0.ncell + kAdjThreads - 1) / kAdjThreads;
  cudaStream_t st = (cudaStream_t)stream;
  // adjoint_k1 in two launches: the planes from the first material's to the last's, and the rest
  AdjParams<T> p = p0;
  p.ra = p.ncell;
  p.rb = 0;
  for (int m = 0; m < p.nmat; ++m) {
    p.ra = std::min<int64_t>(p.ra, (int64_t)p.mat[m].zlo * p.plane);
    p.rb = std::max<int64_t>(p.rb, (int64_t)p.mat[m].zhi * p.plane);
  }
  if (p.rb <= p.ra) p.ra = p.rb = 0;
  const int64_t nheavy = (p.rb - p.ra + kAdjThreads - 1) / kAdjThreads;
  const int64_t nlight = (p.ncell - (p.rb - p.ra) + kAdjThreads - 1) / kAdjThreads;
  if (nlight > 0) adjoint_k1<T, 0, TE, true><<<(unsigned)nlight, kAdjThreads, 0, st>>>(p);
  if (nheavy > 0) {
    switch (nbmax) {
      case 0: adjoint_k1<T, 0, TE><<<(unsigned)nheavy, kAdjThreads, 0, st>>>(p); break;
      case 4: adjoint_k1<T, 4, TE><<<(unsigned)nheavy, kAdjThreads, 0, st>>>(p); break;
      case 8: adjoint_k1<T, 8, TE><<<(unsigned)nheavy, kAdjThreads, 0, st>>>(p); break;
      case 16: adjoint_k1<T, 16, TE><<<(unsigned)nheavy, kAdjThreads, 0, st>>>(p); break;
      default: adjoint_k1<T, 32, TE><<<(unsigned)nheavy, kAdjThreads, 0, st>>>(p); break;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  adjoint_k2<T, TE><<<(unsigned)nblk, kAdjThreads, 0, st>>>(p);
  return (int)cudaGetLastError();
}

// te = 1: the TE form (y-invariant TE forward run, adjoint sources on E_y and H_x only)
template <typename T>
int launch_adjoint_impl(const AdjParams<T>& p, int nbmax, int te, void* stream) {
  return te ? launch_adjoint_form<T, true>(p, nbmax, stream) : launch_adjoint_form<T, false>(p, nbmax, stream);
}

}  // namespace fdtdbath
