// cavity1d.cuh -- persistent kernel for x-polarized 1D cavities (nx = ny = 1): all steps of a
// call in one launch, the whole state in registers.
//
// A cavity is advanced by one thread-block cluster of C CTAs.  CTA r owns the contiguous cell
// range [bounds[r], bounds[r+1]) -- the host balances these ranges by work (a bath cell costs
// about N_b + 2 vacuum cells) -- and thread t of it owns one cell.  For the whole launch each
// thread keeps its cell's E_x, H_y, CPML memories, D (FP64 path), the two levels of P_x and
// of every bath mode Y_j in registers; only monitor values and energy partial sums leave the
// SM each step, and the state is written back at the end.
//
// One step is the paper's loop (Eq. FDTD-1D, Sec. II.C): the D/E half-step with the soft source
// (its per-step amplitude comes from a host-computed table), the polarization and bath update
// (Eq. Pz_update-LB / Pz_1D_Lorentz / Yzj_finite_difference), a cluster barrier, the H half-
// step, a cluster barrier.  A half-step publishes its field in shared memory; the neighbour
// across a CTA boundary is read from the other CTA's shared memory (distributed shared memory),
// which the cluster barrier makes visible.
//
// Only the x polarization (E_x, H_y, P_x and its bath) is advanced; the host uses this kernel
// while every other component is zero (x-polarized sources, no other field written), which
// the linear update then keeps exactly zero.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace fdtdbath {

__device__ __forceinline__ int psiE_plane1d(int k, int nz, int npml) {
  if (k < npml) return k;
  if (k >= nz - npml) return npml + (k - (nz - npml));
  return -1;
}
__device__ __forceinline__ int psiH_plane1d(int k, int nz, int npml) {
  if (npml <= 0) return -1;
  if (k < npml) return k;
  if (k >= nz - npml - 1) return npml + (k - (nz - npml - 1));
  return -1;
}

template <typename T, bool INC, int NBMAX>
__global__ void __launch_bounds__(kCav1DThreads) cavity1d_kernel(const Cav1DParams<T> p) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ T sE[kCav1DThreads];
  __shared__ T sH[kCav1DThreads];
  constexpr int NBA = NBMAX > 0 ? NBMAX : 1;
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
  // energy partials: one per warp of the cluster and quantity (NW per quantity)
  const int NW = C * nwarp, wslot = rank * nwarp + warp;
  const int nz = p.nz;
  const int lo = p.bounds[rank], hi = p.bounds[rank + 1];
  const int cnt = hi - lo;
  const int z = lo + t;
  const bool own = t < cnt;
  const T S = p.S, dt = p.dt;

  // ---- the cell's constants and state, into registers ----
  int mi = -1;
  for (int m = 0; m < p.nmat; ++m)
    if (own && z >= p.mat[m].zlo && z < p.mat[m].zhi) mi = m;
  const int ipE = own ? psiE_plane1d(z, nz, p.npml) : -1;
  const int ipH = own ? psiH_plane1d(z, nz, p.npml) : -1;
  const T bE = ipE >= 0 ? p.pmlE[2 * z] : T(1), cE = ipE >= 0 ? p.pmlE[2 * z + 1] : T(0);
  const T bH = ipH >= 0 ? p.pmlH[2 * z] : T(1), cH = ipH >= 0 ? p.pmlH[2 * z + 1] : T(0);
  T e = own ? p.E[z] : T(0);
  T h = own ? p.H[nz + z] : T(0);          // H_y
  T psE = ipE >= 0 ? p.psiE[ipE] : T(0);   // memory of the E_x update (from dH_y/dz)
  T psH = ipH >= 0 ? p.psiH[p.psiH_stride + ipH] : T(0);   // memory of the H_y update
  const bool mat = mi >= 0;
  const bool osc = mat && p.mat[mi].kind != kVacuum;
  const bool bath = mat && p.mat[mi].kind == kLorentzBath && NBMAX > 0;
  const int nb = bath ? p.mat[mi].nb : 0;
  int r = 0, yc = 0, ystr = 0;
  T Pa = T(0), Pb = T(0), D = T(0);
  T Y[NBA], Ym[NBA];
  const int cur0 = p.pcur0;
  if (mat) {
    const MatK<T>& M = p.mat[mi];
    const int rl = z - M.zlo;
    r = (int)M.base + rl;
    yc = (int)M.ybase + rl;   // component 0
    ystr = (int)M.ncell;
    Pa = p.Pslot[cur0][r];
    Pb = p.Pslot[cur0 ^ 1][r];
    if (!INC) D = p.D[r];
  }
#pragma unroll
  for (int j = 0; j < NBA; ++j) {
    Y[j] = T(0);
    Ym[j] = T(0);
    if (j < nb) {
      Y[j] = p.Yslot[cur0][yc + j * ystr];
      Ym[j] = p.Yslot[cur0 ^ 1][yc + j * ystr];
    }
  }
  // per-material constants
  T cEm = T(0), c1m = T(0), Wm = T(0), c2 = T(0), invA = T(1), inv_eps = T(1), rho_idt2 = T(0),
    w0r2dt2 = T(0), eps = T(1);
  if (mat) {
    const MatK<T>& M = p.mat[mi];
    cEm = M.cE;
    c1m = M.c1m;
    Wm = M.W;
    c2 = M.c2;
    invA = M.inv_A;
    inv_eps = M.inv_eps;
    rho_idt2 = M.rho_idt2;
    w0r2dt2 = M.w0r2dt2;
    eps = M.eps;
    if (p.sig) {
      // per-cell oscillator strength sigma(r) (Eq. EOM_Lorentz): drive and energy weight
      const T sg = p.sig[r];
      cEm = M.dcE * sg;
      rho_idt2 = sg > T(0) ? M.rho_s / sg : T(0);
    }
  }
  const T* cfm = mat ? p.coef + p.mat[mi].coef_off * kCoefStride : p.coef;
  const bool in_box = own && z >= p.ebox_lo && z < p.ebox_hi;
  const bool is_src = own && p.nsrc > 0 && z == p.src_z;
  // neighbours across the CTA boundaries (distributed shared memory)
  const T* sH_prev = rank > 0 ? cluster.map_shared_rank(sH, rank - 1) : nullptr;
  const T* sE_next = rank + 1 < C ? cluster.map_shared_rank(sE, rank + 1) : nullptr;
  const int cnt_prev = rank > 0 ? p.bounds[rank] - p.bounds[rank - 1] : 0;

  sH[t] = h;
  cluster.sync();

  for (int s = 0; s < p.nsteps; ++s) {
    const int64_t n = p.step0 + s;
    double* rec = p.partial + (int64_t)(n % p.ring_cap) * p.ring_stride;
    const bool en = p.energy_on && (n % p.every) == 0;
    // energy terms of the cell and their warp sums in the state precision (FP64 arithmetic is
    // slow on this part: in the FP32 path it would dominate the step), FP64 from the warp sums on
    T uE = T(0), uP = T(0), uB = T(0), uH = T(0);
    // ---------------- D/E half-step, polarization and bath ----------------
    if (own) {
      T hm;   // H_y(z-1)
      if (t > 0) hm = sH[t - 1];
      else hm = sH_prev ? sH_prev[cnt_prev - 1] : T(0);
      const T dzHy = h - hm;
      T curl;
      if (ipE >= 0) {
        psE = bE * psE + cE * dzHy;
        curl = T(0) - (dzHy + psE);
      } else {
        curl = T(0) - dzHy;
      }
      const T J = is_src ? (T)p.src_tab[s] : T(0);
      if (!mat) {
        e = e + S * curl;
        if (is_src) e = e + dt * J;
      } else if (!INC) {
        D = D + S * curl;
        if (is_src) D = D + dt * J;
        e = inv_eps * (D - Pa);
      } else {
        T inc = S * curl;
        if (is_src) inc = inc + dt * J;
        e = e + (inc - (Pa - Pb)) * inv_eps;
      }
      if (osc) {
        T bsum = T(0);
        T V[NBA];
#pragma unroll
        for (int j = 0; j < NBA; ++j) {
          V[j] = T(0);
          if (j < nb) {
            const T* cf = cfm + j * kCoefStride;
            if (!INC) {
              bsum = bath_sum_lit(bsum, cf[0], cf[1], cf[2], Y[j], Ym[j]);   // k_j (a_j Y^n + b_j Y^{n-1})
            } else {
              V[j] = Y[j] - Ym[j];
              bsum = bsum + (cf[0] * Y[j] + cf[1] * V[j]);             // k_j ((a_j+b_j) Y - b_j V)
            }
          }
        }
        T Pn, Vn, V0;
        if (!INC) {
          T num = cEm * e - c1m * Pa - c2 * Pb;
          if (bath) num = num - T(0.5) * dt * bsum;
          Pn = invA * num;
          Vn = Pn - Pa;
          V0 = Pa - Pb;
        } else {
          V0 = Pa - Pb;
          T num = cEm * e - Wm * Pa + c2 * V0;
          if (bath) num = num - T(0.5) * dt * bsum;
          Vn = num * invA;
          Pn = Pa + Vn;
        }
        const T dP = Vn + V0;
        T ub = T(0);
#pragma unroll
        for (int j = 0; j < NBA; ++j) {
          if (j < nb) {
            const T* cf = cfm + j * kCoefStride;
            T Yn, Vy;
            if (!INC) {
              Yn = bath_new_lit(cf[1], cf[3], cf[4], Y[j], Ym[j], Pn - Pb);
              Vy = Yn - Y[j];
            } else {
              Vy = cf[2] * Y[j] + cf[3] * V[j] + cf[4] * dP;
              Yn = Y[j] + Vy;
            }
            Ym[j] = Y[j];
            Y[j] = Yn;
            if (en) ub = INC ? ub + (Vy * Vy + cf[5] * Yn * Yn) : bath_energy_lit(ub, Vy, cf[5], Yn);
          }
        }
        Pb = Pa;
        Pa = Pn;
        if (en && in_box) {
          uP = rho_idt2 * (Vn * Vn + w0r2dt2 * Pn * Pn);
          uB = rho_idt2 * ub;
        }
      }
      if (en && in_box) uE = eps * (e * e);
      if (p.nmon > 0 && z == p.mon_z) {
        rec[p.monE_off + 0] = (double)e;
        rec[p.monE_off + 1] = 0.0;
      }
    }
    sE[t] = e;
    if (en) {
      // one partial per warp and quantity into the ring (summed there in fixed order later, so
      // no serial FP64 sum sits between the half-steps)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        uE += __shfl_down_sync(0xffffffffu, uE, o);
        uP += __shfl_down_sync(0xffffffffu, uP, o);
        uB += __shfl_down_sync(0xffffffffu, uB, o);
      }
      if (lane == 0) {
        rec[p.enE_off + wslot] = (double)uE;
        rec[p.enE_off + NW + wslot] = (double)uP;
        rec[p.enE_off + 2 * NW + wslot] = (double)uB;
      }
    }
    cluster.sync();
    // ---------------- H half-step ----------------
    if (own) {
      T ep;   // E_x(z+1)
      if (t + 1 < cnt) ep = sE[t + 1];
      else ep = sE_next ? sE_next[0] : T(0);
      const T dzEx = ep - e;
      if (ipH >= 0) {
        psH = bH * psH + cH * dzEx;
        h = h - S * ((dzEx + psH) - T(0));
      } else {
        h = h - S * (dzEx - T(0));
      }
      if (en && in_box) uH = h * h;
      if (p.nmon > 0 && (z == p.mon_z - 1 || z == p.mon_z)) {
        const int off = z == p.mon_z ? 1 : 0;
        rec[p.monH_off + off] = 0.0;
        rec[p.monH_off + 2 + off] = (double)h;
      }
    }
    sH[t] = h;
    if (en) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) uH += __shfl_down_sync(0xffffffffu, uH, o);
      if (lane == 0) rec[p.enH_off + wslot] = (double)uH;
    }
    cluster.sync();
  }

  // ---- write the state back ----
  if (own) {
    p.E[z] = e;
    p.H[nz + z] = h;
    if (ipE >= 0) p.psiE[ipE] = psE;
    if (ipH >= 0) p.psiH[p.psiH_stride + ipH] = psH;
    if (mat) {
      const int cur = cur0 ^ (p.nsteps & 1);   // slot of P^{n+1/2} after the launch
      p.Pslot[cur][r] = Pa;
      p.Pslot[cur ^ 1][r] = Pb;
      if (!INC) p.D[r] = D;
#pragma unroll
      for (int j = 0; j < NBA; ++j) {
        if (j < nb) {
          p.Yslot[cur][yc + j * ystr] = Y[j];
          p.Yslot[cur ^ 1][yc + j * ystr] = Ym[j];
        }
      }
    }
  }
  // no CTA may exit while a neighbour can still read its shared memory
  cluster.sync();
}

}  // namespace fdtdbath
