// te2d.cuh -- the fused step of the y-invariant TE form (ny = 1, every source on E_y: Sec. II.C's
// 2D case) over the z-chunks without bath modes, FP32.
//
// It computes what step3d_kernel<float, true, 0, 1, false, true, 128> computes there -- the H
// half-step of the previous step (H_x, H_z from E_y^{n-1/2}, Eq. 1b with the CPML memory of the
// z-derivative), this step's E_y half-step (Eq. 1a, D = E + P, soft E_y sources) and the Lorentz /
// Drude update of P_y (Eq. Pz_1D_Lorentz) -- with the same expressions in the same order.  The
// general kernel stages one row of E_y, H_x, H_z per plane into shared memory through 128-wide
// single-row tiles and two barriers per plane; with one row and no y-neighbours the step needs
// no shared memory at all:
//
//   * one warp owns a 32 VX-cell segment of the row (lane l the VX = 4 cells x0 + VX l ...) and
//     marches along a z-chunk; every global access of a thread is one 16-byte vector, and the next
//     plane's E_y, H_x, H_z are loaded a plane ahead into registers;
//   * H_x^n of the plane below and E_y of the plane above stay in registers from plane to plane;
//   * x-neighbours pass between lanes by shuffles; at the segment's ends lane 31 reads E_y of the
//     next segment's first cell (an input) and lane 0 recomputes H_z^n of the cell before the
//     segment, so warps share nothing and no barrier is needed;
//   * monitor and energy partials are per 32-cell slot, as the general kernel writes them: each
//     slot is eight lanes of one warp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace fdtdbath {

namespace te2d {

constexpr int WARPS = 2;       // warps per CTA
// per-plane table bits (material index + 1 in the low four bits)
enum : int { kBox = 0x10, kMonE = 0x20, kMonH = 0x40, kSrc = 0x80, kPmlE = 0x100, kPmlH = 0x200 };

// VX-cell vectors of a thread (VX = 4: one 16-byte access)
template <int VX>
struct V;
template <>
struct V<4> {
  static __device__ __forceinline__ void ld(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
  static __device__ __forceinline__ void st(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct V<1> {
  static __device__ __forceinline__ void ld(const float* p, float* o) { o[0] = *p; }
  static __device__ __forceinline__ void st(float* p, const float* v) { *p = v[0]; }
};
// the sum of v over the LPS lanes of each 32-cell slot, on every lane
template <int LPS>
__device__ __forceinline__ double slot_sum(double v) {
#pragma unroll
  for (int o = LPS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace te2d

// One launch over the chunks p.chunk_ids[0 .. gridDim.y): CTA (bx, by) takes the row segments
// WARPS bx + w of chunk by.  The host runs it on FP32 TE-form grids with nx a multiple of
// 32 VX WARPS and no source plane inside a layer.  NB = 0: the chunks without bath modes, VX = 4;
// NB > 0: the chunks of Lorentz-Bath layers with at most NB modes, VX = 1 (the cell's P_y and
// modes in registers), the general kernel's bath arithmetic for the y component.
template <typename T, int VX, int NB>
__device__ __forceinline__ void te2d_body(const Step3DParams<T>& p, int bx, int cy) {
  using namespace te2d;
  static_assert(sizeof(T) == 4, "the FP32 TE form");
  static_assert(NB == 0 || VX == 1, "bath modes: one cell per thread");
  using VV = V<VX>;
  constexpr int SEG = 32 * VX;   // cells per warp (the row segment)
  constexpr int LPS = 32 / VX;   // lanes per 32-cell slot
  constexpr int NBA = NB > 0 ? NB : 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int seg = bx * WARPS + w;
  const int x0 = seg * SEG, i0 = x0 + VX * lane;
  const int nx = p.nx, nz = p.nz;
  const int plane = (int)p.plane, ncell = (int)p.ncell;   // plane = nx (ny = 1)
  const int chunk = p.chunk_ids[cy];
  const int zb = p.zstart[chunk], ze = p.zstart[chunk + 1];
  const T S = p.S, dt = p.dt;
  const int nmc = (int)p.nmatcell;
  const int pstrE = 2 * p.npml * plane;
  const int xl = x0 == 0 ? nx - 1 : x0 - 1;          // the cell before the segment
  const int xr = x0 + SEG == nx ? 0 : x0 + SEG;      // the cell after it
  const T* __restrict__ Ein = p.Ein;
  const T* __restrict__ Hin = p.Hin;
  // E_y and H_x, H_z of the general layout [3][nz][1][nx]
  const T* Ey_in = Ein + ncell;
  const T* Hx_in = Hin;
  const T* Hz_in = Hin + 2 * ncell;
  T* Ey_out = p.Eout + ncell;
  T* Hx_out = p.Hout;
  T* Hz_out = p.Hout + 2 * ncell;

  // ---- the chunk's plane table and (NB > 0) the coefficient rows, per CTA ----
  __shared__ int sInfo[kMaxChunk];
  __shared__ T sCoef[NB > 0 ? kMaxMat * NBA * kCoefStride : 1];
  for (int t = threadIdx.x; t < ze - zb; t += blockDim.x) {
    const int k = zb + t;
    int info = 0;
    for (int m = 0; m < p.nmat; ++m)
      if (k >= p.mat[m].zlo && k < p.mat[m].zhi) info = m + 1;
    if (k >= p.ebox_lo && k < p.ebox_hi) info |= kBox;
    for (int m = 0; m < p.nmon; ++m) {
      if (k == p.mon_z[m]) info |= kMonE;
      if (k == p.mon_z[m] || k == p.mon_z[m] - 1) info |= kMonH;
    }
    for (int q = 0; q < p.nsrc; ++q)
      if (k == p.src_z[q]) info |= kSrc;
    if (k < p.npml || k >= nz - p.npml) info |= kPmlE;
    if (p.npml > 0 && (k < p.npml || k >= nz - p.npml - 1)) info |= kPmlH;
    sInfo[t] = info;
  }
  if (NB > 0)
    for (int t = threadIdx.x; t < kCoefStride * p.nmodes; t += blockDim.x) sCoef[t] = p.coef[t];
  __syncthreads();

  // ---- prologue: H_x^n of plane zb-1 (the z-difference of the E update at zb); zb-1 is never
  // inside the CPML (chunk starts are planned that way) ----
  T hxm[VX];
  T ey0[VX], ey1[VX], hx[VX], hz[VX];
#pragma unroll
  for (int v = 0; v < VX; ++v) hxm[v] = T(0);
  VV::ld(Ey_in + zb * plane + i0, ey0);
  if (zb > 0) {
    T e_m[VX], h_m[VX];
    VV::ld(Ey_in + (zb - 1) * plane + i0, e_m);
    VV::ld(Hx_in + (zb - 1) * plane + i0, h_m);
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      const T dzEy = ey0[v] - e_m[v];
      hxm[v] = h_m[v] - S * (T(0) - dzEy);
    }
  }
  // the planes' E_y (k+1), H_x, H_z (k) for the first plane
  if (zb + 1 < nz) VV::ld(Ey_in + (zb + 1) * plane + i0, ey1);
  else
#pragma unroll
    for (int v = 0; v < VX; ++v) ey1[v] = T(0);
  VV::ld(Hx_in + zb * plane + i0, hx);
  VV::ld(Hz_in + zb * plane + i0, hz);
  // E_y after the segment (lane 31), E_y and H_z before it (lane 0), of the plane
  T eyr = lane == 31 ? Ey_in[zb * plane + xr] : T(0);
  T eyl = lane == 0 ? Ey_in[zb * plane + xl] : T(0);
  T hzl = lane == 0 ? Hz_in[zb * plane + xl] : T(0);

  T uE = T(0), uP = T(0), uB = T(0), uH = T(0);
  for (int k = zb; k < ze; ++k) {
    // ---- the next plane's inputs, a plane ahead ----
    T ey2[VX], hxn[VX], hzn[VX];
    const bool more = k + 1 < ze;
    if (more) {
      if (k + 2 < nz) VV::ld(Ey_in + (k + 2) * plane + i0, ey2);
      else
#pragma unroll
        for (int v = 0; v < VX; ++v) ey2[v] = T(0);
      VV::ld(Hx_in + (k + 1) * plane + i0, hxn);
      VV::ld(Hz_in + (k + 1) * plane + i0, hzn);
    }
    T eyr_n = T(0), eyl_n = T(0), hzl_n = T(0);
    if (more && lane == 31) eyr_n = Ey_in[(k + 1) * plane + xr];
    if (more && lane == 0) {
      eyl_n = Ey_in[(k + 1) * plane + xl];
      hzl_n = Hz_in[(k + 1) * plane + xl];
    }
    // the plane's kind (uniform over the CTA)
    const int info = sInfo[k - zb];
    const int mi = (info & 0xF) - 1;
    const bool in_box = (info & kBox) != 0;
    const bool pmlE = (info & kPmlE) != 0, pmlH = (info & kPmlH) != 0;
    const int ipE = k < p.npml ? k : k - nz + 2 * p.npml;
    const int ipH = k < p.npml ? k : k - nz + 1 + 2 * p.npml;
    const int q = k * plane + i0;
    T psx[VX], psy[VX], Pa[VX], Pb[VX];
    if (pmlH) VV::ld(p.psiHin + ipH * plane + i0, psx);
    if (pmlE) VV::ld(p.psiE + pstrE + ipE * plane + i0, psy);
    const MatK<T>* M = mi >= 0 ? &p.mat[mi] : nullptr;
    const bool osc = M && M->kind != kVacuum;
    const int r = M ? (int)M->base + (k - M->zlo) * plane + i0 : 0;
    if (osc) {
      VV::ld(p.Pa + nmc + r, Pa);
      VV::ld(p.Pb + nmc + r, Pb);
    }
    // Lorentz-Bath planes (NB > 0): the cell's y-component modes, Y^n and Y^{n-1}
    T bY[NBA], bV[NBA];
    int nbm = 0, yB = 0, mstr = 0;
    const bool bath = NB > 0 && osc && M->kind == kLorentzBath && M->nb > 0;
    if (bath) {
      nbm = M->nb;
      mstr = (int)M->ncell;
      yB = (int)M->ybase + (k - M->zlo) * plane + i0;
#pragma unroll
      for (int jj = 0; jj < NBA; ++jj)
        if (jj < nbm) {
          bY[jj] = p.Ya[yB + (nbm + jj) * mstr];
          bV[jj] = p.Yb[yB + (nbm + jj) * mstr];
        }
    }
    // ---- H^n of plane k (Eq. 1b: H_x from dE_y/dz with its CPML memory, H_z from dE_y/dx) ----
    const T bH = pmlH ? p.pmlH[2 * k] : T(1), cH = pmlH ? p.pmlH[2 * k + 1] : T(0);
    T eyi = __shfl_down_sync(0xffffffffu, ey0[0], 1);   // E_y after the thread's last cell
    if (lane == 31) eyi = eyr;
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      const T dzEy = ey1[v] - ey0[v];
      const T dxEy = (v + 1 < VX ? ey0[v + 1 < VX ? v + 1 : 0] : eyi) - ey0[v];
      if (pmlH) {
        psx[v] = bH * psx[v] + cH * dzEy;
        hx[v] = hx[v] - S * (T(0) - (dzEy + psx[v]));
      } else {
        hx[v] = hx[v] - S * (T(0) - dzEy);
      }
      hz[v] = hz[v] - S * (dxEy - T(0));
    }
    VV::st(Hx_out + q, hx);
    VV::st(Hz_out + q, hz);
    if (pmlH) VV::st(p.psiHout + ipH * plane + i0, psx);
    // H_z^n at x-1 of the thread's first cell: the lane before, or on lane 0 recomputed for the
    // cell before the segment
    T hzx0 = __shfl_up_sync(0xffffffffu, hz[VX - 1], 1);
    if (lane == 0) hzx0 = hzl - S * ((ey0[0] - eyl) - T(0));
    if (p.eH_on && in_box)
#pragma unroll
      for (int v = 0; v < VX; ++v) uH += hx[v] * hx[v] + T(0) * T(0) + hz[v] * hz[v];
    // H monitors (planes zm-1 and zm): sums of H_x (and of the zero H_y) per 32-cell slot
    for (int m = 0; m < ((info & kMonH) ? p.nmon : 0); ++m) {
      const int zm = p.mon_z[m];
      if ((k != zm - 1 && k != zm) || !p.mon_partial_H) continue;
      double sx = 0.0;
#pragma unroll
      for (int v = 0; v < VX; ++v) sx += (double)hx[v];
      sx = slot_sum<LPS>(sx);
      if ((lane & (LPS - 1)) == 0) {
        const int slot = x0 / 32 + lane / LPS;
        const int off = k == zm ? 1 : 0;
        p.mon_partial_H[(int64_t)(4 * m + off) * p.nbxy + slot] = sx;
        p.mon_partial_H[(int64_t)(4 * m + 2 + off) * p.nbxy + slot] = 0.0;
      }
    }
    // ---- E_y^{n+1/2} of plane k (Eq. 1a, D = E + P) and P_y (Eq. Pz_1D_Lorentz) ----
    const T bE = pmlE ? p.pmlE[2 * k] : T(1), cE_ = pmlE ? p.pmlE[2 * k + 1] : T(0);
    T J[VX];
    bool hasJ = false;
#pragma unroll
    for (int v = 0; v < VX; ++v) J[v] = T(0);
    for (int s = 0; s < ((info & kSrc) ? p.nsrc : 0); ++s) {
      if (p.src_z[s] != k || p.src_comp[s] != 1) continue;
      hasJ = true;
      if (p.src_cos[s]) {
        T cs[VX], sn[VX];
        VV::ld(p.src_cos[s] + i0, cs);
        VV::ld(p.src_sin[s] + i0, sn);
#pragma unroll
        for (int v = 0; v < VX; ++v) J[v] += p.src_a[s] * cs[v] + p.src_b[s] * sn[v];
      } else {
#pragma unroll
        for (int v = 0; v < VX; ++v) J[v] += p.src_a[s];
      }
    }
    T Ey[VX], Pn[VX];
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      const T dzHx = hx[v] - hxm[v];
      const T dxHz = hz[v] - (v > 0 ? hz[v > 0 ? v - 1 : 0] : hzx0);
      T curl;
      if (pmlE) {
        psy[v] = bE * psy[v] + cE_ * dzHx;
        curl = (dzHx + psy[v]) - dxHz;
      } else {
        curl = dzHx - dxHz;
      }
      if (!M) {
        T e = ey0[v] + S * curl;
        if (hasJ) e = e + dt * J[v];
        Ey[v] = e;
        if (p.eE_on && in_box) uE += T(1) * (T(0) * T(0) + e * e + T(0) * T(0));
      } else {
        // D-free: E += (dt curl H + dt J - (P^{n+1/2} - P^{n-1/2})) / eps_inf
        T inc = S * curl;
        if (hasJ) inc = inc + dt * J[v];
        const T pa = osc ? Pa[v] : T(0), pb = osc ? Pb[v] : T(0);
        const T e = ey0[v] + (inc - (pa - pb)) * M->inv_eps;
        Ey[v] = e;
        if (osc) {
          // increment form: V^{n+1} = [cE E - w0^2 dt^2 P^n + c2 V^n - dt/2 sum(...)] / A
          const T V0 = pa - pb;
          T num = M->cE * e - M->W * pa + M->c2 * V0;
          T Vn;
          if (NB > 0 && bath) {
            // Eq. Pz_update-LB's bath sum (ascending j), then Eq. Yzj_finite_difference with the
            // coefficient rows {k(a+b), -k b, a+b, -(b+1), c, (w dt)^2}
            const T* cfm = sCoef + M->coef_off * kCoefStride;
            T bsum = T(0);
#pragma unroll
            for (int jj = 0; jj < NBA; ++jj)
              if (jj < nbm) {
                bV[jj] = bY[jj] - bV[jj];   // V_j = Y^n - Y^{n-1}
                bsum = bsum + (cfm[jj * kCoefStride] * bY[jj] + cfm[jj * kCoefStride + 1] * bV[jj]);
              }
            num = num - T(0.5) * dt * bsum;
            Vn = num * M->inv_A;
            Pn[v] = pa + Vn;
            const T dP = Vn + V0;   // P^{n+3/2} - P^{n-1/2}
            T ub = T(0);
#pragma unroll
            for (int jj = 0; jj < NBA; ++jj)
              if (jj < nbm) {
                const T* cf = cfm + jj * kCoefStride;
                const T Vy = cf[2] * bY[jj] + cf[3] * bV[jj] + cf[4] * dP;
                const T Ynew = bY[jj] + Vy;
                p.Yb[yB + (nbm + jj) * mstr] = Ynew;   // overwrites Y^{n-1}
                if (p.eE_on) ub = ub + (Vy * Vy + cf[5] * Ynew * Ynew);
              }
            if (p.eE_on && in_box) uB += M->rho_idt2 * ub;
          } else {
            Vn = num * M->inv_A;
            Pn[v] = pa + Vn;
          }
          if (p.eE_on && in_box) uP += M->rho_idt2 * (Vn * Vn + M->w0r2dt2 * Pn[v] * Pn[v]);
        }
        if (p.eE_on && in_box) uE += M->eps * (T(0) * T(0) + e * e + T(0) * T(0));
      }
    }
    VV::st(Ey_out + q, Ey);
    if (pmlE) VV::st(p.psiE + pstrE + ipE * plane + i0, psy);
    if (osc) VV::st(p.Pb + nmc + r, Pn);   // overwrites P^{n-1/2}
    // E monitors (plane zm): sums of the zero E_x and of E_y per 32-cell slot
    for (int m = 0; m < ((info & kMonE) ? p.nmon : 0); ++m) {
      if (k != p.mon_z[m] || !p.mon_partial_E) continue;
      double sy = 0.0;
#pragma unroll
      for (int v = 0; v < VX; ++v) sy += (double)Ey[v];
      sy = slot_sum<LPS>(sy);
      if ((lane & (LPS - 1)) == 0) {
        const int slot = x0 / 32 + lane / LPS;
        p.mon_partial_E[(int64_t)(2 * m) * p.nbxy + slot] = 0.0;
        p.mon_partial_E[(int64_t)(2 * m + 1) * p.nbxy + slot] = sy;
      }
    }
    // ---- the next plane ----
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      hxm[v] = hx[v];
      ey0[v] = ey1[v];
      if (more) {
        ey1[v] = ey2[v];
        hx[v] = hxn[v];
        hz[v] = hzn[v];
      }
    }
    eyr = eyr_n;
    eyl = eyl_n;
    hzl = hzl_n;
  }
  // ---- energy partials, one per 32-cell slot and chunk (zero outside the box) ----
  if (p.eE_on || p.eH_on) {
    const double e = slot_sum<LPS>((double)uE), pp = slot_sum<LPS>((double)uP);
    const double bb = slot_sum<LPS>((double)uB), h = slot_sum<LPS>((double)uH);
    if ((lane & (LPS - 1)) == 0) {
      const int64_t slot = (int64_t)chunk * p.nbxy + x0 / 32 + lane / LPS;
      if (p.eE_on) {
        p.en_partial_E[slot] = e;
        p.en_partial_E[(int64_t)p.nbxy * p.nchunks_total + slot] = pp;
        p.en_partial_E[(int64_t)2 * p.nbxy * p.nchunks_total + slot] = bb;
      }
      if (p.eH_on) p.en_partial_H[slot] = h;
    }
  }
}

template <typename T, int VX, int NB>
__global__ void __launch_bounds__(32 * te2d::WARPS) te2d_kernel(const Step3DParams<T> p) {
  te2d_body<T, VX, NB>(p, blockIdx.x, blockIdx.y);
}

// Both kinds of chunks in one launch (p.chunk_ids: the nplain chunks without bath modes, then the
// bath chunks): two launches side by side on two streams overlapped well on some runs only.  A
// one-dimensional grid, the bath chunks' CTAs (the longer ones) first.
template <typename T, int NB>
__global__ void __launch_bounds__(32 * te2d::WARPS) te2d_fused_kernel(const Step3DParams<T> p, int nplain,
                                                                      int nbath) {
  const int bxB = p.nx / (32 * te2d::WARPS), bxP = p.nx / (128 * te2d::WARPS);
  const int b = (int)blockIdx.x;
  if (b < nbath * bxB) {
    te2d_body<T, 1, NB>(p, b % bxB, nplain + b / bxB);
  } else {
    const int b2 = b - nbath * bxB;
    te2d_body<T, 4, 0>(p, b2 % bxP, b2 / bxP);
  }
}

}  // namespace fdtdbath
