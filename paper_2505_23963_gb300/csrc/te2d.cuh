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

constexpr int VX = 4;          // cells per thread
constexpr int SEG = 32 * VX;   // cells per warp (the row segment)
constexpr int WARPS = 2;       // warps per CTA

__device__ __forceinline__ void ld4(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
// the sum of v over the eight lanes of each 32-cell slot (lanes 8h .. 8h+7), on every lane
__device__ __forceinline__ double slot_sum(double v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace te2d

// One launch over the chunks p.chunk_ids[0 .. gridDim.y): CTA (bx, by) takes the row segments
// WARPS bx + w of chunk by.  The host runs it on FP32 TE-form grids with nx a multiple of SEG and
// no source plane inside a layer.
template <typename T>
__global__ void __launch_bounds__(32 * te2d::WARPS) te2d_kernel(const Step3DParams<T> p) {
  using namespace te2d;
  static_assert(sizeof(T) == 4, "the FP32 TE form");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int seg = blockIdx.x * WARPS + w;
  const int x0 = seg * SEG, i0 = x0 + VX * lane;
  const int nx = p.nx, nz = p.nz;
  const int plane = (int)p.plane, ncell = (int)p.ncell;   // plane = nx (ny = 1)
  const int chunk = p.chunk_ids[blockIdx.y];
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

  // ---- prologue: H_x^n of plane zb-1 (the z-difference of the E update at zb); zb-1 is never
  // inside the CPML (chunk starts are planned that way) ----
  T hxm[VX];
  T ey0[VX], ey1[VX], hx[VX], hz[VX];
#pragma unroll
  for (int v = 0; v < VX; ++v) hxm[v] = T(0);
  ld4(Ey_in + zb * plane + i0, ey0);
  if (zb > 0) {
    T e_m[VX], h_m[VX];
    ld4(Ey_in + (zb - 1) * plane + i0, e_m);
    ld4(Hx_in + (zb - 1) * plane + i0, h_m);
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      const T dzEy = ey0[v] - e_m[v];
      hxm[v] = h_m[v] - S * (T(0) - dzEy);
    }
  }
  // the planes' E_y (k+1), H_x, H_z (k) for the first plane
  if (zb + 1 < nz) ld4(Ey_in + (zb + 1) * plane + i0, ey1);
  else
#pragma unroll
    for (int v = 0; v < VX; ++v) ey1[v] = T(0);
  ld4(Hx_in + zb * plane + i0, hx);
  ld4(Hz_in + zb * plane + i0, hz);
  // E_y after the segment (lane 31), E_y and H_z before it (lane 0), of the plane
  T eyr = lane == 31 ? Ey_in[zb * plane + xr] : T(0);
  T eyl = lane == 0 ? Ey_in[zb * plane + xl] : T(0);
  T hzl = lane == 0 ? Hz_in[zb * plane + xl] : T(0);

  T uE = T(0), uP = T(0), uH = T(0);
  for (int k = zb; k < ze; ++k) {
    // ---- the next plane's inputs, a plane ahead ----
    T ey2[VX], hxn[VX], hzn[VX];
    const bool more = k + 1 < ze;
    if (more) {
      if (k + 2 < nz) ld4(Ey_in + (k + 2) * plane + i0, ey2);
      else
#pragma unroll
        for (int v = 0; v < VX; ++v) ey2[v] = T(0);
      ld4(Hx_in + (k + 1) * plane + i0, hxn);
      ld4(Hz_in + (k + 1) * plane + i0, hzn);
    }
    T eyr_n = T(0), eyl_n = T(0), hzl_n = T(0);
    if (more && lane == 31) eyr_n = Ey_in[(k + 1) * plane + xr];
    if (more && lane == 0) {
      eyl_n = Ey_in[(k + 1) * plane + xl];
      hzl_n = Hz_in[(k + 1) * plane + xl];
    }
    // the plane's kind (uniform over the warp)
    int mi = -1;
    for (int m = 0; m < p.nmat; ++m)
      if (k >= p.mat[m].zlo && k < p.mat[m].zhi) mi = m;
    const bool in_box = k >= p.ebox_lo && k < p.ebox_hi;
    const bool pmlE = k < p.npml || k >= nz - p.npml;
    const bool pmlH = p.npml > 0 && (k < p.npml || k >= nz - p.npml - 1);
    const int ipE = k < p.npml ? k : k - nz + 2 * p.npml;
    const int ipH = k < p.npml ? k : k - nz + 1 + 2 * p.npml;
    const int q = k * plane + i0;
    T psx[VX], psy[VX], Pa[VX], Pb[VX];
    if (pmlH) ld4(p.psiHin + ipH * plane + i0, psx);
    if (pmlE) ld4(p.psiE + pstrE + ipE * plane + i0, psy);
    const MatK<T>* M = mi >= 0 ? &p.mat[mi] : nullptr;
    const bool osc = M && M->kind != kVacuum;
    const int r = M ? (int)M->base + (k - M->zlo) * plane + i0 : 0;
    if (osc) {
      ld4(p.Pa + nmc + r, Pa);
      ld4(p.Pb + nmc + r, Pb);
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
    st4(Hx_out + q, hx);
    st4(Hz_out + q, hz);
    if (pmlH) st4(p.psiHout + ipH * plane + i0, psx);
    // H_z^n at x-1 of the thread's first cell: the lane before, or on lane 0 recomputed for the
    // cell before the segment
    T hzx0 = __shfl_up_sync(0xffffffffu, hz[VX - 1], 1);
    if (lane == 0) hzx0 = hzl - S * ((ey0[0] - eyl) - T(0));
    if (p.eH_on && in_box)
#pragma unroll
      for (int v = 0; v < VX; ++v) uH += hx[v] * hx[v] + T(0) * T(0) + hz[v] * hz[v];
    // H monitors (planes zm-1 and zm): sums of H_x (and of the zero H_y) per 32-cell slot
    for (int m = 0; m < p.nmon; ++m) {
      const int zm = p.mon_z[m];
      if ((k != zm - 1 && k != zm) || !p.mon_partial_H) continue;
      double sx = 0.0;
#pragma unroll
      for (int v = 0; v < VX; ++v) sx += (double)hx[v];
      sx = slot_sum(sx);
      if ((lane & 7) == 0) {
        const int slot = x0 / 32 + lane / 8;
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
    for (int s = 0; s < p.nsrc; ++s) {
      if (p.src_z[s] != k || p.src_comp[s] != 1) continue;
      hasJ = true;
      if (p.src_cos[s]) {
        T cs[VX], sn[VX];
        ld4(p.src_cos[s] + i0, cs);
        ld4(p.src_sin[s] + i0, sn);
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
          // increment form: V^{n+1} = [cE E - w0^2 dt^2 P^n + c2 V^n] / A
          const T V0 = pa - pb;
          const T num = M->cE * e - M->W * pa + M->c2 * V0;
          const T Vn = num * M->inv_A;
          Pn[v] = pa + Vn;
          if (p.eE_on && in_box) uP += M->rho_idt2 * (Vn * Vn + M->w0r2dt2 * Pn[v] * Pn[v]);
        }
        if (p.eE_on && in_box) uE += M->eps * (T(0) * T(0) + e * e + T(0) * T(0));
      }
    }
    st4(Ey_out + q, Ey);
    if (pmlE) st4(p.psiE + pstrE + ipE * plane + i0, psy);
    if (osc) st4(p.Pb + nmc + r, Pn);   // overwrites P^{n-1/2}
    // E monitors (plane zm): sums of the zero E_x and of E_y per 32-cell slot
    for (int m = 0; m < p.nmon; ++m) {
      if (k != p.mon_z[m] || !p.mon_partial_E) continue;
      double sy = 0.0;
#pragma unroll
      for (int v = 0; v < VX; ++v) sy += (double)Ey[v];
      sy = slot_sum(sy);
      if ((lane & 7) == 0) {
        const int slot = x0 / 32 + lane / 8;
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
    const double e = slot_sum((double)uE), pp = slot_sum((double)uP), h = slot_sum((double)uH);
    if ((lane & 7) == 0) {
      const int64_t slot = (int64_t)chunk * p.nbxy + x0 / 32 + lane / 8;
      if (p.eE_on) {
        p.en_partial_E[slot] = e;
        p.en_partial_E[(int64_t)p.nbxy * p.nchunks_total + slot] = pp;
        p.en_partial_E[(int64_t)2 * p.nbxy * p.nchunks_total + slot] = 0.0;
      }
      if (p.eH_on) p.en_partial_H[slot] = h;
    }
  }
}

}  // namespace fdtdbath
