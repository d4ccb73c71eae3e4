// tb2.cuh -- two steps per pass over grids without polarizable material (temporal blocking).
//
// One launch advances every cell by two full steps of the Yee scheme (Eq. FDTD-1D in the 3D curl
// form, Eq. 1a / Eq. 1b): H^n, E^{n+1/2}, H^{n+1}, E^{n+3/2}, with the CPML memories of both
// half-steps and the soft plane sources of both steps, and records the monitor and energy partial
// sums of both steps.  It reads E^{n-1/2}, H^{n-1} and the memories once and writes E^{n+3/2},
// H^{n+1} and the memories once, so the state crosses HBM once per two steps instead of twice.
//
// Decomposition: a CTA owns a 32 x 8 (x, y) tile and marches along a z-chunk [zb, ze).  The
// first step's values (level 1) never leave the chip: per plane the CTA computes
//   H^n       on the tile grown by 2 cells at -x / -y and 1 at +x / +y (the H1 box),
//   E^{n+1/2} on the tile grown by 1 cell on every side (the E1 box),
//   H^{n+1}   on the tile grown by 1 cell at -x / -y (the H2 box),
//   E^{n+3/2} on the tile,
// the second step lagging one plane behind the first (H^{n+1}(k) needs E^{n+1/2}(k+1)).  The
// boxes overlap those of the neighbouring tiles, whose border values are recomputed here from
// the same inputs by the same expressions.  Along z the chunk's first two planes below and one
// plane above are recomputed the same way (ghost planes), so chunks are independent.  Every
// output goes to the other buffer (E, H, both CPML memories), so no CTA ever reads a value that
// another CTA has already advanced.
//
// Frames: all shared-memory planes use one geometry, columns x0-4 .. x0+35 and rows from y0-2
// (origin (x0-4, y0-2), 16-byte aligned rows for the copies): rows up to y0+9 for E^{n-1/2},
// whose +y neighbours the H1 box reads, up to y0+8 for the rest; E^{n-1/2} and H^{n-1} are staged
// by 16-byte cp.async copies kTbAhead planes ahead.  72 KB of shared memory and at most 80
// registers (FP32) let three CTAs share an SM.  The arithmetic of each half-step
// is the general step kernel's (h_update, the curl differences in the same order, the source
// term added last), so with FP64 (built without contraction) the fields agree bit for bit with
// two single steps.
#pragma once

#include <cuda_runtime.h>

#include "step3d.cuh"

namespace fdtdbath {

constexpr int kTbThreads = kTbTX * kTbTY;   // Tb2Params, kTbTX, kTbTY: internal.h
constexpr int kTbRingE = 3;    // E^{n-1/2} frames: planes k, k+1 (read), k+2 (landing)
constexpr int kTbRingH = 2;    // H^{n-1} frames: plane k (read), k+1 (landing)
constexpr int kTbRingH1 = 3;   // H^n and the H-side memories after step n: planes k-2 .. k
constexpr int kTbRingE1 = 2;   // E^{n+1/2}: planes k-1, k
constexpr int kTbFX = kTbTX + 8, kTbFY = kTbTY + 4, kTbFE = kTbFX * kTbFY, kTbFH = kTbFX * (kTbFY - 1);
// halo cells (box minus tile) of the three boxes, in frame columns [c0, c1) and rows [r0, r1)
constexpr int kTbH1c0 = 2, kTbH1c1 = kTbTX + 5, kTbH1r0 = 0, kTbH1r1 = kTbTY + 3;
constexpr int kTbE1c0 = 3, kTbE1c1 = kTbTX + 5, kTbE1r0 = 1, kTbE1r1 = kTbTY + 3;
constexpr int kTbH2c0 = 3, kTbH2c1 = kTbTX + 4, kTbH2r0 = 1, kTbH2r1 = kTbTY + 2;
__host__ __device__ constexpr int tb_halo(int c0, int c1, int r0, int r1) { return (c1 - c0) * (r1 - r0) - kTbTX * kTbTY; }
static_assert(tb_halo(kTbH1c0, kTbH1c1, kTbH1r0, kTbH1r1) <= kTbThreads, "one H1 halo cell per thread");
static_assert(tb_halo(kTbE1c0, kTbE1c1, kTbE1r0, kTbE1r1) <= kTbThreads, "one E1 halo cell per thread");
static_assert(tb_halo(kTbH2c0, kTbH2c1, kTbH2r0, kTbH2r1) <= kTbThreads, "one H2 halo cell per thread");

// shared-memory elements: the E^{n-1/2}, H^{n-1}, H^n and E^{n+1/2} rings and H^{n+1} of one plane
// (three components each), the ring of the H-side memories after step n (two components); then
// eight doubles of block-sum scratch
constexpr int kTbSmemElems = kTbRingE * 3 * kTbFE + (kTbRingH + kTbRingH1 + kTbRingE1) * 3 * kTbFH + 3 * kTbFH +
                             kTbRingH1 * 2 * kTbFH;
template <typename T>
constexpr size_t tb2_smem_bytes() {
  return (size_t)kTbSmemElems * sizeof(T) + 8 * sizeof(double);
}

// halo cell t of a box: the box's rows above the tile, then those below it, then the columns left
// and right of the tile row by row; returns the frame offset
__device__ __forceinline__ int tb_halo_cell(int t, int c0, int c1, int r0, int r1) {
  const int W = c1 - c0;
  const int ntop = (2 - r0) * W;
  if (t < ntop) return (r0 + t / W) * kTbFX + c0 + t % W;
  t -= ntop;
  const int nbot = (r1 - (2 + kTbTY)) * W;
  if (t < nbot) return (2 + kTbTY + t / W) * kTbFX + c0 + t % W;
  t -= nbot;
  const int nl = 4 - c0, nr = c1 - (4 + kTbTX);
  const int r = t % (nl + nr);
  return (2 + t / (nl + nr)) * kTbFX + (r < nl ? c0 + r : 4 + kTbTX + (r - nl));
}

template <typename T>
__global__ void __launch_bounds__(kTbThreads, sizeof(T) == 4 ? 3 : 1) tb2_kernel(const Tb2Params<T> q) {
  const Step3DParams<T>& p = q.p;
  constexpr int FE = kTbFE, F = kTbFH, FX = kTbFX;   // E^{n-1/2} frames: 12 rows, the rest 11
  constexpr int VE = 16 / (int)sizeof(T);            // elements per 16-byte copy
  constexpr int CPR = FX / VE;                       // copies per frame row
  constexpr int NPE = kTbFY * CPR;                   // E frame: rows 0 .. kTbFY-1
  constexpr int NPH = (kTbFY - 1) * CPR;             // H frame: rows 0 .. kTbFY-2
  constexpr int CE = (NPE + kTbThreads - 1) / kTbThreads, CH = (NPH + kTbThreads - 1) / kTbThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sE0 = reinterpret_cast<T*>(smem_raw);           // [kTbRingE][3][FE]  E^{n-1/2}
  T* sH0 = sE0 + kTbRingE * 3 * FE;                  // [kTbRingH][3][F]   H^{n-1}
  T* sH1 = sH0 + kTbRingH * 3 * F;                   // [kTbRingH1][3][F]  H^n
  T* sE1 = sH1 + kTbRingH1 * 3 * F;                  // [kTbRingE1][3][F]  E^{n+1/2}
  T* sH2 = sE1 + kTbRingE1 * 3 * F;                  // [3][F]             H^{n+1}
  T* sPH = sH2 + 3 * F;                              // [kTbRingH1][2][F]  H-side memories after step n
  double* sred = reinterpret_cast<double*>(sPH + kTbRingH1 * 2 * F);

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kTbTX + tx;
  const int x0 = blockIdx.x * kTbTX, y0 = blockIdx.y * kTbTY;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  // every array index fits in 32 bits (checked when the simulation is created)
  const int plane = (int)p.plane, ncell = (int)p.ncell;
  const int chunk = p.chunk_ids[blockIdx.z];
  const int zb = p.zstart[chunk], ze = p.zstart[chunk + 1];
  const T dt = p.dt, S = p.S;
  const int nbxy = p.nbxy;
  const int bxy = blockIdx.y * gridDim.x + blockIdx.x;   // partial-sum slot of this tile
  const int pstrH = (2 * p.npml + 1) * plane, pstrE = 2 * p.npml * plane;

  // own cell and the halo cells this thread computes in each box (frame offset, grid column)
  const int own_f = (ty + 2) * FX + tx + 4;
  const int own_g = (y0 + ty) * nx + x0 + tx;
  auto gcol = [&](int f) {
    const int r = f / FX, c = f - r * FX;
    return wrapi(y0 - 2 + r, ny) * nx + wrapi(x0 - 4 + c, nx);
  };
  constexpr int NH1 = tb_halo(kTbH1c0, kTbH1c1, kTbH1r0, kTbH1r1);
  constexpr int NE1 = tb_halo(kTbE1c0, kTbE1c1, kTbE1r0, kTbE1r1);
  constexpr int NH2 = tb_halo(kTbH2c0, kTbH2c1, kTbH2r0, kTbH2r1);
  // the two boxes of each phase on different warps: H^n halo cells on threads 0.., H^{n+1} halo
  // cells on threads 160.. (phase 1), E^{n+1/2} halo cells on the last threads (phase 2)
  constexpr int H2T0 = 160, E1T0 = kTbThreads - NE1;
  static_assert(NH1 <= H2T0 && H2T0 + NH2 <= kTbThreads, "halo threads");
  const int h1_f = tid < NH1 ? tb_halo_cell(tid, kTbH1c0, kTbH1c1, kTbH1r0, kTbH1r1) : -1;
  const int e1_f = tid >= E1T0 ? tb_halo_cell(tid - E1T0, kTbE1c0, kTbE1c1, kTbE1r0, kTbE1r1) : -1;
  const int h2_f = (tid >= H2T0 && tid < H2T0 + NH2) ? tb_halo_cell(tid - H2T0, kTbH2c0, kTbH2c1, kTbH2r0, kTbH2r1) : -1;
  const int h1_g = h1_f >= 0 ? gcol(h1_f) : 0;
  const int e1_g = e1_f >= 0 ? gcol(e1_f) : 0;
  const int h2_g = h2_f >= 0 ? gcol(h2_f) : 0;

  // 16-byte copies this thread stages per plane: E frame positions from the low threads up, H frame
  // positions from the high threads down (frame offset, grid offset of the first element)
  int ce_s[CE], ce_g[CE], ch_s[CH], ch_g[CH];
#pragma unroll
  for (int r = 0; r < CE; ++r) {
    const int idx = tid + r * kTbThreads;
    ce_s[r] = -1;
    ce_g[r] = 0;
    if (idx < NPE) {
      const int row = idx / CPR, c = idx - row * CPR;
      ce_s[r] = row * FX + c * VE;
      ce_g[r] = wrapi(y0 - 2 + row, ny) * nx + wrapi(x0 - 4 + c * VE, nx);
    }
  }
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    const int idx = (kTbThreads - 1 - tid) + r * kTbThreads;
    ch_s[r] = -1;
    ch_g[r] = 0;
    if (idx < NPH) {
      const int row = idx / CPR, c = idx - row * CPR;
      ch_s[r] = row * FX + c * VE;
      ch_g[r] = wrapi(y0 - 2 + row, ny) * nx + wrapi(x0 - 4 + c * VE, nx);
    }
  }
  const T* __restrict__ Ein = p.Ein;
  const T* __restrict__ Hin = p.Hin;
  // E^{n-1/2} of plane k (zero beyond the grid), H^{n-1} of plane k < nz
  auto issueE = [&](int k) {
    T* dst = sE0 + (k % kTbRingE) * 3 * FE;
#pragma unroll
    for (int r = 0; r < CE; ++r) {
      if (ce_s[r] < 0) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (k < nz) {
          cp_async16(dst + c * FE + ce_s[r], Ein + c * ncell + k * plane + ce_g[r]);
        } else {
#pragma unroll
          for (int v = 0; v < VE; ++v) dst[c * FE + ce_s[r] + v] = T(0);
        }
      }
    }
  };
  auto issueH = [&](int k) {
    T* dst = sH0 + (k % kTbRingH) * 3 * F;
#pragma unroll
    for (int r = 0; r < CH; ++r) {
      if (ch_s[r] < 0) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) cp_async16(dst + c * F + ch_s[r], Hin + c * ncell + k * plane + ch_g[r]);
    }
  };

  // planes: H^n from kA (two planes below the chunk; none below the grid) to ze, E^{n+1/2} from a1
  // to ze, H^{n+1} from a1 and E^{n+3/2} on the chunk.  Iteration k computes, in two phases with
  // one barrier between them, {H^n(k), H^{n+1}(k-2)} and then {E^{n+1/2}(k), E^{n+3/2}(k-2)}: the
  // second step lags two planes behind the first, so no phase waits for its own results.
  const int kA = zb >= 2 ? zb - 2 : 0;
  const int a1 = zb >= 1 ? zb - 1 : 0;
  const int kE_last = ze + 1;                        // last E^{n-1/2} plane read
  const int kH_last = ze < nz ? ze : nz - 1;         // last H^{n-1} plane read

  // source current of a plane at grid column g: the step's amplitudes (a, b) per source
  auto source = [&](int k, int g, const T* sa, const T* sb, T* J, bool* has) {
    J[0] = J[1] = J[2] = T(0);
    has[0] = has[1] = has[2] = false;
    for (int s = 0; s < p.nsrc; ++s) {
      if (p.src_z[s] != k) continue;
      T v = sa[s];
      if (p.src_cos[s]) v = sa[s] * p.src_cos[s][g] + sb[s] * p.src_sin[s][g];
      const int sc = p.src_comp[s];
      if (sc == 0) {
        J[0] += v;
        has[0] = true;
      } else if (sc == 1) {
        J[1] += v;
        has[1] = true;
      } else {
        J[2] += v;
        has[2] = true;
      }
    }
  };
  auto src_plane = [&](int k) {
    for (int s = 0; s < p.nsrc; ++s)
      if (p.src_z[s] == k) return true;
    return false;
  };
  auto in_box = [&](int k) { return k >= p.ebox_lo && k < p.ebox_hi; };
  // H-side monitor partials of a plane from the own cells' values (rows of one step)
  auto mon_H = [&](int k, T vx, T vy, double* rows) {
    for (int mm = 0; mm < p.nmon; ++mm) {
      const int zm = p.mon_z[mm];
      if (k == zm - 1 || k == zm) {
        const int off = (k == zm) ? 1 : 0;
        const double sx = block_sum((double)vx, sred);
        const double sy = block_sum((double)vy, sred);
        if (tid == 0 && rows) {
          rows[(int64_t)(4 * mm + off) * nbxy + bxy] = sx;
          rows[(int64_t)(4 * mm + 2 + off) * nbxy + bxy] = sy;
        }
      }
    }
  };
  auto mon_E = [&](int k, T vx, T vy, double* rows) {
    for (int mm = 0; mm < p.nmon; ++mm) {
      if (k == p.mon_z[mm]) {
        const double sx = block_sum((double)vx, sred);
        const double sy = block_sum((double)vy, sred);
        if (tid == 0 && rows) {
          rows[(int64_t)(2 * mm) * nbxy + bxy] = sx;
          rows[(int64_t)(2 * mm + 1) * nbxy + bxy] = sy;
        }
      }
    }
  };

  // per-thread energy sums of both steps (state precision, block-reduced in FP64 at the end)
  T uE1 = T(0), uH1 = T(0), uE2 = T(0), uH2 = T(0);
  // own-cell values carried between planes: H^{n+1} of the plane below E^{n+3/2}'s plane, and
  // E^{n+1/2} with the E-side memories after step n of the two planes before the current one
  T hm[2] = {T(0), T(0)};
  T q0[3] = {T(0), T(0), T(0)}, q1[3] = {T(0), T(0), T(0)};
  T pq0[2] = {T(0), T(0)}, pq1[2] = {T(0), T(0)};

  issueE(kA);
  issueE(kA + 1);
  issueH(kA);
  cp_async_commit();

  for (int k = kA; k <= ze + 1; ++k) {
    cp_async_wait<0>();   // E(k+1) and H(k), requested one plane ago
    __syncthreads();      // ... and every read of the previous plane's phases is done
    if (k + 2 <= kE_last) issueE(k + 2);   // into the slot of E(k-1)
    if (k + 1 <= kH_last) issueH(k + 1);   // into the slot of H(k-1)
    cp_async_commit();

    const int m = k - 2;                                   // plane of the second step
    const bool doH1 = k <= ze && k < nz;
    const bool doE1 = k >= a1 && k <= ze && k < nz;
    const bool own1 = k >= zb && k < ze;                   // plane k belongs to the chunk
    const bool doL2 = m >= a1 && m < ze;                   // H^{n+1}(m)
    const bool out2 = m >= zb && m < ze;                   // E^{n+3/2}(m), stored outputs
    T* h1 = sH1 + (k % kTbRingH1) * 3 * F;                 // H^n(k)
    const T* h1m = sH1 + ((k + 2) % kTbRingH1) * 3 * F;    // H^n(k-1)
    T* ph1 = sPH + (k % kTbRingH1) * 2 * F;
    T* e1 = sE1 + (k & 1) * 3 * F;                         // E^{n+1/2}(k)

    // ---------------- phase 1: H^n(k) on the H1 box, H^{n+1}(m) on the H2 box ----------------
    T h1own[3] = {T(0), T(0), T(0)}, h2own[3] = {T(0), T(0), T(0)};
    if (doH1) {
      const T* e0 = sE0 + (k % kTbRingE) * 3 * FE;
      const T* e0n = sE0 + ((k + 1) % kTbRingE) * 3 * FE;
      const T* hin = sH0 + (k % kTbRingH) * 3 * F;
      const int ip = psiH_plane(k, nz, p.npml);
      T b = T(1), c = T(0);
      if (ip >= 0) {
        b = p.pmlH[2 * k];
        c = p.pmlH[2 * k + 1];
      }
      auto cell = [&](int f, int g, T* o) {
        HIn<T> e;
        e.ex0 = e0[f];
        e.ex_k1 = e0n[f];
        e.ex_j1 = e0[f + FX];
        e.ey0 = e0[FE + f];
        e.ey_k1 = e0n[FE + f];
        e.ey_i1 = e0[FE + f + 1];
        e.ez0 = e0[2 * FE + f];
        e.ez_j1 = e0[2 * FE + f + FX];
        e.ez_i1 = e0[2 * FE + f + 1];
        T hx = hin[f], hy = hin[F + f], hz = hin[2 * F + f];
        T psx = T(0), psy = T(0);
        if (ip >= 0) {
          psx = p.psiHin[ip * plane + g];
          psy = p.psiHin[pstrH + ip * plane + g];
        }
        h_update<T>(e, hx, hy, hz, &psx, &psy, b, c, ip >= 0, S);
        h1[f] = hx;
        h1[F + f] = hy;
        h1[2 * F + f] = hz;
        if (ip >= 0) {
          ph1[f] = psx;
          ph1[F + f] = psy;
        }
        o[0] = hx;
        o[1] = hy;
        o[2] = hz;
      };
      cell(own_f, own_g, h1own);
      if (h1_f >= 0) {
        T d[3];
        cell(h1_f, h1_g, d);
      }
    }
    if (doL2) {
      const T* ea = sE1 + (m & 1) * 3 * F;                 // E^{n+1/2}(m)
      const T* eb = sE1 + ((m + 1) & 1) * 3 * F;           // E^{n+1/2}(m+1)
      const T* ha = sH1 + ((k + 1) % kTbRingH1) * 3 * F;   // H^n(m)
      const T* pa = sPH + ((k + 1) % kTbRingH1) * 2 * F;
      const int ip = psiH_plane(m, nz, p.npml);
      T b = T(1), c = T(0);
      if (ip >= 0) {
        b = p.pmlH[2 * m];
        c = p.pmlH[2 * m + 1];
      }
      auto cell = [&](int f, int g, bool write_out, T* o) {
        HIn<T> e;
        e.ex0 = ea[f];
        e.ex_k1 = eb[f];
        e.ex_j1 = ea[f + FX];
        e.ey0 = ea[F + f];
        e.ey_k1 = eb[F + f];
        e.ey_i1 = ea[F + f + 1];
        e.ez0 = ea[2 * F + f];
        e.ez_j1 = ea[2 * F + f + FX];
        e.ez_i1 = ea[2 * F + f + 1];
        T hx = ha[f], hy = ha[F + f], hz = ha[2 * F + f];
        T psx = T(0), psy = T(0);
        if (ip >= 0) {
          psx = pa[f];
          psy = pa[F + f];
        }
        h_update<T>(e, hx, hy, hz, &psx, &psy, b, c, ip >= 0, S);
        sH2[f] = hx;
        sH2[F + f] = hy;
        sH2[2 * F + f] = hz;
        if (write_out) {
          const int qo = m * plane + g;
          p.Hout[qo] = hx;
          p.Hout[ncell + qo] = hy;
          p.Hout[2 * ncell + qo] = hz;
          if (ip >= 0) {
            p.psiHout[ip * plane + g] = psx;
            p.psiHout[pstrH + ip * plane + g] = psy;
          }
        }
        o[0] = hx;
        o[1] = hy;
        o[2] = hz;
      };
      cell(own_f, own_g, out2, h2own);
      if (h2_f >= 0) {
        T d[3];
        cell(h2_f, h2_g, false, d);
      }
    }
    // H-side monitor and energy partials: step n (H^n of the chunk's planes), step n+1 (H^{n+1})
    if (doH1 && own1) {
      mon_H(k, h1own[0], h1own[1], p.mon_partial_H);
      if (p.eH_on && in_box(k)) uH1 += h1own[0] * h1own[0] + h1own[1] * h1own[1] + h1own[2] * h1own[2];
    }
    if (out2) {
      mon_H(m, h2own[0], h2own[1], q.mon_partial_H2);
      if (q.eH_on2 && in_box(m)) uH2 += h2own[0] * h2own[0] + h2own[1] * h2own[1] + h2own[2] * h2own[2];
    }
    __syncthreads();

    // ---------------- phase 2: E^{n+3/2}(m) on the tile, E^{n+1/2}(k) on the E1 box ----------------
    if (out2) {
      const int f = own_f;
      const T Hx = sH2[f], Hy = sH2[F + f], Hz = sH2[2 * F + f];
      const T dyHz = Hz - sH2[2 * F + f - FX];
      const T dzHy = Hy - hm[1];
      const T dzHx = Hx - hm[0];
      const T dxHz = Hz - sH2[2 * F + f - 1];
      const T dxHy = Hy - sH2[F + f - 1];
      const T dyHx = Hx - sH2[f - FX];
      T curl[3];
      const int ip = psiE_plane(m, nz, p.npml);
      if (ip >= 0) {
        const T b = p.pmlE[2 * m], c = p.pmlE[2 * m + 1];
        const int pq = ip * plane + own_g;
        const T px = b * pq0[0] + c * dzHy;
        const T py = b * pq0[1] + c * dzHx;
        q.psiEout[pq] = px;
        q.psiEout[pstrE + pq] = py;
        curl[0] = dyHz - (dzHy + px);
        curl[1] = (dzHx + py) - dxHz;
      } else {
        curl[0] = dyHz - dzHy;
        curl[1] = dzHx - dxHz;
      }
      curl[2] = dxHy - dyHx;
      T J[3];
      bool has[3];
      if (src_plane(m)) {
        source(m, own_g, q.src_a2, q.src_b2, J, has);
      } else {
        J[0] = J[1] = J[2] = T(0);
        has[0] = has[1] = has[2] = false;
      }
      T Ev[3];
      const int qo = m * plane + own_g;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        T e = q0[cc] + S * curl[cc];
        if (has[cc]) e = e + dt * J[cc];
        Ev[cc] = e;
        p.Eout[cc * ncell + qo] = e;
      }
      if (q.eE_on2 && in_box(m)) uE2 += T(1) * (Ev[0] * Ev[0] + Ev[1] * Ev[1] + Ev[2] * Ev[2]);
      mon_E(m, Ev[0], Ev[1], q.mon_partial_E2);
    }
    T e1own[3] = {T(0), T(0), T(0)}, pe1own[2] = {T(0), T(0)};
    if (doE1) {
      const T* e0 = sE0 + (k % kTbRingE) * 3 * FE;
      const bool below0 = k == 0;                   // no H below the grid
      const int ip = psiE_plane(k, nz, p.npml);
      T b = T(1), c = T(0);
      if (ip >= 0) {
        b = p.pmlE[2 * k];
        c = p.pmlE[2 * k + 1];
      }
      const bool srck = src_plane(k);
      auto cell = [&](int f, int g, T* Ev, T* pe) {
        const T Hx = h1[f], Hy = h1[F + f], Hz = h1[2 * F + f];
        const T hxm = below0 ? T(0) : h1m[f];
        const T hym = below0 ? T(0) : h1m[F + f];
        const T dyHz = Hz - h1[2 * F + f - FX];
        const T dzHy = Hy - hym;
        const T dzHx = Hx - hxm;
        const T dxHz = Hz - h1[2 * F + f - 1];
        const T dxHy = Hy - h1[F + f - 1];
        const T dyHx = Hx - h1[f - FX];
        T curl[3];
        if (ip >= 0) {
          const int pq = ip * plane + g;
          const T px = b * p.psiE[pq] + c * dzHy;
          const T py = b * p.psiE[pstrE + pq] + c * dzHx;
          pe[0] = px;
          pe[1] = py;
          curl[0] = dyHz - (dzHy + px);
          curl[1] = (dzHx + py) - dxHz;
        } else {
          curl[0] = dyHz - dzHy;
          curl[1] = dzHx - dxHz;
        }
        curl[2] = dxHy - dyHx;
        T J[3];
        bool has[3];
        if (srck) {
          source(k, g, p.src_a, p.src_b, J, has);
        } else {
          J[0] = J[1] = J[2] = T(0);
          has[0] = has[1] = has[2] = false;
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          T e = e0[cc * FE + f] + S * curl[cc];
          if (has[cc]) e = e + dt * J[cc];
          Ev[cc] = e;
          e1[cc * F + f] = e;
        }
      };
      cell(own_f, own_g, e1own, pe1own);
      if (e1_f >= 0) {
        T d[3], dp[2];
        cell(e1_f, e1_g, d, dp);
      }
      if (own1) {
        if (p.eE_on && in_box(k)) uE1 += T(1) * (e1own[0] * e1own[0] + e1own[1] * e1own[1] + e1own[2] * e1own[2]);
        mon_E(k, e1own[0], e1own[1], p.mon_partial_E);
      }
    } else if (k == nz) {
      // plane nz: no E above the grid (read by H^{n+1}(nz-1) on the next plane)
      for (int t = tid; t < 3 * F; t += kTbThreads) e1[t] = T(0);
    }
    if (k >= a1) {   // the carried own values move one plane on
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        q0[cc] = q1[cc];
        q1[cc] = e1own[cc];
      }
      pq0[0] = pq1[0];
      pq0[1] = pq1[1];
      pq1[0] = pe1own[0];
      pq1[1] = pe1own[1];
    }
    if (doL2) {
      hm[0] = h2own[0];
      hm[1] = h2own[1];
    }
  }
  cp_async_wait<0>();

  // energy partials of both steps (every block writes its slot; the polarization and bath terms
  // are zero without polarizable material)
  const int64_t nrow = (int64_t)nbxy * p.nchunks_total, slot = (int64_t)chunk * nbxy + bxy;
  if (p.eE_on) {
    const double a = block_sum(uE1, sred);
    if (tid == 0) {
      p.en_partial_E[slot] = a;
      p.en_partial_E[nrow + slot] = 0.0;
      p.en_partial_E[2 * nrow + slot] = 0.0;
    }
  }
  if (p.eH_on) {
    const double a = block_sum(uH1, sred);
    if (tid == 0) p.en_partial_H[slot] = a;
  }
  if (q.eE_on2) {
    const double a = block_sum(uE2, sred);
    if (tid == 0) {
      q.en_partial_E2[slot] = a;
      q.en_partial_E2[nrow + slot] = 0.0;
      q.en_partial_E2[2 * nrow + slot] = 0.0;
    }
  }
  if (q.eH_on2) {
    const double a = block_sum(uH2, sred);
    if (tid == 0) q.en_partial_H2[slot] = a;
  }
}

template <typename T>
int tb2_launch(const Tb2Params<T>& q, int nchunks, void* stream) {
  auto kern = tb2_kernel<T>;
  constexpr size_t smem = tb2_smem_bytes<T>();
  static bool attr_set = false;   // once per process: more than 48 KB of shared memory
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  dim3 grid(q.p.nx / kTbTX, q.p.ny / kTbTY, nchunks), block(kTbTX, kTbTY);
  kern<<<grid, block, smem, (cudaStream_t)stream>>>(q);
  return (int)cudaGetLastError();
}

}  // namespace fdtdbath
