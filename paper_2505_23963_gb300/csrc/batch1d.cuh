// batch1d.cuh -- one persistent launch advancing a batch of independent x-polarized 1D cavities
// (the paper's 1D scheme, Eq. FDTD-1D with Eq. Pz_update-LB / Pz_1D_Lorentz /
// Yzj_finite_difference, Sec. II.C) for all steps of a call.
//
// The host packs the cavities into thread-block clusters and cuts each cluster's cells into one
// contiguous range per CTA (batch.h).  For the whole launch a CTA keeps its cells' E_x, H_y, the
// two levels of P_x (and D_x on the FP64 path), CPML memories and the two levels of every bath
// mode in shared memory; the canonical arrays are touched only at the start and the end.
//
// One step, two phases separated by barriers (the cluster barrier when the cluster has more
// than one CTA: a cell at a CTA boundary reads its neighbour's field from the other CTA's shared
// memory):
//   phase A  the D/E half-step of every cell with the soft source; Lorentz / Drude polarization
//            updates (Eq. Pz_1D_Lorentz), which are per cell and cheap;
//   phase B  the H half-step of every cell and, for Lorentz-Bath cells, the polarization and bath
//            updates (Eq. Pz_update-LB, Yzj_finite_difference).  H does not read P, so the bath
//            work shares the phase with H and needs no barrier of its own.
// Cells are dealt to threads round-robin over the CTA's whole range (cell l to thread l mod T),
// so per-run remainders do not pile up on the first threads.  A thread updates the bath of its
// Lorentz-Bath cells mode by mode (the mode's coefficients read once, the cells' bath sums in
// registers); bath state is laid out [level][mode][cell], so a warp reads consecutive words.
// Two-level recursions swap level slots by step parity.
//
// Energy records (every `every` steps): per segment of the CTA, the box sums of eps E^2, of the
// oscillator energy rho/dt^2 ((P^{n+3/2}-P^{n+1/2})^2 + (w0 dt)^2 P^2), of the bath energy and of
// H^2.  A thread accumulates in the state precision, a warp reduces by shuffles in that precision,
// and the warp partials are summed in FP64 in a fixed order.
//
// The step loop runs in chunks of kBatchChunk steps and touches no global memory inside a chunk:
// the chunk's source amplitudes (a host-computed table) are staged into shared memory before it,
// its energy records are buffered in shared memory and written out after it.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "batch.h"

namespace fdtdbath {

template <typename T>
struct BatchCtx {
  T* sE;
  T* sH;
  T* sm;           // dynamic shared memory, element view (P / Y blocks)
  T* psiE;         // per psi slot
  T* psiH;
  T* bE;
  T* cE;
  T* bH;
  T* cH;
  const T* coef;   // staged coefficient rows
  const T* remH;   // previous CTA's last H_y (distributed shared memory), or null
  const T* remE;   // next CTA's first E_x, or null
  T S, dt;
  int par;         // slot of P^{n+1/2} / Y^{n+1/2}
};

// l: this thread's next cell (cell l belongs to thread l mod T); runs are contiguous, so the
// cursor left by one run is the thread's first cell of the next.
template <typename T, bool INC, int KIND>
__device__ __forceinline__ void batch_phase_a(const BatchRun R, const BatchSeg G, const MatK<T>* smat,
                                              const BatchCtx<T>& c, T J, bool en, T& a0, T& a1, int& l) {
  const int len = R.l1 - R.l0;
  const T S = c.S, dt = c.dt;
  const int nt = (int)blockDim.x;
  for (; l < R.l1; l += nt) {
    const int i = l - R.l0;
    const T h = c.sH[l];
    T hm;
    if (l > G.l0) hm = c.sH[l - 1];
    else hm = G.link_left ? *c.remH : T(0);
    const T dzHy = h - hm;
    T curl;
    if (R.psiE) {
      const int q = R.psi0 + i;
      const T ps = c.bE[q] * c.psiE[q] + c.cE[q] * dzHy;
      c.psiE[q] = ps;
      curl = T(0) - (dzHy + ps);
    } else {
      curl = T(0) - dzHy;
    }
    const bool src = l == G.src_l;
    T e = c.sE[l];
    if (KIND == kRunVacuum) {
      e = e + S * curl;
      if (src) e = e + dt * J;
      if (en && R.inbox) a0 += e * e;
    } else {
      const MatK<T> M = smat[R.mslot];            // by value: registers, not shared-memory reloads
      T* Pc = c.sm + R.p0 + c.par * len;          // P^{n+1/2}
      T* Po = c.sm + R.p0 + (c.par ^ 1) * len;    // P^{n-1/2}, receives P^{n+3/2}
      const T Pa = Pc[i], Pb = Po[i];
      if (!INC) {
        T* Dp = c.sm + R.p0 + 2 * len;
        T D = Dp[i] + S * curl;
        if (src) D = D + dt * J;
        Dp[i] = D;
        e = M.inv_eps * (D - Pa);
      } else {
        T inc = S * curl;
        if (src) inc = inc + dt * J;
        e = e + (inc - (Pa - Pb)) * M.inv_eps;
      }
      if (KIND == kRunOsc) {
        T Pn, Vn;
        if (!INC) {
          const T num = M.cE * e - M.c1m * Pa - M.c2 * Pb;
          Pn = M.inv_A * num;
          Vn = Pn - Pa;
        } else {
          const T num = M.cE * e - M.W * Pa + M.c2 * (Pa - Pb);
          Vn = num * M.inv_A;
          Pn = Pa + Vn;
        }
        Po[i] = Pn;
        if (en && R.inbox) a1 += M.rho_idt2 * (Vn * Vn + M.w0r2dt2 * Pn * Pn);
      }
      if (en && R.inbox) a0 += M.eps * (e * e);
    }
    c.sE[l] = e;
  }
}

// Phase B, H half-step of one run.
template <typename T>
__device__ __forceinline__ void batch_phase_h(const BatchRun R, const BatchSeg G, const BatchCtx<T>& c,
                                              bool en, T& a3, int& l) {
  const T S = c.S;
  const int nt = (int)blockDim.x;
  for (; l < R.l1; l += nt) {
    const T e = c.sE[l];
    T ep;
    if (l + 1 < G.l1) ep = c.sE[l + 1];
    else ep = G.link_right ? *c.remE : T(0);
    const T dzEx = ep - e;
    T h = c.sH[l];
    if (R.psiH) {
      const int q = R.psi0 + (l - R.l0);
      const T ps = c.bH[q] * c.psiH[q] + c.cH[q] * dzEx;
      c.psiH[q] = ps;
      h = h - S * ((dzEx + ps) - T(0));
    } else {
      h = h - S * (dzEx - T(0));
    }
    c.sH[l] = h;
    if (en && R.inbox) a3 += h * h;
  }
}

// Phase B, Lorentz-Bath polarization and bath update of one run.  The thread owns the run's cells
// i = i0 + k T (k < K <= KMAX), the same cells as in the other phases.  Modes are the outer loop so
// each mode's coefficient row is read once per thread; per-cell bath sums live in registers.  The
// sums run over j in ascending order, the order of Eq. Pz_update-LB as the FP64 oracle evaluates it.
template <typename T, bool INC, int KMAX>
__device__ __forceinline__ void batch_phase_bath(const BatchRun R, const MatK<T>* smat, const BatchCtx<T>& c,
                                                 bool en, T& a1, T& a2) {
  const int len = R.l1 - R.l0, nb = R.nb, nt = (int)blockDim.x;
  int i0 = ((int)threadIdx.x - R.l0) % nt;
  if (i0 < 0) i0 += nt;
  const int K = i0 < len ? (len - 1 - i0) / nt + 1 : 0;
  const MatK<T> M = smat[R.mslot];
  const T* cfm = c.coef + M.coef_off * kCoefStride;
  const T dt = c.dt;
  T* Pc = c.sm + R.p0 + c.par * len;
  T* Po = c.sm + R.p0 + (c.par ^ 1) * len;
  const T* Yc = c.sm + R.y0 + c.par * nb * len;   // Y^{n+1/2}   [mode][cell]
  T* Yo = c.sm + R.y0 + (c.par ^ 1) * nb * len;   // Y^{n-1/2}, receives Y^{n+3/2}
  T ub = T(0);
  for (int kb = 0; kb < K; kb += KMAX) {   // blocks of KMAX cells of this thread
    const int Kc = min(KMAX, K - kb);
    T acc[KMAX];
  #pragma unroll
    for (int k = 0; k < KMAX; ++k) acc[k] = T(0);
    for (int j = 0; j < nb; ++j) {
      const T* cf = cfm + j * kCoefStride;
      const T c0 = cf[0], c1 = cf[1], c2 = cf[2];
  #pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k < Kc) {
          const int i = i0 + (kb + k) * nt;
          const T y = Yc[j * len + i], ym = Yo[j * len + i];
          if (!INC) acc[k] = bath_sum_lit(acc[k], c0, c1, c2, y, ym);   // k_j (a_j Y^n + b_j Y^{n-1})
          else acc[k] = acc[k] + (c0 * y + c1 * (y - ym));       // k_j ((a_j+b_j) Y - b_j V)
        }
      }
    }
    // polarization; acc becomes the increment P^{n+3/2} - P^{n-1/2} the bath update needs
  #pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (k < Kc) {
        const int i = i0 + (kb + k) * nt;
        const T e = c.sE[R.l0 + i], Pa = Pc[i], Pb = Po[i];
        T Pn, Vn;
        if (!INC) {
          T num = M.cE * e - M.c1m * Pa - M.c2 * Pb;
          num = num - T(0.5) * dt * acc[k];
          Pn = M.inv_A * num;
          Vn = Pn - Pa;
          acc[k] = Pn - Pb;
        } else {
          const T V0 = Pa - Pb;
          T num = M.cE * e - M.W * Pa + M.c2 * V0;
          num = num - T(0.5) * dt * acc[k];
          Vn = num * M.inv_A;
          Pn = Pa + Vn;
          acc[k] = Vn + V0;
        }
        Po[i] = Pn;
        if (en && R.inbox) a1 += M.rho_idt2 * (Vn * Vn + M.w0r2dt2 * Pn * Pn);
      }
    }
    for (int j = 0; j < nb; ++j) {
      const T* cf = cfm + j * kCoefStride;
      const T c1 = cf[1], c2 = cf[2], c3 = cf[3], c4 = cf[4], c5 = cf[5];
  #pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k < Kc) {
          const int i = i0 + (kb + k) * nt;
          const T y = Yc[j * len + i], ym = Yo[j * len + i];
          T Yn, Vy;
          if (!INC) {
            Yn = bath_new_lit(c1, c3, c4, y, ym, acc[k]);
            Vy = Yn - y;
          } else {
            Vy = c2 * y + c3 * (y - ym) + c4 * acc[k];
            Yn = y + Vy;
          }
          Yo[j * len + i] = Yn;
          if (en) ub = INC ? ub + (Vy * Vy + c5 * Yn * Yn) : bath_energy_lit(ub, Vy, c5, Yn);
        }
      }
    }
  }
  if (en && R.inbox) a2 += M.rho_idt2 * ub;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, bool INC>
__global__ void __launch_bounds__(kBatchMaxThreads) batch1d_kernel(const BatchParams<T> p) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ BatchCta sc;
  __shared__ BatchSeg sseg[kBatchMaxSeg];
  __shared__ BatchRun srun[kBatchMaxRun];
  __shared__ MatK<T> smat[kBatchMaxMat];
  __shared__ double sredA[kBatchMaxSeg][kBatchMaxWarps][2];  // per warp: eps E^2, Lorentz/Drude P energy
  __shared__ double sredB[kBatchMaxSeg][kBatchMaxWarps][3];  // per warp: bath-layer P energy, bath, H^2
  __shared__ T sJ[kBatchChunk][kBatchMaxSeg];                // source amplitude per step of the chunk
  __shared__ double srec[kBatchChunk][kBatchMaxSeg][4];      // energy records of the chunk
  __shared__ int scoef0[kBatchMaxMat];

  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nwarp = nt >> 5;
  const int cta = blockIdx.x;

  // ---- descriptors into shared memory ----
  if (t == 0) sc = p.ctas[cta];
  __syncthreads();
  const int nseg = sc.nseg, nrun = sc.nrun, nmat = sc.nmat;
  for (int i = t; i < nseg; i += nt) sseg[i] = p.segs[sc.seg0 + i];
  for (int i = t; i < nrun; i += nt) srun[i] = p.runs[sc.run0 + i];
  for (int i = t; i < nmat; i += nt) smat[i] = p.mats[p.matslot[sc.mat0 + i]];
  __syncthreads();
  if (t == 0) {
    int row = 0;
    for (int s = 0; s < nmat; ++s) {
      scoef0[s] = row;
      row += smat[s].kind == kLorentzBath ? smat[s].nb : 0;
    }
  }
  __syncthreads();
  T* scoef = reinterpret_cast<T*>(dsm + sc.off_coef);
  for (int s = 0; s < nmat; ++s) {
    const int nbs = smat[s].kind == kLorentzBath ? smat[s].nb : 0;
    const T* src = p.coef + smat[s].coef_off * kCoefStride;
    for (int i = t; i < nbs * kCoefStride; i += nt) scoef[scoef0[s] * kCoefStride + i] = src[i];
  }
  __syncthreads();
  if (t < nmat) smat[t].coef_off = scoef0[t];

  BatchCtx<T> c;
  c.sE = reinterpret_cast<T*>(dsm + sc.off_E);
  c.sH = reinterpret_cast<T*>(dsm + sc.off_H);
  c.sm = reinterpret_cast<T*>(dsm + sc.off_P);
  c.psiE = reinterpret_cast<T*>(dsm + sc.off_psi);
  c.psiH = c.psiE + sc.npsi;
  c.bE = c.psiH + sc.npsi;
  c.cE = c.bE + sc.npsi;
  c.bH = c.cE + sc.npsi;
  c.cH = c.bH + sc.npsi;
  c.coef = scoef;
  c.S = p.S;
  c.dt = p.dt;
  c.par = 0;
  c.remH = nullptr;
  c.remE = nullptr;
  if (C > 1) {
    // the neighbours' arrays sit at their own offsets: H_y at the previous CTA's off_H, E_x at
    // offset 0 of the next CTA
    if (nseg > 0 && sseg[0].link_left && rank > 0)
      c.remH = reinterpret_cast<const T*>(cluster.map_shared_rank(dsm, rank - 1) + sc.prev_off_H) +
               (sc.prev_ncell - 1);
    if (nseg > 0 && sseg[nseg - 1].link_right && rank + 1 < C)
      c.remE = reinterpret_cast<const T*>(cluster.map_shared_rank(dsm, rank + 1));
  }

  // ---- state into shared memory ----
  for (int r = 0; r < nrun; ++r) {
    const BatchRun R = srun[r];
    const BatchSeg& G = sseg[R.seg];
    const int len = R.l1 - R.l0;
    for (int l = R.l0 + t; l < R.l1; l += nt) {
      const int i = l - R.l0;
      const int64_t g = G.g0 + (l - G.l0);
      c.sE[l] = p.E[g];
      c.sH[l] = p.H[g];
      if (R.psiE || R.psiH) {
        const int q = R.psi0 + i;
        c.psiE[q] = p.psiE[g];
        c.psiH[q] = p.psiH[g];
        c.bE[q] = p.bE[g];
        c.cE[q] = p.cE[g];
        c.bH[q] = p.bH[g];
        c.cH[q] = p.cH[g];
      }
      if (R.kind != kRunVacuum) {
        c.sm[R.p0 + i] = p.P[g];
        c.sm[R.p0 + len + i] = p.PM[g];
        if (!INC) c.sm[R.p0 + 2 * len + i] = p.D[g];
      }
    }
    if (R.kind == kRunBath) {
      // bath block [level][cell][mode] from the canonical [mode][cell] arrays
      const MatK<T>& M = smat[R.mslot];
      const int64_t yg = M.ybase + (G.z0 + (R.l0 - G.l0) - M.zlo);
      for (int q = t; q < len * R.nb; q += nt) {
        const int j = q / len, i = q - j * len;
        c.sm[R.y0 + q] = p.Y0[yg + (int64_t)j * M.ncell + i];
        c.sm[R.y0 + R.nb * len + q] = p.Y1[yg + (int64_t)j * M.ncell + i];
      }
    }
  }

  const int64_t step0 = *p.ctr;
  int ephase = (int)(step0 % p.every);
  int ering = (int)((step0 / p.every) % p.ring_cap);
  if (C > 1) cluster.sync();   // the shared state must be complete before a neighbour reads it
  else __syncthreads();
  for (int s0 = 0; s0 < p.nsteps; s0 += kBatchChunk) {
    const int m = min(kBatchChunk, p.nsteps - s0);
    const int64_t n0 = step0 + s0;
    for (int i = t; i < m * nseg; i += nt) {
      const int sg = i / m, k = i - sg * m;
      const BatchSeg& G = sseg[sg];
      sJ[k][sg] = (G.src_l >= 0 && n0 + k < G.src_len) ? (T)p.src_tab[G.src_off + n0 + k] : T(0);
    }
    __syncthreads();
    const int ering0 = ering;
    int nrec = 0;        // energy records of this chunk so far
    bool en_prev = false;
    for (int k = 0; k < m; ++k) {
      const bool en = p.energy_on && ephase == 0;
      // phase-B sums of the previous step, complete since the last barrier
      if (en_prev && t < 3 * nseg) {
        const int sg = t / 3, q = t - 3 * sg;
        double v = 0.0;
        for (int w = 0; w < nwarp; ++w) v += sredB[sg][w][q];
        if (q == 0) srec[nrec - 1][sg][1] += v;
        else srec[nrec - 1][sg][q + 1] = v;
      }
      // ---------------- phase A: D/E half-step, Lorentz / Drude polarization ----------------
      {
        T a0 = T(0), a1 = T(0);
        int cur = -1, l = t;
        for (int r = 0; r < nrun; ++r) {
          // off the energy steps a thread skips the runs that hold none of its cells (l is its
          // next cell; on energy steps every lane walks every run for the per-segment warp sums)
          if (!en && l >= srun[r].l1) continue;
          const BatchRun R = srun[r];
          if (en && R.seg != cur) {
            if (cur >= 0) {
              a0 = warp_sum(a0);
              a1 = warp_sum(a1);
              if (lane == 0) {
                sredA[cur][warp][0] = (double)a0;
                sredA[cur][warp][1] = (double)a1;
              }
            }
            cur = R.seg;
            a0 = a1 = T(0);
          }
          const BatchSeg G = sseg[R.seg];
          const T J = sJ[k][R.seg];
          if (R.kind == kRunVacuum) batch_phase_a<T, INC, kRunVacuum>(R, G, smat, c, J, en, a0, a1, l);
          else if (R.kind == kRunOsc) batch_phase_a<T, INC, kRunOsc>(R, G, smat, c, J, en, a0, a1, l);
          else batch_phase_a<T, INC, kRunBath>(R, G, smat, c, J, en, a0, a1, l);
        }
        if (en && cur >= 0) {
          a0 = warp_sum(a0);
          a1 = warp_sum(a1);
          if (lane == 0) {
            sredA[cur][warp][0] = (double)a0;
            sredA[cur][warp][1] = (double)a1;
          }
        }
      }
      if (C > 1) cluster.sync();
      else __syncthreads();
      if (en && t < 2 * nseg) {
        const int sg = t >> 1, q = t & 1;
        double v = 0.0;
        for (int w = 0; w < nwarp; ++w) v += sredA[sg][w][q];
        srec[nrec][sg][q] = v;
      }
      // ---------------- phase B: H half-step, Lorentz-Bath polarization and bath ----------------
      {
        T a1 = T(0), a2 = T(0), a3 = T(0);
        int cur = -1, l = t;
        for (int r = 0; r < nrun; ++r) {
          // off the energy steps a thread skips the runs that hold none of its cells (l is its
          // next cell; on energy steps every lane walks every run for the per-segment warp sums)
          if (!en && l >= srun[r].l1) continue;
          const BatchRun R = srun[r];
          if (en && R.seg != cur) {
            if (cur >= 0) {
              a1 = warp_sum(a1);
              a2 = warp_sum(a2);
              a3 = warp_sum(a3);
              if (lane == 0) {
                sredB[cur][warp][0] = (double)a1;
                sredB[cur][warp][1] = (double)a2;
                sredB[cur][warp][2] = (double)a3;
              }
            }
            cur = R.seg;
            a1 = a2 = a3 = T(0);
          }
          batch_phase_h<T>(R, sseg[R.seg], c, en, a3, l);
          if (R.kind == kRunBath) {
            const int kc = (R.l1 - R.l0 + nt - 1) / nt;   // cells of the run per thread
            if (kc <= 2) batch_phase_bath<T, INC, 2>(R, smat, c, en, a1, a2);
            else if (kc <= 4) batch_phase_bath<T, INC, 4>(R, smat, c, en, a1, a2);
            else if (kc <= 8) batch_phase_bath<T, INC, 8>(R, smat, c, en, a1, a2);
            else batch_phase_bath<T, INC, kBatchMaxCellsPerThread>(R, smat, c, en, a1, a2);
          }
        }
        if (en && cur >= 0) {
          a1 = warp_sum(a1);
          a2 = warp_sum(a2);
          a3 = warp_sum(a3);
          if (lane == 0) {
            sredB[cur][warp][0] = (double)a1;
            sredB[cur][warp][1] = (double)a2;
            sredB[cur][warp][2] = (double)a3;
          }
        }
      }
      if (C > 1) cluster.sync();
      else __syncthreads();
      c.par ^= 1;   // P^{n+3/2} / Y^{n+3/2} now sit in the other slot
      if (en) ++nrec;
      en_prev = en;
      if (++ephase == p.every) {
        ephase = 0;
        if (++ering == p.ring_cap) ering = 0;
      }
    }
    // the chunk's last phase-B sums, then its records out to the ring
    if (en_prev && t < 3 * nseg) {
      const int sg = t / 3, q = t - 3 * sg;
      double v = 0.0;
      for (int w = 0; w < nwarp; ++w) v += sredB[sg][w][q];
      if (q == 0) srec[nrec - 1][sg][1] += v;
      else srec[nrec - 1][sg][q + 1] = v;
    }
    __syncthreads();
    for (int i = t; i < nrec * nseg * 4; i += nt) {
      const int q = i & 3, sg = (i >> 2) % nseg, r = (i >> 2) / nseg;
      const int64_t ring = (ering0 + r) % p.ring_cap;
      p.partial[ring * p.ring_stride + sseg[sg].slot * 4 + q] = srec[r][sg][q];
    }
  }

  // ---- write the state back ----
  for (int r = 0; r < nrun; ++r) {
    const BatchRun R = srun[r];
    const BatchSeg& G = sseg[R.seg];
    const int len = R.l1 - R.l0;
    for (int l = R.l0 + t; l < R.l1; l += nt) {
      const int i = l - R.l0;
      const int64_t g = G.g0 + (l - G.l0);
      p.E[g] = c.sE[l];
      p.H[g] = c.sH[l];
      if (R.psiE || R.psiH) {
        const int q = R.psi0 + i;
        p.psiE[g] = c.psiE[q];
        p.psiH[g] = c.psiH[q];
      }
      if (R.kind != kRunVacuum) {
        p.P[g] = c.sm[R.p0 + c.par * len + i];
        p.PM[g] = c.sm[R.p0 + (c.par ^ 1) * len + i];
        if (!INC) p.D[g] = c.sm[R.p0 + 2 * len + i];
      }
    }
    if (R.kind == kRunBath) {
      const MatK<T>& M = smat[R.mslot];
      const int64_t yg = M.ybase + (G.z0 + (R.l0 - G.l0) - M.zlo);
      for (int q = t; q < len * R.nb; q += nt) {
        const int j = q / len, i = q - j * len;
        p.Y0[yg + (int64_t)j * M.ncell + i] = c.sm[R.y0 + c.par * R.nb * len + q];
        p.Y1[yg + (int64_t)j * M.ncell + i] = c.sm[R.y0 + (c.par ^ 1) * R.nb * len + q];
      }
    }
  }
  // no CTA may leave while a neighbour can still map its shared memory
  if (C > 1) cluster.sync();
}

template <typename T, bool INC>
int launch_batch1d_impl(const BatchParams<T>& p, int nctas, int cluster, int threads, int smem,
                        void* stream) {
  auto kern = batch1d_kernel<T, INC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, p);
  return (int)e;
}

template <typename T, bool INC>
int batch1d_occupancy_impl(int cluster, int threads, int smem, int* max_clusters, int* static_smem) {
  auto kern = batch1d_kernel<T, INC>;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return (int)e;
  *static_smem = (int)fa.sharedSizeBytes;
  *max_clusters = 0;
  if (threads > fa.maxThreadsPerBlock) return 0;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cluster);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  *max_clusters = n;
  return 0;
}

}  // namespace fdtdbath
