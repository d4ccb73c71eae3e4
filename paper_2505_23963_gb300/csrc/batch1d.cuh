// batch1d.cuh -- one persistent launch advancing a batch of independent x-polarized 1D cavities
// (the paper's 1D scheme, Eq. FDTD-1D with Eq. Pz_update-LB / Pz_1D_Lorentz /
// Yzj_finite_difference, Sec. II.C) for all steps of a call.
//
// The host packs the cavities into thread-block clusters and cuts each cluster's cells into one
// contiguous range per CTA (batch.h).  For the whole launch a CTA keeps its cells' E_x, H_y, the
// two levels of P_x (and D_x on the FP64 path), CPML memories and the two levels of every bath
// mode in shared memory; the canonical arrays are touched only at the start and the end.
//
// One step: the D/E half-step with the soft source, the polarization and bath updates of every
// run (typed: vacuum, Lorentz/Drude, Lorentz-Bath with N_b a template bound); a barrier; the H
// half-step; a barrier.  The barrier is the cluster barrier when the cluster has more than one CTA:
// a cell at a CTA boundary reads its neighbour's field from the other CTA's shared memory.
// Two-level recursions swap their level slots by step parity instead of copying.
//
// Energy records (every `every` steps): per segment of the CTA, the box sums of eps E^2, of the
// oscillator energy rho/dt^2 ((P^{n+3/2}-P^{n+1/2})^2 + (w0 dt)^2 P^2), of the bath energy and of
// H^2.  A thread accumulates in the state precision, a warp reduces by shuffles in that precision,
// and the warp partials are summed in FP64 in a fixed order.
//
// The source amplitude of each cavity comes from a host-computed table, staged into shared
// memory a chunk of steps at a time.
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

// D/E half-step of one run plus, for material runs, the polarization and bath updates.
// KIND: kRunVacuum, kRunOsc, kRunBath; NBC: compile-time bound on the run's bath modes.
template <typename T, bool INC, int KIND, int NBC>
__device__ __forceinline__ void batch_e_run(const BatchRun& R, const BatchSeg& G, const MatK<T>* smat,
                                            const BatchCtx<T>& c, T J, bool en, T& a0, T& a1, T& a2) {
  constexpr int NBA = NBC > 0 ? NBC : 1;
  const int len = R.l1 - R.l0;
  const T S = c.S, dt = c.dt;
  for (int l = R.l0 + (int)threadIdx.x; l < R.l1; l += (int)blockDim.x) {
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
      const MatK<T>& M = smat[R.mslot];
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
      T bsum = T(0);
      T Y[NBA], Ym[NBA];
      const int nb = KIND == kRunBath ? R.nb : 0;
      T* Yc = c.sm + R.y0 + c.par * nb * len + i;           // Y_j^{n+1/2} at Yc[j*len]
      T* Yo = c.sm + R.y0 + (c.par ^ 1) * nb * len + i;     // Y_j^{n-1/2}, receives Y_j^{n+3/2}
      const T* cfm = c.coef + M.coef_off * kCoefStride;
      if (KIND == kRunBath) {
#pragma unroll
        for (int j = 0; j < NBA; ++j) {
          Y[j] = T(0);
          Ym[j] = T(0);
          if (j < nb) {
            Y[j] = Yc[j * len];
            Ym[j] = Yo[j * len];
            const T* cf = cfm + j * kCoefStride;
            if (!INC) {
              bsum = bsum + cf[0] * (cf[1] * Y[j] + cf[2] * Ym[j]);   // k_j (a_j Y^n + b_j Y^{n-1})
            } else {
              const T Vj = Y[j] - Ym[j];
              bsum = bsum + (cf[0] * Y[j] + cf[1] * Vj);               // k_j ((a_j+b_j) Y - b_j V)
            }
          }
        }
      }
      T Pn, Vn, V0;
      if (!INC) {
        T num = M.cE * e - M.c1m * Pa - M.c2 * Pb;
        if (KIND == kRunBath) num = num - T(0.5) * dt * bsum;
        Pn = M.inv_A * num;
        Vn = Pn - Pa;
        V0 = Pa - Pb;
      } else {
        V0 = Pa - Pb;
        T num = M.cE * e - M.W * Pa + M.c2 * V0;
        if (KIND == kRunBath) num = num - T(0.5) * dt * bsum;
        Vn = num * M.inv_A;
        Pn = Pa + Vn;
      }
      Po[i] = Pn;
      T ub = T(0);
      if (KIND == kRunBath) {
        const T dP = Vn + V0;
#pragma unroll
        for (int j = 0; j < NBA; ++j) {
          if (j < nb) {
            const T* cf = cfm + j * kCoefStride;
            T Yn, Vy;
            if (!INC) {
              Yn = cf[1] * Y[j] + cf[3] * Ym[j] + cf[4] * (Pn - Pb);
              Vy = Yn - Y[j];
            } else {
              Vy = cf[2] * Y[j] + cf[3] * (Y[j] - Ym[j]) + cf[4] * dP;
              Yn = Y[j] + Vy;
            }
            Yo[j * len] = Yn;
            if (en) ub += Vy * Vy + cf[5] * Yn * Yn;
          }
        }
      }
      if (en && R.inbox) {
        a0 += M.eps * (e * e);
        a1 += M.rho_idt2 * (Vn * Vn + M.w0r2dt2 * Pn * Pn);
        a2 += M.rho_idt2 * ub;
      }
    }
    c.sE[l] = e;
  }
}

// H half-step of one run.
template <typename T>
__device__ __forceinline__ void batch_h_run(const BatchRun& R, const BatchSeg& G, const BatchCtx<T>& c,
                                            bool en, T& a3) {
  const T S = c.S;
  for (int l = R.l0 + (int)threadIdx.x; l < R.l1; l += (int)blockDim.x) {
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
  __shared__ double sredE[kBatchMaxSeg][kBatchMaxWarps][3];
  __shared__ double sredH[kBatchMaxSeg][kBatchMaxWarps];
  __shared__ T sJ[kBatchChunk][kBatchMaxSeg];          // source amplitude per step of the chunk
  __shared__ double srec[kBatchChunk][kBatchMaxSeg][4]; // energy records of the chunk
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
      if (R.kind == kRunBath) {
        const MatK<T>& M = smat[R.mslot];
        const int z = G.z0 + (l - G.l0);
        const int64_t yg = M.ybase + (z - M.zlo);
        for (int j = 0; j < R.nb; ++j) {
          c.sm[R.y0 + j * len + i] = p.Y0[yg + (int64_t)j * M.ncell];
          c.sm[R.y0 + (R.nb + j) * len + i] = p.Y1[yg + (int64_t)j * M.ncell];
        }
      }
    }
  }

  // The step loop runs in chunks of kBatchChunk steps.  Inside a chunk it touches no global
  // memory: the chunk's source amplitudes are staged into shared memory before it and its energy
  // records are buffered in shared memory and written out after it.  (A cluster barrier has
  // release semantics: a global access still in flight in any thread would hold the barrier for
  // its whole latency, every step.)
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
      // H-half sums of the previous step, complete since the last barrier
      if (en_prev && t < nseg) {
        double v = 0.0;
        for (int w = 0; w < nwarp; ++w) v += sredH[t][w];
        srec[nrec - 1][t][3] = v;
      }
      // ---------------- D/E half-step, polarization and bath ----------------
      {
        T a0 = T(0), a1 = T(0), a2 = T(0);
        int cur = -1;
        for (int r = 0; r < nrun; ++r) {
          const BatchRun& R = srun[r];
          if (en && R.seg != cur) {
            if (cur >= 0) {
              a0 = warp_sum(a0);
              a1 = warp_sum(a1);
              a2 = warp_sum(a2);
              if (lane == 0) {
                sredE[cur][warp][0] = (double)a0;
                sredE[cur][warp][1] = (double)a1;
                sredE[cur][warp][2] = (double)a2;
              }
            }
            cur = R.seg;
            a0 = a1 = a2 = T(0);
          }
          const BatchSeg& G = sseg[R.seg];
          const T J = sJ[k][R.seg];
          if (R.kind == kRunVacuum) {
            batch_e_run<T, INC, kRunVacuum, 0>(R, G, smat, c, J, en, a0, a1, a2);
          } else if (R.kind == kRunOsc) {
            batch_e_run<T, INC, kRunOsc, 0>(R, G, smat, c, J, en, a0, a1, a2);
          } else if (R.nb <= 4) {
            batch_e_run<T, INC, kRunBath, 4>(R, G, smat, c, J, en, a0, a1, a2);
          } else if (R.nb <= 8) {
            batch_e_run<T, INC, kRunBath, 8>(R, G, smat, c, J, en, a0, a1, a2);
          } else if (R.nb <= 16) {
            batch_e_run<T, INC, kRunBath, 16>(R, G, smat, c, J, en, a0, a1, a2);
          } else {
            batch_e_run<T, INC, kRunBath, 32>(R, G, smat, c, J, en, a0, a1, a2);
          }
        }
        if (en && cur >= 0) {
          a0 = warp_sum(a0);
          a1 = warp_sum(a1);
          a2 = warp_sum(a2);
          if (lane == 0) {
            sredE[cur][warp][0] = (double)a0;
            sredE[cur][warp][1] = (double)a1;
            sredE[cur][warp][2] = (double)a2;
          }
        }
      }
      if (C > 1) cluster.sync();
      else __syncthreads();
      c.par ^= 1;   // P^{n+3/2} / Y^{n+3/2} now sit in the other slot
      // ---------------- H half-step ----------------
      if (en && t < 3 * nseg) {
        const int sg = t / 3, q = t - 3 * sg;
        double v = 0.0;
        for (int w = 0; w < nwarp; ++w) v += sredE[sg][w][q];
        srec[nrec][sg][q] = v;
      }
      {
        T a3 = T(0);
        int cur = -1;
        for (int r = 0; r < nrun; ++r) {
          const BatchRun& R = srun[r];
          if (en && R.seg != cur) {
            if (cur >= 0) {
              a3 = warp_sum(a3);
              if (lane == 0) sredH[cur][warp] = (double)a3;
            }
            cur = R.seg;
            a3 = T(0);
          }
          batch_h_run<T>(R, sseg[R.seg], c, en, a3);
        }
        if (en && cur >= 0) {
          a3 = warp_sum(a3);
          if (lane == 0) sredH[cur][warp] = (double)a3;
        }
      }
      if (C > 1) cluster.sync();
      else __syncthreads();
      if (en) ++nrec;
      en_prev = en;
      if (++ephase == p.every) {
        ephase = 0;
        if (++ering == p.ring_cap) ering = 0;
      }
    }
    // the chunk's last H-half sums, then its records out to the ring
    if (en_prev && t < nseg) {
      double v = 0.0;
      for (int w = 0; w < nwarp; ++w) v += sredH[t][w];
      srec[nrec - 1][t][3] = v;
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
      if (R.kind == kRunBath) {
        const MatK<T>& M = smat[R.mslot];
        const int z = G.z0 + (l - G.l0);
        const int64_t yg = M.ybase + (z - M.zlo);
        for (int j = 0; j < R.nb; ++j) {
          p.Y0[yg + (int64_t)j * M.ncell] = c.sm[R.y0 + (c.par * R.nb + j) * len + i];
          p.Y1[yg + (int64_t)j * M.ncell] = c.sm[R.y0 + ((c.par ^ 1) * R.nb + j) * len + i];
        }
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
