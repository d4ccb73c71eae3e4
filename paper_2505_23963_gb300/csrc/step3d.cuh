// step3d.cuh -- fused Yee + CPML + source + Lorentz/Drude/Lorentz-Bath step, one launch per step.
//
// One launch performs, for every cell, the H half-step of the previous step (H^n from
// E^{n-1/2}, Eq. 1b) followed by this step's D/E half-step (Eq. 1a, D = E + P), the
// polarization update ("evaluate P^{n+3/2}" of Eq. FDTD-1D with Eq. Pz_1D_Lorentz or
// Eq. Pz_update-LB) and the bath-mode update (Eq. Yzj_finite_difference), with one
// independent bath set per P component (Sec. II.C, 3D extension).
//
// Decomposition: a CTA owns a TX x TY column tile in (x, y) and marches along a chunk of
// z planes.  Per plane it stages E^{n-1/2} of plane k+1 (tile + 1-cell frame) in shared
// memory, recomputes H^n on the tile plus the -x / -y halo (H is read by neighbours'
// E updates), writes H^n of its own cells, then updates E, P and the bath modes of its own
// cells with H^n of planes k (shared) and k-1 (registers).  E, H and the H-side CPML
// memories are double-buffered so neighbouring CTAs never see a half-updated plane;
// P, Y, D and the E-side CPML memories are cell-local and updated in place.  Every state
// word is read once and written once per step; halo re-reads hit L1/L2.
//
// Bath modes: up to 8 per component (FP32; 4 in FP64) the plane's bath state is loaded into
// registers before the stencil and the three components go through the modes together; up to
// 32 each component's modes are held in registers between the bath sum and the mode update;
// above 32 (up to 128) they are streamed from memory twice, in batches of 16.
//
// Tiles: 32 x 8 (32 x 1 when ny < 8); the TE form of y-invariant grids (ny = 1, E_y sources)
// uses 128 x 1 tiles and carries only E_y, H_x, H_z and the y polarization and bath modes.
//
// Two arithmetic forms:
//   INC = false (FP64): the literal form -- D stored in material cells, E = (D - P)/eps,
//     two time levels of P and Y with the new level overwriting the oldest; every
//     expression is evaluated in the order the equations print it.
//   INC = true (FP32): increment arithmetic on the same two stored levels -- E updated D-free
//     (E += (dt curl H + dt J - V)/eps with V = P^{n+1/2} - P^{n-1/2}), and P and every Y_j
//     advanced through their increment, X^{n+1} = X^n + V^{n+1}, written over X^{n-1}.
//     Algebraically identical to Eq. Pz_update-LB / Yzj_finite_difference but without
//     representing 2 - w^2 dt^2, whose FP32 rounding would shift every oscillator frequency.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace fdtdbath {

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ int psiE_plane(int k, int nz, int npml) {
  if (k < npml) return k;
  if (k >= nz - npml) return npml + (k - (nz - npml));
  return -1;
}
__device__ __forceinline__ int psiH_plane(int k, int nz, int npml) {
  if (npml <= 0) return -1;
  if (k < npml) return k;
  if (k >= nz - npml - 1) return npml + (k - (nz - npml - 1));
  return -1;
}

// Fixed-order block reduction; the result (FP64) is valid in thread 0.  Within a warp the sum runs
// in the argument's precision (FP64 arithmetic is slow on this part), across warps in FP64.
template <typename V>
__device__ __forceinline__ double block_sum(V v, double* scratch) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((tid & 31) == 0) scratch[tid >> 5] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (int w = 0; w < nw; ++w) s += scratch[w];
  return s;
}

// H update of one cell (Eq. 1b, mu0 = 1) from the 9 E values it needs, in the form of
// Eq. FDTD-1D (S = dt/dx times differences of neighbours):
//   Hx -= S (dEz|y - (dEy|z + psi_x)),  Hy -= S ((dEx|z + psi_y) - dEz|x),  Hz -= S (dEy|x - dEx|y);
// psi <- b psi + c dE|z inside the CPML (memory in units of a field difference).
// Warp-wide sum of v written by lane 0 to dst (skipped when dst is null), as the one-warp
// block_sum would produce it (0.0 + the warp's sum).
template <typename V>
__device__ __forceinline__ void warp_sum_to(V v, double* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && dst) *dst = 0.0 + (double)v;
}

template <typename T>
struct HIn {
  T ex0, ex_k1, ex_j1;  // Ex(i,j,k), Ex(i,j,k+1), Ex(i,j+1,k)
  T ey0, ey_k1, ey_i1;  // Ey(i,j,k), Ey(i,j,k+1), Ey(i+1,j,k)
  T ez0, ez_j1, ez_i1;  // Ez(i,j,k), Ez(i,j+1,k), Ez(i+1,j,k)
};

template <typename T>
__device__ __forceinline__ void h_update(const HIn<T>& e, T& hx, T& hy, T& hz, T* psix, T* psiy,
                                         T b, T c, bool pml, T S) {
  const T dyEz = e.ez_j1 - e.ez0;
  const T dzEy = e.ey_k1 - e.ey0;
  const T dzEx = e.ex_k1 - e.ex0;
  const T dxEz = e.ez_i1 - e.ez0;
  const T dxEy = e.ey_i1 - e.ey0;
  const T dyEx = e.ex_j1 - e.ex0;
  if (pml) {
    *psix = b * (*psix) + c * dzEy;
    *psiy = b * (*psiy) + c * dzEx;
    hx = hx - S * (dyEz - (dzEy + *psix));
    hy = hy - S * ((dzEx + *psiy) - dxEz);
  } else {
    hx = hx - S * (dyEz - dzEy);
    hy = hy - S * (dzEx - dxEz);
  }
  hz = hz - S * (dxEy - dyEx);
}

// cp.async (LDGSTS) of one element into shared memory, and its group bookkeeping
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(sizeof(T)));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Depth of the plane pipeline: the E_in frame of plane k+kAheadE and the H_in frame of plane
// k+kAheadE-1 are requested while plane k is computed; kAheadE-1 commit groups stay in flight.
constexpr int kAheadE = 4;
constexpr int kRingE = 6;   // E frames: k-1 (still read by the E update of k-1), k .. k+kAheadE
constexpr int kRingH = 4;   // H frames: k .. k+kAheadE-1

// plane-info bits of the per-chunk table
enum : int { kPlaneMat = 0xF, kPlaneEbox = 0x10, kPlaneMonE = 0x20, kPlaneMonH = 0x40, kPlaneSrc = 0x80 };

template <typename T>
__device__ __forceinline__ void cp_async16(T* sdst, const T* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc));
}

// the six coefficients of a bath-mode row, read with vector shared-memory loads
__device__ __forceinline__ void load_coef6(const float* cf, float* o) {
  const float4 a = *reinterpret_cast<const float4*>(cf);
  const float2 b = *reinterpret_cast<const float2*>(cf + 4);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
}
__device__ __forceinline__ void load_coef6(const double* cf, double* o) {
  const double2 a = *reinterpret_cast<const double2*>(cf);
  const double2 b = *reinterpret_cast<const double2*>(cf + 2);
  const double2 c = *reinterpret_cast<const double2*>(cf + 4);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y; o[4] = c.x; o[5] = c.y;
}

// Shared-memory frames of one plane.  Rows start 16-byte aligned at x0-4 so that whole rows
// can be staged with 16-byte copies: the E frame spans x0-4 .. x0+35 (the tile, one halo cell
// on each side, padding) and rows y0-1 .. y0+TY; the H frame spans x0-4 .. x0+31 and rows
// y0-1 .. y0+TY-1 (the tile and its -x / -y halo).  Frame column = x - (x0 - 4), so the
// halo-relative column hx (x = x0-1+hx) sits at hx + kXO.
constexpr int kXO = 3;
template <int TY, int TXW = kTX>
struct Tile {
  static constexpr int TX = TXW, FX = TXW + 8, FY = TY + 2, HX = TXW + 4, HY = TY + 1;
  static constexpr int NTHR = TXW * TY;
  static constexpr int FE = FY * FX;                 // E frame elements per component
  static constexpr int FH = HY * HX;                 // H frame elements per component
};

// Bath-mode storage: the state precision (two levels Y^n, Y^{n-1} in two arrays: load2 reads
// both, put writes the new level over the older one), or bf16 pairs (value Y and increment
// V = Y^n - Y^{n-1} of a mode side by side in one 32-bit word, updated in place by put_pair;
// the arithmetic stays FP32).
template <typename T, bool YB>
struct BathStore {
  using S = T;
  static __device__ __forceinline__ T load(const S* p) { return *p; }
  static __device__ __forceinline__ void load2(const S* pa, const S* pb, T& a, T& b) {
    a = *pa;
    b = *pb;
  }
  static __device__ __forceinline__ void put(S* p, T v) { *p = v; }
  static __device__ __forceinline__ void put_pair(S* p, T y, T v) { *p = y; }   // not used
};
template <>
struct BathStore<float, true> {
  using S = __nv_bfloat162;
  static __device__ __forceinline__ void load2(const S* pa, const S*, float& y, float& v) {
    const __nv_bfloat162 q = *pa;
    y = __low2float(q);
    v = __high2float(q);
  }
  static __device__ __forceinline__ void put(S* p, float v) {}   // not used
  static __device__ __forceinline__ void put_pair(S* p, float y, float v) {
    *p = __halves2bfloat162(__float2bfloat16_rn(y), __float2bfloat16_rn(v));
  }
};

template <typename T, int NBMAX, int TY, int TXW = kTX>
struct StepBounds {
  static constexpr int threads = TXW * TY;
  // wide single-row tiles (the TE form, 9 KB of frames per CTA): eight CTAs of TXW threads per SM
  // for the bath-free kernel, five with up to 8 bath modes, four otherwise
  static constexpr int min_blocks = TXW > kTX ? (NBMAX == 0 ? 8 : (NBMAX <= 8 ? 5 : 4))
      : (TY == 8 ? (NBMAX == 0 ? (sizeof(T) == 4 ? 4 : 2) : ((sizeof(T) == 8 && NBMAX >= 16) ? 1 : 2)) : 8);
};

template <typename T, bool INC, int NBMAX, int TY, bool YB = false, bool TE = false, int TXW = kTX>
__global__ void __launch_bounds__(StepBounds<T, NBMAX, TY, TXW>::threads, StepBounds<T, NBMAX, TY, TXW>::min_blocks)
step3d_kernel(const Step3DParams<T> p) {
  // TE: a y-invariant grid (ny = 1) driven only through E_y, whose E_x, E_z, H_y, P_x, P_z and
  // x / z bath modes are exactly zero at every step (the host checks that they start at zero and
  // that nothing writes them).  Those components are constants here: never staged, loaded or
  // stored, and every expression that uses one sees T(0), so the live components come out
  // bit-identical to the general form's.
  auto liveE = [](int c) { return !TE || c == 1; };   // E, P, bath components carried
  auto liveH = [](int c) { return !TE || c != 1; };   // H components carried
  // With ny = 1 the TE form needs no y neighbour (the y-differences it keeps are of E_x, E_z,
  // H_y, all zero): of the frames it stages only the tile's own row, and of the halo only the
  // -x column.
  using YS = BathStore<T, YB>;   // bath-mode storage (YB: bf16 value / increment pairs)
  using YT = typename YS::S;
  using G = Tile<TY, TXW>;
  constexpr int TX = G::TX, FX = G::FX, HX = G::HX, NTHR = G::NTHR;
  // Stored frames.  The general form keeps the three components of E rows y0-1 .. y0+TY and of H
  // rows y0-1 .. y0+TY-1; the TE form only the tile's own row of E_y and of H_x, H_z.  RO is the
  // first stored frame row, FE / FH the stored elements per component, eo / ho component offsets.
  constexpr int RO = TE ? 1 : 0;
  constexpr int FE = TE ? FX : G::FE, FH = TE ? HX : G::FH;
  constexpr int NEC = TE ? 1 : 3, NHC = TE ? 2 : 3;   // stored components per frame slot
  auto eo = [](int c) { return TE ? 0 : c * FE; };
  auto ho = [](int c) { return TE ? (c == 2 ? FH : 0) : c * FH; };
  constexpr int FY = G::FY, HY = G::HY;
  constexpr int VE = 16 / (int)sizeof(T);      // elements per 16-byte copy
  constexpr int NCE = FY * (FX / VE), NCH = HY * (HX / VE);   // 16-byte chunks per frame component
  constexpr int CE = (NCE + NTHR - 1) / NTHR, CH = (NCH + NTHR - 1) / NTHR;
  // bath modes preloaded for all three components with the rest of the plane's state
  constexpr int NBP = NBMAX <= (sizeof(T) == 4 ? 8 : 4) ? NBMAX : 0;
  constexpr int NBA = NBMAX > 0 ? NBMAX : 1;
  constexpr bool kStream = NBMAX > 32;   // bath modes streamed from memory (N_b up to kMaxBathStep)
  constexpr int kStreamBatch = 16;      // modes whose loads are issued together when streaming
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // E_in frames, ring of kRingE planes [kRingE][3][FE]: planes k, k+1 feed H^n(k), plane k
  // also the E update of k (after the second barrier), planes up to k+kAheadE are in flight;
  // the slot refilled at the top of step k+1 held plane k+1+kAheadE-kRingE <= k-1, last read
  // before this step's first barrier.  H_in frames likewise, ring of kRingH planes.
  T* sE = reinterpret_cast<T*>(smem_raw);
  T* sHin = sE + kRingE * NEC * FE;              // H_in frames: [kRingH][3][FH]
  T* sH = sHin + kRingH * NHC * FH;              // H^n of the current plane: [3][FH]
  T* sCoef = sH + NHC * FH;                      // bath coefficients:            [modes][8]
  int* sInfo = reinterpret_cast<int*>(sCoef + kCoefStride * p.nmodes);   // [kMaxChunk]
  double* sred = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(sInfo + kMaxChunk) + 15) & ~uintptr_t(15));

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int i = x0 + tx, j = y0 + ty;
  const bool own = (i < p.nx) && (j < p.ny);
  const int chunk = p.chunk_ids[blockIdx.z];
  const int zb = p.zstart[chunk], ze = p.zstart[chunk + 1];
  // every array index fits in 32 bits (checked when the simulation is created)
  const int plane = (int)p.plane, ncell = (int)p.ncell;
  const int qxy = own ? j * p.nx + i : 0;
  const T dt = p.dt, S = p.S;
  // partial-sum slots: p.nbxy per z-chunk and quantity, one per tile of the 32 x TYS tiling
  // (TYS = 8, or 1 for grids with fewer than 8 rows) whatever this launch's tile height: a block of
  // a taller tile writes its sum into the slot of its first TYS-row tile and zero into the others,
  // so every slot of a chunk is rewritten by whichever kernel processes the chunk
  constexpr int TYS = TY >= 8 ? 8 : TY;
  constexpr int RS = TY / TYS;                       // slot rows per block (TYS-row tiles)
  constexpr int WS = TX / kTX;                       // slot columns per block (32-wide tiles)
  const int nbxy = p.nbxy;
  // 32-wide tiles along x: the launch's blocks, or WS of them per block of wide tiles
  const int ncol_s = WS == 1 ? (int)gridDim.x : (p.nx + kTX - 1) / kTX;
  const int nrow_s = nbxy / ncol_s;                  // TYS-row tiles along y
  const int sx0 = blockIdx.x * WS, sy0 = blockIdx.y * RS;
  const int bxy = sy0 * ncol_s + sx0;
  auto put_slot = [&](double* row, double v) {      // row: slot 0 of this chunk's quantity
    row[bxy] = v;
#pragma unroll
    for (int r = 1; r < RS; ++r)
      if (sy0 + r < nrow_s) row[bxy + r * ncol_s] = 0.0;
#pragma unroll
    for (int w = 1; w < WS; ++w)   // wide tiles are single-row (RS = 1)
      if (sx0 + w < ncol_s) row[bxy + w] = 0.0;
  };
  // Wide single-row tiles write one warp sum per 32-wide slot tile (warp_sum_to): a warp is one
  // such tile and its value is the one a 32-wide block produces, so the sums and their order do
  // not depend on the tile width.  wslot(row): this warp's slot of row, or null.
  static_assert(WS == 1 || TY == 1, "wide tiles are single-row");
  auto wslot = [&](double* row) -> double* {
    const int w = tid >> 5;
    return (row && sx0 + w < ncol_s) ? row + bxy + w : nullptr;
  };
  const T* __restrict__ Ein = p.Ein;
  const T* __restrict__ Hin = p.Hin;

  for (int q = tid; q < kCoefStride * p.nmodes; q += NTHR) sCoef[q] = p.coef[q];

  // per-plane facts of this chunk: material index + 1, energy box, monitor and source planes
  for (int t = tid; t < ze - zb; t += NTHR) {
    const int k = zb + t;
    int info = 0;
    for (int m = 0; m < p.nmat; ++m)
      if (k >= p.mat[m].zlo && k < p.mat[m].zhi) info = m + 1;
    if (k >= p.ebox_lo && k < p.ebox_hi) info |= kPlaneEbox;
    for (int m = 0; m < p.nmon; ++m) {
      if (k == p.mon_z[m]) info |= kPlaneMonE;
      if (k == p.mon_z[m] || k == p.mon_z[m] - 1) info |= kPlaneMonH;
    }
    for (int q = 0; q < p.nsrc; ++q)
      if (k == p.src_z[q]) info |= kPlaneSrc;
    sInfo[t] = info;
  }

  // 16-byte chunks this thread stages every plane (when nx is a multiple of VE): frame offset
  // and periodic (x, y) offset of the chunk's first element; E chunks from the low threads up,
  // H chunks from the high threads down
  int ce_s[CE], ce_g[CE], ch_s[CH], ch_g[CH];
  constexpr int cpr_e = FX / VE, cpr_h = HX / VE;
#pragma unroll
  for (int r = 0; r < CE; ++r) {
    const int idx = tid + r * NTHR;
    ce_s[r] = -1;
    ce_g[r] = 0;
    if (idx < (TE ? cpr_e : NCE) && p.vec16) {
      const int yy = TE ? 1 : idx / cpr_e, cx = TE ? idx : idx - yy * cpr_e;   // TE: own row only
      ce_s[r] = (yy - RO) * FX + cx * VE;
      ce_g[r] = wrapi(y0 - 1 + yy, p.ny) * p.nx + wrapi(x0 - 4 + cx * VE, p.nx);
    }
  }
#pragma unroll
  for (int r = 0; r < CH; ++r) {
    const int idx = (NTHR - 1 - tid) + r * NTHR;
    ch_s[r] = -1;
    ch_g[r] = 0;
    if (idx < (TE ? cpr_h : NCH) && p.vec16) {
      const int yy = TE ? 1 : idx / cpr_h, cx = TE ? idx : idx - yy * cpr_h;   // TE: own row only
      ch_s[r] = (yy - RO) * HX + cx * VE;
      ch_g[r] = wrapi(y0 - 1 + yy, p.ny) * p.nx + wrapi(x0 - 4 + cx * VE, p.nx);
    }
  }

  // H tasks of this thread: its own cell, and up to two cells of the -y row / -x column halo
  const int own_fe = (ty + 1 - RO) * FX + (tx + 1 + kXO), own_fh = (ty + 1 - RO) * HX + (tx + 1 + kXO);
  // (TE: the -x column only)
  constexpr int NHALO = TE ? TY : TX + TY;
  constexpr int NHT = (NHALO + NTHR - 1) / NTHR;
  int ht_fe[NHT], ht_fh[NHT], ht_g[NHT];
#pragma unroll
  for (int r = 0; r < NHT; ++r) {
    const int t = tid + r * NTHR;
    ht_fe[r] = -1;
    ht_fh[r] = 0;
    ht_g[r] = 0;
    if (t < NHALO) {
      const int hy = TE ? t + 1 : (t < TX ? 0 : t - TX + 1), hx = TE ? 0 : (t < TX ? t + 1 : 0);
      ht_fe[r] = (hy - RO) * FX + hx + kXO;
      ht_fh[r] = (hy - RO) * HX + hx + kXO;
      ht_g[r] = wrapi(y0 - 1 + hy, p.ny) * p.nx + wrapi(x0 - 1 + hx, p.nx);
    }
  }
  auto slotE = [&](int k) -> T* { return sE + (k % kRingE) * NEC * FE; };
  auto slotH = [&](int k) -> T* { return sHin + (k & (kRingH - 1)) * NHC * FH; };

  // asynchronous staging of the E_in frame of plane k (tile + 1 cell, periodic in x, y)
  auto issueE = [&](int k) {
    T* dst = slotE(k);
    const bool in = k < p.nz;
    const T* src = Ein + k * plane;
    if (p.vec16) {
#pragma unroll
      for (int r = 0; r < CE; ++r) {
        if (ce_s[r] < 0) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (!liveE(c)) continue;
          if (in) {
            cp_async16(dst + eo(c) + ce_s[r], src + c * ncell + ce_g[r]);
          } else {
#pragma unroll
            for (int v = 0; v < VE; ++v) dst[eo(c) + ce_s[r] + v] = T(0);
          }
        }
      }
    } else {
      for (int idx = tid; idx < FY * (TX + 2); idx += NTHR) {
        const int yy = idx / (TX + 2), hx = idx - yy * (TX + 2);
        if (TE && yy != 1) continue;
        const int g = wrapi(y0 - 1 + yy, p.ny) * p.nx + wrapi(x0 - 1 + hx, p.nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (!liveE(c)) continue;
          T* d = dst + eo(c) + (yy - RO) * FX + hx + kXO;
          if (in) cp_async_elem(d, src + c * ncell + g);
          else *d = T(0);
        }
      }
    }
  };
  // asynchronous staging of the H_in frame of plane k (tile + the -x / -y halo)
  auto issueH = [&](int k) {
    T* dst = slotH(k);
    const T* src = Hin + k * plane;
    if (p.vec16) {
#pragma unroll
      for (int r = 0; r < CH; ++r) {
        if (ch_s[r] < 0) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (liveH(c)) cp_async16(dst + ho(c) + ch_s[r], src + c * ncell + ch_g[r]);
      }
    } else {
      for (int idx = tid; idx < HY * (TX + 1); idx += NTHR) {
        const int yy = idx / (TX + 1), hx = idx - yy * (TX + 1);
        if (TE && yy != 1) continue;
        const int g = wrapi(y0 - 1 + yy, p.ny) * p.nx + wrapi(x0 - 1 + hx, p.nx);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (liveH(c)) cp_async_elem(dst + ho(c) + (yy - RO) * HX + hx + kXO, src + c * ncell + g);
      }
    }
  };

  // H^n at E-frame cell fe / H-frame cell fh / grid column gxy of plane k; e0/e1 = E frames of
  // planes k and k+1 (the E frame's origin is the H frame's, (x0-1, y0-1), one cell wider)
  auto computeH = [&](int fe, int fh, int gxy, int k, bool write_out, const T* e0, const T* e1,
                      const T* hin) {
    T hx_ = hin[ho(0) + fh], hy_ = TE ? T(0) : hin[ho(1) + fh], hz_ = hin[ho(2) + fh];
    if (p.doH) {
      HIn<T> e;
      e.ex0 = TE ? T(0) : e0[fe];
      e.ex_k1 = TE ? T(0) : e1[fe];
      e.ex_j1 = TE ? T(0) : e0[fe + FX];
      e.ey0 = e0[eo(1) + fe];
      e.ey_k1 = e1[eo(1) + fe];
      e.ey_i1 = e0[eo(1) + fe + 1];
      e.ez0 = TE ? T(0) : e0[eo(2) + fe];
      e.ez_j1 = TE ? T(0) : e0[eo(2) + fe + FX];
      e.ez_i1 = TE ? T(0) : e0[eo(2) + fe + 1];
      const int ip = psiH_plane(k, p.nz, p.npml);
      T psx = T(0), psy = T(0), b = T(1), c = T(0);
      const int pstride = (2 * p.npml + 1) * plane;
      const int pq = ip * plane + gxy;
      if (ip >= 0) {
        b = p.pmlH[2 * k];
        c = p.pmlH[2 * k + 1];
        psx = p.psiHin[pq];
        psy = TE ? T(0) : p.psiHin[pstride + pq];
      }
      h_update<T>(e, hx_, hy_, hz_, &psx, &psy, b, c, ip >= 0, S);
      if (write_out) {
        const int q = k * plane + gxy;
        p.Hout[q] = hx_;
        if (!TE) p.Hout[ncell + q] = hy_;
        p.Hout[2 * ncell + q] = hz_;
        if (ip >= 0) {
          p.psiHout[pq] = psx;
          if (!TE) p.psiHout[pstride + pq] = psy;
        }
      }
    }
    sH[ho(0) + fh] = hx_;
    if (!TE) sH[ho(1) + fh] = hy_;
    sH[ho(2) + fh] = hz_;
  };

  // ---- prologue: H^n of plane zb-1 at the own cell (for d/dz of the E update at zb) ----
  T hxm = T(0), hym = T(0);
  if (p.doE && zb > 0 && own) {
    const int q = (zb - 1) * plane + qxy;
    hxm = Hin[q];
    hym = TE ? T(0) : Hin[ncell + q];
    if (p.doH) {
      // zb-1 is never inside the CPML (chunk starts are planned that way)
      const int ip1 = (i + 1) % p.nx, jp1 = (j + 1) % p.ny;
      const int qj1 = (zb - 1) * plane + jp1 * p.nx + i;
      const int qi1 = (zb - 1) * plane + j * p.nx + ip1;
      HIn<T> e;
      e.ex0 = TE ? T(0) : Ein[q];
      e.ex_k1 = TE ? T(0) : Ein[q + plane];
      e.ex_j1 = TE ? T(0) : Ein[qj1];
      e.ey0 = Ein[ncell + q];
      e.ey_k1 = Ein[ncell + q + plane];
      e.ey_i1 = Ein[ncell + qi1];
      e.ez0 = TE ? T(0) : Ein[2 * ncell + q];
      e.ez_j1 = TE ? T(0) : Ein[2 * ncell + qj1];
      e.ez_i1 = TE ? T(0) : Ein[2 * ncell + qi1];
      T hz_dummy = T(0), psx = T(0), psy = T(0);
      h_update<T>(e, hxm, hym, hz_dummy, &psx, &psy, T(1), T(0), false, S);
    }
  }

  // per-thread energy accumulators (state precision; reduced in FP64 per block)
  T uE = T(0), uP = T(0), uB = T(0), uH = T(0);
  __syncthreads();   // coefficient and plane tables ready

  // prologue: E frames zb .. zb+kAheadE-1 and H frames zb .. zb+kAheadE-2, one commit group
  // per plane so that group g carries E(zb+1+g) and H(zb+g)
  issueE(zb);
  issueE(zb + 1);
  issueH(zb);
  cp_async_commit();
#pragma unroll
  for (int a = 1; a < kAheadE - 1; ++a) {
    if (zb + a < ze) {
      issueE(zb + 1 + a);
      issueH(zb + a);
    }
    cp_async_commit();
  }
  for (int k = zb; k < ze; ++k) {
    // ---------------- material state of plane k: loads issued before the stencil ----------
    const int info = sInfo[k - zb];
    const int mi = (info & kPlaneMat) - 1;
    const bool in_box = (info & kPlaneEbox) != 0;
    const bool mat_here = p.doE && own && mi >= 0 && p.mat[mi].kind != kVacuum;
    T rPa[3], rPb[3], rD[3];
    T rY[3][NBP > 0 ? NBP : 1], rV[3][NBP > 0 ? NBP : 1];
    T rS = T(0);   // sigma(r) of the cell when the simulation has a per-cell map
    int r = 0, rl = 0, mstride = 0, yb0 = 0;
    const int nmc = (int)p.nmatcell;
    if (p.doE && own && mi >= 0) {
      const MatK<T>& M = p.mat[mi];
      rl = (k - M.zlo) * plane + qxy;
      r = (int)M.base + rl;
      mstride = (int)M.ncell;
      yb0 = (int)M.ybase + rl;
      if (p.sig) rS = p.sig[r];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (!liveE(c)) {
          rPa[c] = rPb[c] = rD[c] = T(0);
          continue;
        }
        rPa[c] = p.Pa[c * nmc + r];
        rPb[c] = p.Pb[c * nmc + r];
        if (!INC) rD[c] = p.D[c * nmc + r];
      }
      if (NBP > 0 && M.kind == kLorentzBath) {
        const YT* ya = reinterpret_cast<const YT*>(p.Ya) + yb0;
        const YT* yb = reinterpret_cast<const YT*>(p.Yb) + yb0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (!liveE(c)) continue;
#pragma unroll
          for (int jj = 0; jj < (NBP > 0 ? NBP : 1); ++jj) {
            if (jj < M.nb) {
              YS::load2(ya + (c * M.nb + jj) * mstride, yb + (c * M.nb + jj) * mstride, rY[c][jj], rV[c][jj]);
            }
          }
        }
      }
    }
    // ---------------- prefetch the frames kAheadE-1 planes ahead ----------------
    if (k + kAheadE - 1 < ze) {
      issueE(k + kAheadE);
      issueH(k + kAheadE - 1);
    }
    cp_async_commit();
    // groups g0..g(t+3) are committed (t = k - zb; group g carries E(zb+1+g), H(zb+g));
    // leaving the three newest in flight guarantees g(t): E(k+1) and H(k) have landed
    cp_async_wait<kAheadE - 1>();
    __syncthreads();
    // ---------------- H^n of plane k (own cells + -x/-y halo) ----------------
    {
      const T* e0 = slotE(k);
      const T* e1 = slotE(k + 1);
      const T* hin = slotH(k);
      // own cell (threads past the grid edge compute wrapped values that are never stored)
      computeH(own_fe, own_fh, qxy, k, own, e0, e1, hin);
      // halo: row y0-1 (TX cells) and column x0-1 (TY cells), recomputed, never stored
#pragma unroll
      for (int t = 0; t < NHT; ++t)
        if (ht_fe[t] >= 0) computeH(ht_fe[t], ht_fh[t], ht_g[t], k, false, e0, e1, hin);
    }
    __syncthreads();

    // H-side monitor and energy partials
    if (p.doH) {
      if (info & kPlaneMonH)
      for (int m = 0; m < p.nmon; ++m) {
        const int zm = p.mon_z[m];
        if (k == zm - 1 || k == zm) {
          const int off = (k == zm) ? 1 : 0;
          T vx = own ? sH[own_fh] : T(0);
          T vy = own && !TE ? sH[ho(1) + own_fh] : T(0);
          if constexpr (WS > 1) {
            double* rows = p.mon_partial_H;
            warp_sum_to((double)vx, wslot(rows ? rows + (int64_t)(4 * m + off) * nbxy : nullptr));
            warp_sum_to((double)vy, wslot(rows ? rows + (int64_t)(4 * m + 2 + off) * nbxy : nullptr));
          } else {
            double sx = block_sum((double)vx, sred);
            double sy = block_sum((double)vy, sred);
            if (tid == 0 && p.mon_partial_H) {
              put_slot(p.mon_partial_H + (int64_t)(4 * m + off) * nbxy, sx);
              put_slot(p.mon_partial_H + (int64_t)(4 * m + 2 + off) * nbxy, sy);
            }
          }
        }
      }
      if (p.eH_on && own && in_box) {
        T a = sH[ho(0) + own_fh], b = TE ? T(0) : sH[ho(1) + own_fh], c = sH[ho(2) + own_fh];
        uH += a * a + b * b + c * c;
      }
    }

    // ---------------- D/E, P, Y of plane k (own cells) ----------------
    if (p.doE) {
      T Ev[3] = {T(0), T(0), T(0)};
      if (own) {
        const int q = k * plane + qxy;
        const T* e0 = slotE(k);
        const int fh = own_fh;
        const T Hx = sH[ho(0) + fh], Hy = TE ? T(0) : sH[ho(1) + fh], Hz = sH[ho(2) + fh];
        // differences of H^n for dt curl H^n = S [...] (Eq. FDTD-1D form)
        // (TE: ny = 1, the row above is this row and the y-differences vanish)
        const T dyHz = Hz - (TE ? Hz : sH[ho(2) + fh - HX]);
        const T dzHy = Hy - hym;
        const T dzHx = Hx - hxm;
        const T dxHz = Hz - sH[ho(2) + fh - 1];
        const T dxHy = Hy - (TE ? T(0) : sH[ho(1) + fh - 1]);
        const T dyHx = Hx - (TE ? Hx : sH[ho(0) + fh - HX]);
        T curl[3];
        const int ip = psiE_plane(k, p.nz, p.npml);
        if (ip >= 0) {
          const T b = p.pmlE[2 * k], c = p.pmlE[2 * k + 1];
          const int pq = ip * plane + qxy;
          const int pstride = 2 * p.npml * plane;
          T px = TE ? T(0) : b * p.psiE[pq] + c * dzHy;
          T py = b * p.psiE[pstride + pq] + c * dzHx;
          if (!TE) p.psiE[pq] = px;
          p.psiE[pstride + pq] = py;
          curl[0] = dyHz - (dzHy + px);
          curl[1] = (dzHx + py) - dxHz;
        } else {
          curl[0] = dyHz - dzHy;
          curl[1] = dzHx - dxHz;
        }
        curl[2] = dxHy - dyHx;
        // soft source current on this plane (per component, kept in scalars)
        T J0 = T(0), J1 = T(0), J2 = T(0);
        bool h0 = false, h1 = false, h2 = false;
        if (info & kPlaneSrc)
        for (int s = 0; s < p.nsrc; ++s) {
          if (p.src_z[s] == k) {
            T v = p.src_a[s];
            if (p.src_cos[s]) v = p.src_a[s] * p.src_cos[s][qxy] + p.src_b[s] * p.src_sin[s][qxy];
            const int sc = p.src_comp[s];
            if (sc == 0) { J0 += v; h0 = true; }
            else if (sc == 1) { J1 += v; h1 = true; }
            else { J2 += v; h2 = true; }
          }
        }
        const T J[3] = {J0, J1, J2};
        const bool hasJ[3] = {h0, h1, h2};
        if (mi < 0) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if (!liveE(c)) continue;   // Ev[c] stays 0
            T e = e0[eo(c) + own_fe] + S * curl[c];
            if (hasJ[c]) e = e + dt * J[c];
            Ev[c] = e;
            p.Eout[c * ncell + q] = e;
          }
        } else {
          const MatK<T>& M = p.mat[mi];
          const bool bath = (M.kind == kLorentzBath) && (NBMAX > 0);
          const T* cfm = sCoef + M.coef_off * kCoefStride;
          // the drive coefficient eps0 w0^2 dt^2 sigma(r) and the energy weight rho(r)/dt^2 of
          // this cell (Eq. EOM_Lorentz's sigma(r); rho = 1/(sigma w0^2))
          const T cEr = p.sig ? M.dcE * rS : M.cE;
          const T rhor = p.sig ? (rS > T(0) ? M.rho_s / rS : T(0)) : M.rho_idt2;
          YT* const ya = reinterpret_cast<YT*>(p.Ya) + yb0;
          YT* const yb = reinterpret_cast<YT*>(p.Yb) + yb0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if (!liveE(c)) continue;   // Ev[c] stays 0
            T E;
            const T Pa = rPa[c];
            const T Pb = rPb[c];
            if (!INC) {
              // D^{n+1/2} = D^{n-1/2} + S [curl differences] (+ dt J);  E = (1/eps_inf)(D - P^{n+1/2})
              T D = rD[c] + S * curl[c];
              if (hasJ[c]) D = D + dt * J[c];
              p.D[c * nmc + r] = D;
              E = M.inv_eps * (D - Pa);
            } else {
              // D-free: E += (dt curl H + dt J - (P^{n+1/2} - P^{n-1/2})) / eps_inf
              T inc = S * curl[c];
              if (hasJ[c]) inc = inc + dt * J[c];
              E = e0[eo(c) + own_fe] + (inc - (Pa - Pb)) * M.inv_eps;
            }
            Ev[c] = E;
            p.Eout[c * ncell + q] = E;
            // bath modes already in registers: all three components together below
            if (!mat_here || (NBP > 0 && bath)) continue;
            // ---- polarization (and bath) update, one component at a time ----
            // Up to 32 modes the component's modes are held in registers between the bath sum and
            // the mode update; above (kStream) they are streamed twice from memory, the second
            // pass re-reading what the first read (about 200 words per cell, an L2 hit).
            T Yl[kStream ? 1 : NBA], Vl[kStream ? 1 : NBA];
            const int nb = bath ? M.nb : 0;
            const int yc = c * M.nb * mstride;
            T bsum = T(0);
            if constexpr (kStream) {
              // batches of kStreamBatch modes: all their loads issued before any is used
              for (int j0 = 0; j0 < nb; j0 += kStreamBatch) {
                T ys[kStreamBatch], vs[kStreamBatch];
#pragma unroll
                for (int u = 0; u < kStreamBatch; ++u) {
                  if (j0 + u < nb) {
                    YS::load2(ya + yc + (j0 + u) * mstride, yb + yc + (j0 + u) * mstride, ys[u], vs[u]);
                  }
                }
#pragma unroll
                for (int u = 0; u < kStreamBatch; ++u) {
                  if (j0 + u < nb) {
                    T cf[6];
                    load_coef6(cfm + (j0 + u) * kCoefStride, cf);
                    if (!INC) {
                      bsum = bath_sum_lit(bsum, cf[0], cf[1], cf[2], ys[u], vs[u]);
                    } else {
                      const T v = YB ? vs[u] : ys[u] - vs[u];
                      bsum = bsum + (cf[0] * ys[u] + cf[1] * v);
                    }
                  }
                }
              }
            }
#pragma unroll
            for (int jj = 0; jj < (kStream ? 0 : NBA); ++jj) {
              if (jj < nb) {
                if (NBP > 0) {
                  Yl[jj] = rY[c][jj < NBP ? jj : 0];
                  Vl[jj] = rV[c][jj < NBP ? jj : 0];
                } else {
                  YS::load2(ya + yc + jj * mstride, yb + yc + jj * mstride, Yl[jj], Vl[jj]);
                }
                T cf[6];
                load_coef6(cfm + jj * kCoefStride, cf);
                if (!INC) {
                  bsum = bath_sum_lit(bsum, cf[0], cf[1], cf[2], Yl[jj], Vl[jj]);   // k_j (a_j Y^n + b_j Y^{n-1})
                } else {
                  if (!YB) Vl[jj] = Yl[jj] - Vl[jj];                         // V_j = Y^n - Y^{n-1}
                  bsum = bsum + (cf[0] * Yl[jj] + cf[1] * Vl[jj]);           // k_j ((a_j+b_j) Y - b_j V)
                }
              }
            }
            T Pn, Vn, V0;
            if (!INC) {
              // Eq. Pz_update-LB (Eq. Pz_1D_Lorentz when there is no bath):
              // P^{n+1} = (1/A) [cE E - (w0^2 dt^2 - 2) P^n - c2 P^{n-1} - dt/2 sum_j k_j(a_j Y^n + b_j Y^{n-1})]
              T num = cEr * E - M.c1m * Pa - M.c2 * Pb;
              if (bath) num = num - T(0.5) * dt * bsum;
              Pn = M.inv_A * num;
              p.Pb[c * nmc + r] = Pn;   // overwrites P^{n-1}
              Vn = Pn - Pa;
              V0 = Pa - Pb;
            } else {
              // increment form: V^{n+1} = [cE E - w0^2 dt^2 P^n + c2 V^n - dt/2 sum(...)] / A
              V0 = Pa - Pb;
              T num = cEr * E - M.W * Pa + M.c2 * V0;
              if (bath) num = num - T(0.5) * dt * bsum;
              Vn = num * M.inv_A;
              Pn = Pa + Vn;
              p.Pb[c * nmc + r] = Pn;   // overwrites P^{n-1}
            }
            T ub = T(0);
            const T dP = Vn + V0;   // P^{n+1} - P^{n-1}
            if constexpr (kStream) {
              for (int j0 = 0; j0 < nb; j0 += kStreamBatch) {
                T ys[kStreamBatch], vs[kStreamBatch];
#pragma unroll
                for (int u = 0; u < kStreamBatch; ++u) {
                  if (j0 + u < nb) {
                    YS::load2(ya + yc + (j0 + u) * mstride, yb + yc + (j0 + u) * mstride, ys[u], vs[u]);
                  }
                }
#pragma unroll
                for (int u = 0; u < kStreamBatch; ++u) {
                  const int jj = j0 + u;
                  if (jj >= nb) break;
                  const T y = ys[u];
                  T v = vs[u];
                  if (INC && !YB) v = y - v;
                  T cf[6];
                  load_coef6(cfm + jj * kCoefStride, cf);
                  T Ynew, Vy;
                  if (!INC) {
                    Ynew = bath_new_lit(cf[1], cf[3], cf[4], y, v, Pn - Pb);
                    Vy = Ynew - y;
                  } else {
                    Vy = cf[2] * y + cf[3] * v + cf[4] * dP;
                    Ynew = y + Vy;
                  }
                  if (YB) {
                    YS::put_pair(ya + yc + jj * mstride, Ynew, Vy);
                  } else {
                    YS::put(yb + yc + jj * mstride, Ynew);
                  }
                  if (p.eE_on) ub = INC ? ub + (Vy * Vy + cf[5] * Ynew * Ynew) : bath_energy_lit(ub, Vy, cf[5], Ynew);
                }
              }
            }
#pragma unroll
            for (int jj = 0; jj < (kStream ? 0 : NBA); ++jj) {
              if (jj < nb) {
                T cf[6];
                load_coef6(cfm + jj * kCoefStride, cf);
                T Ynew, Vy;
                if (!INC) {
                  // Eq. Yzj_finite_difference: Y^{n+1} = a Y^n + (b+1) Y^{n-1} + c (P^{n+1} - P^{n-1})
                  Ynew = bath_new_lit(cf[1], cf[3], cf[4], Yl[jj], Vl[jj], Pn - Pb);
                  Vy = Ynew - Yl[jj];
                } else {
                  // V_Y^{n+1} = (a+b) Y^n - (b+1) V_Y^n + c (V_P^{n+1} + V_P^n);  Y^{n+1} = Y^n + V_Y^{n+1}
                  Vy = cf[2] * Yl[jj] + cf[3] * Vl[jj] + cf[4] * dP;
                  Ynew = Yl[jj] + Vy;
                }
                if (YB) {
                  YS::put_pair(ya + yc + jj * mstride, Ynew, Vy);   // in place: Y^{n+1} and V^{n+1}
                } else {
                  YS::put(yb + yc + jj * mstride, Ynew);   // overwrites Y^{n-1}
                }
                if (p.eE_on) ub = INC ? ub + (Vy * Vy + cf[5] * Ynew * Ynew) : bath_energy_lit(ub, Vy, cf[5], Ynew);   // (w_j dt)^2 Y^2
              }
            }
            if (p.eE_on && in_box) {
              // rho/dt^2 (V^2 + (w0 dt)^2 P^2) = rho (V/dt)^2 + rho w0^2 P^2, likewise per mode
              uP += rhor * (Vn * Vn + M.w0r2dt2 * Pn * Pn);
              uB += rhor * ub;
            }
          }
          if (NBP > 0 && bath && mat_here) {
            // ---- polarization and bath update of the three components together, modes outer:
            // each mode's coefficient row is read once for the three components; per component
            // the arithmetic and its order are those of the loop above (sums over ascending j) ----
            const int nb = M.nb;
            T bsum[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int jj = 0; jj < (NBP > 0 ? NBP : 1); ++jj) {
              if (jj < nb) {
                T cf[6];
                load_coef6(cfm + jj * kCoefStride, cf);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  if (!liveE(c)) continue;
                  const T y = rY[c][jj];
                  if (!INC) {
                    bsum[c] = bath_sum_lit(bsum[c], cf[0], cf[1], cf[2], y, rV[c][jj]);
                  } else {
                    if (!YB) rV[c][jj] = y - rV[c][jj];   // V_j = Y^n - Y^{n-1}
                    bsum[c] = bsum[c] + (cf[0] * y + cf[1] * rV[c][jj]);
                  }
                }
              }
            }
            T Pn[3], Vn[3], dP[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              if (!liveE(c)) continue;
              const T Pa = rPa[c], Pb = rPb[c];
              T V0;
              if (!INC) {
                T num = cEr * Ev[c] - M.c1m * Pa - M.c2 * Pb;
                num = num - T(0.5) * dt * bsum[c];
                Pn[c] = M.inv_A * num;
                Vn[c] = Pn[c] - Pa;
                V0 = Pa - Pb;
              } else {
                V0 = Pa - Pb;
                T num = cEr * Ev[c] - M.W * Pa + M.c2 * V0;
                num = num - T(0.5) * dt * bsum[c];
                Vn[c] = num * M.inv_A;
                Pn[c] = Pa + Vn[c];
              }
              p.Pb[c * nmc + r] = Pn[c];   // overwrites P^{n-1}
              dP[c] = Vn[c] + V0;          // P^{n+1} - P^{n-1}
            }
            T ub[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int jj = 0; jj < (NBP > 0 ? NBP : 1); ++jj) {
              if (jj < nb) {
                T cf[6];
                load_coef6(cfm + jj * kCoefStride, cf);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  if (!liveE(c)) continue;
                  const int yo = c * nb * mstride + jj * mstride;
                  const T y = rY[c][jj], v = rV[c][jj];
                  T Ynew, Vy;
                  if (!INC) {
                    Ynew = bath_new_lit(cf[1], cf[3], cf[4], y, v, Pn[c] - rPb[c]);
                    Vy = Ynew - y;
                  } else {
                    Vy = cf[2] * y + cf[3] * v + cf[4] * dP[c];
                    Ynew = y + Vy;
                  }
                  if (YB) {
                    YS::put_pair(ya + yo, Ynew, Vy);
                  } else {
                    YS::put(yb + yo, Ynew);
                  }
                  if (p.eE_on) ub[c] = INC ? ub[c] + (Vy * Vy + cf[5] * Ynew * Ynew) : bath_energy_lit(ub[c], Vy, cf[5], Ynew);
                }
              }
            }
            if (p.eE_on && in_box) {
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                if (!liveE(c)) continue;
                uP += rhor * (Vn[c] * Vn[c] + M.w0r2dt2 * Pn[c] * Pn[c]);
                uB += rhor * ub[c];
              }
            }
          }
        }
        if (p.eE_on && in_box) {
          T eps = T(1);
          if (mi >= 0) eps = p.mat[mi].eps;
          uE += eps * (Ev[0] * Ev[0] + Ev[1] * Ev[1] + Ev[2] * Ev[2]);
        }
      }
      // E-side monitor partials
      if (info & kPlaneMonE)
      for (int m = 0; m < p.nmon; ++m) {
        if (k == p.mon_z[m]) {
          if constexpr (WS > 1) {
            double* rows = p.mon_partial_E;
            warp_sum_to(own ? (double)Ev[0] : 0.0, wslot(rows ? rows + (int64_t)(2 * m) * nbxy : nullptr));
            warp_sum_to(own ? (double)Ev[1] : 0.0, wslot(rows ? rows + (int64_t)(2 * m + 1) * nbxy : nullptr));
          } else {
            double sx = block_sum(own ? (double)Ev[0] : 0.0, sred);
            double sy = block_sum(own ? (double)Ev[1] : 0.0, sred);
            if (tid == 0 && p.mon_partial_E) {
              put_slot(p.mon_partial_E + (int64_t)(2 * m) * nbxy, sx);
              put_slot(p.mon_partial_E + (int64_t)(2 * m + 1) * nbxy, sy);
            }
          }
        }
      }
      hxm = sH[ho(0) + own_fh];
      hym = TE ? T(0) : sH[ho(1) + own_fh];
    }
  }
  // energy partials of this block (every block writes, zero when outside the box)
  if (p.eE_on) {
    if constexpr (WS > 1) {
      warp_sum_to(uE, wslot(p.en_partial_E + (int64_t)chunk * nbxy));
      warp_sum_to(uP, wslot(p.en_partial_E + ((int64_t)nbxy * p.nchunks_total + chunk * nbxy)));
      warp_sum_to(uB, wslot(p.en_partial_E + ((int64_t)2 * nbxy * p.nchunks_total + chunk * nbxy)));
    } else {
      double a = block_sum(uE, sred);
      double b = block_sum(uP, sred);
      double c = block_sum(uB, sred);
      if (tid == 0) {
        put_slot(p.en_partial_E + (int64_t)chunk * nbxy, a);
        put_slot(p.en_partial_E + ((int64_t)nbxy * p.nchunks_total + chunk * nbxy), b);
        put_slot(p.en_partial_E + ((int64_t)2 * nbxy * p.nchunks_total + chunk * nbxy), c);
      }
    }
  }
  if (p.eH_on) {
    if constexpr (WS > 1) {
      warp_sum_to(uH, wslot(p.en_partial_H + (int64_t)chunk * nbxy));
    } else {
      double a = block_sum(uH, sred);
      if (tid == 0) put_slot(p.en_partial_H + (int64_t)chunk * nbxy, a);
    }
  }
}

inline size_t step3d_smem_bytes(int ty, int nmodes, size_t elem, int tx = kTX, bool te = false) {
  // the TE form stores one row of E_y and of H_x, H_z per frame
  const size_t fe = (size_t)(te ? 1 : ty + 2) * (tx + 8), fh = (size_t)(te ? 1 : ty + 1) * (tx + 4);
  const size_t n = (size_t)kRingE * (te ? 1 : 3) * fe + (size_t)(kRingH + 1) * (te ? 2 : 3) * fh +
                   (size_t)kCoefStride * nmodes;
  return n * elem + kMaxChunk * sizeof(int) + 16 + 8 * sizeof(double);   // block-sum scratch: a double per warp (<= 8)
}

}  // namespace fdtdbath
