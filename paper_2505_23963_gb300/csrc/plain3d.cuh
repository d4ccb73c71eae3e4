// plain3d.cuh -- the fused step of the z-planes without bath modes (vacuum, CPML, Lorentz and
// Drude layers), general 3D form on grids tiled exactly by its tiles; and its Lorentz-Bath form
// for the layers with at most 8 bath modes (FP32).
//
// It computes what step3d_kernel<T, INC, 0, 8> computes for such planes -- the H half-step of
// the previous step (H^n from E^{n-1/2}, Eq. 1b, with the CPML memories of the z-derivative
// terms), this step's D/E half-step (Eq. 1a, D = E + P, soft plane sources) and the Lorentz /
// Drude polarization update (Eq. Pz_1D_Lorentz, one P per component) -- with the same
// expressions in the same order, so that FP64 runs (compiled without FMA contraction) agree with
// it to rounding of the partial sums.  It exists because the general kernel, one cell per thread
// with ~1000 per-thread 16-byte copies and two barriers per plane, spends ~130 integer
// instructions per cell and plane and runs these planes at half of the memory bandwidth.  Here:
//
//   * a CTA owns a TX x 8 column tile (TX = 32 VX) and marches along a z-chunk; compute warp w owns
//     row y0 + w, lane l the VX = 16 / sizeof(T) adjacent cells x0 + VX l ..., so every
//     shared-memory and global access of a thread is one 16-byte vector and the per-plane
//     bookkeeping is paid once per VX cells; plain vacuum planes run a code path without the
//     CPML, layer, source and monitor branches;
//   * one more warp (the helper) stages the planes ahead with the tensor-copy engine
//     (cp.async.bulk.tensor, 5-D maps of the E / H double buffers): per stage ten boxes -- the
//     tile's rows, the rows y0-1 and y0+8 and the 4-cell side columns of E_in(k+1), the tile's rows,
//     row y0-1 and left column of H_in(k) -- each into a box-dense part of the frame, so that the
//     periodic neighbours are plain boxes at wrapped coordinates; stages complete on one mbarrier
//     each (waits bounded in time).  Many small row copies instead (one per frame row) saturated
//     the copy engine at about half of the bandwidth.  The helper also recomputes H^n on the halo
//     row y0-1, so the eight compute warps carry equal work;
//   * the halo cell x0-1 of each row is recomputed by lane 0 of the row's warp; x-neighbours of H^n
//     pass between lanes by shuffles, y-neighbours (H_x, H_z only) through shared memory;
//   * one CTA barrier per plane: H^n of plane k goes to one of two shared buffers, so the E update
//     of plane k and the H update of plane k+1 never touch the same buffer.
//
// Shared-memory ring: E frames in A+1 slots, H_in frames in A slots, H^n (x and z) in two
// buffers.  Stage g of a chunk (plane k = zb + g) brings E_in(k+1) and H_in(k), stage 0 also
// E_in(zb); it is issued after the barrier of plane k-A, when the slots it overwrites
// (E_in(k-A), H_in(k-A)) have been read for the last time.
//
// The Lorentz-Bath form (NB > 0: FP32 increment form, one cell per thread, 32 x 8 tiles) runs the
// z-chunks of the Lorentz-Bath layers with at most NB modes per material, with what
// step3d_kernel<float, true, NB, 8> computes there: the polarization update of Eq.
// Pz_update-LB and the bath-mode update of Eq. Yzj_finite_difference, three components together
// with the modes outer, sums over ascending j.  Per cell and step it reads and writes P (two
// levels) and 2 x 3 NB bath-mode words, far more than the fields, so:
//   * the CTA has the eight compute warps only (no helper: a ninth warp caps the registers at 96
//     for two CTAs per SM, and the 54 state words of a cell then spill); warp 0 also recomputes the
//     halo row y0-1 and lane 0 of warp 0 issues the copies;
//   * the state of plane k of the tile -- P^{n+1/2}, Y^n, P^{n-1/2}, Y^{n-1} -- arrives in a
//     shared buffer by four 4-D tensor copies (one box each, from maps of the two state slots),
//     issued after the barrier of plane k-1, read into registers before the barrier of plane k, so
//     a whole plane of work covers each copy's latency.  Loading it from global memory straight
//     into registers at the start of the plane instead left the loads' latency exposed (long
//     scoreboard stalls 2.6 per issue) and ran the layer at 0.55 of the bandwidth.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "internal.h"

namespace fdtdbath {

namespace plain {

constexpr int TY = 8;                          // rows of a tile = compute warps (one more: the helper)
constexpr int kMaxPlanes = 64;                 // planes per z-chunk of this kernel
constexpr uint64_t kWaitLimitNs = 1000000000;  // a stage not complete after 1 s is an error
// per-plane table bits (material index + 1 in the low four bits)
enum : int {
  kBox = 0x10, kMonE = 0x20, kMonH = 0x40, kSrc = 0x80, kPmlE = 0x100, kPmlH = 0x200, kTop = 0x400,
  kBath = 0x800   // a Lorentz-Bath plane with bath modes
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ unsigned mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for the phase of the given parity to complete; false after kWaitLimitNs without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int r = 0; r < 32; ++r)
      if (mbar_try_wait(b, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}
// Tensor copy global -> this CTA's shared memory (shared-space address sdst, 128-byte aligned) of
// the box of tensor map tmap at coordinates (x, y, z, c, b), completing its bytes on mbarrier bar.
__device__ __forceinline__ void tma_load5(unsigned sdst, const void* tmap, int x, int y, int z, int c, int b,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(sdst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(b), "r"(smem_u32(bar))
      : "memory");
}

// Tensor copy of a 4-D box (coordinates x, y, z, m), as tma_load5.
__device__ __forceinline__ void tma_load4(unsigned sdst, const void* tmap, int x, int y, int z, int m, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(sdst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(m), "r"(smem_u32(bar))
      : "memory");
}

// VX-cell vectors (8 or 16 bytes, naturally aligned)
template <typename T, int VX>
struct Vec;
template <>
struct Vec<float, 4> {
  static __device__ __forceinline__ void ld(const void* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
  static __device__ __forceinline__ void st(void* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec<float, 2> {
  static __device__ __forceinline__ void ld(const void* p, float* o) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x;
    o[1] = v.y;
  }
  static __device__ __forceinline__ void st(void* p, const float* v) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};
template <typename T>
struct Vec<T, 1> {
  static __device__ __forceinline__ void ld(const void* p, T* o) { o[0] = *reinterpret_cast<const T*>(p); }
  static __device__ __forceinline__ void st(void* p, const T* v) { *reinterpret_cast<T*>(p) = v[0]; }
};
template <>
struct Vec<double, 2> {
  static __device__ __forceinline__ void ld(const void* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x;
    o[1] = v.y;
  }
  static __device__ __forceinline__ void st(void* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// H update (Eq. 1b, mu0 = 1) of one cell from the six E differences, in the form of the general
// kernel's h_update: psi <- b psi + c dE|z inside the CPML.
template <typename T>
__device__ __forceinline__ void h_cell(T& hx, T& hy, T& hz, T& psx, T& psy, T dyEz, T dzEy, T dzEx, T dxEz,
                                       T dxEy, T dyEx, bool pml, T b, T c, T S) {
  if (pml) {
    psx = b * psx + c * dzEy;
    psy = b * psy + c * dzEx;
    hx = hx - S * (dyEz - (dzEy + psx));
    hy = hy - S * ((dzEx + psy) - dxEz);
  } else {
    hx = hx - S * (dyEz - dzEy);
    hy = hy - S * (dzEx - dxEz);
  }
  hz = hz - S * (dxEy - dyEx);
}

}  // namespace plain

// Per 32 x 8 partial-sum slot (a tile's rows are its slot's rows): each slot column h (VX per
// block) collects 32/VX lanes per row.  block_slot_sums: the sum of v[q] over each slot's
// lanes (shuffles in V's precision) lands in red[q][row][h] (FP64), written by the compute warps;
// a barrier follows, so slot_total reads it.  Fixed order throughout.
template <int TY, int VX, int NQ, typename V>
__device__ __forceinline__ void block_slot_sums(V (&v)[NQ], double* red, int w, int lane) {
  constexpr int LPS = 32 / VX;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o, LPS);
  if (w < TY && (lane % LPS) == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[(q * TY + w) * VX + lane / LPS] = (double)v[q];
  __syncthreads();
}
// the slot's total over the TY rows (0.0 + the sum in row order)
template <int TY, int VX>
__device__ __forceinline__ double slot_total(const double* red, int q, int h) {
  double s = 0.0;
  for (int ww = 0; ww < TY; ++ww) s += red[(q * TY + ww) * VX + h];
  return s;
}

template <typename T, int VX_, int A, int NB = 0>
struct Plain3DLayout {
  static constexpr int VX = VX_, TY = plain::TY, TX = 32 * VX;
  static constexpr int NE = A + 1, NH = A;   // E and H_in frame slots
  // the helper warp (NB = 0); the bath form in registers runs without it, its warps sized for 128
  // registers.
  // Above 8 modes (NB = 16) two threads share a cell, each with half of its modes (SPLIT warps
  // per tile row: the first computes the fields, both the bath)
  // Above 16 (NB = 128, STREAM) the modes are streamed: batches of MB modes of one component (both
  // levels) pass through an R-slot shared-memory ring filled by tensor copies, twice per component
  // (bath sum, then the mode update); the helper warp returns to issue them (the state held in
  // registers is small again)
  static constexpr bool STREAM = NB > 16;
  static constexpr bool HELPER = NB == 0 || STREAM;
  static constexpr int SPLIT = NB > 8 && !STREAM ? 2 : 1, NBH = NB > 0 && !STREAM ? NB / SPLIT : 1;
  static constexpr int MB = kStreamBatchModes, R = 4;
  static constexpr int NMBAR = A + 1 + (STREAM ? 2 * R : 0);   // frame stages, bath state, ring
  static constexpr int threads = 32 * (TY * SPLIT + (HELPER ? 1 : 0));
  static constexpr unsigned SZ = sizeof(T);
  static constexpr unsigned r128(unsigned b) { return (b + 127u) & ~127u; }
  // An E frame slot (each part one box, box-dense, 128-byte aligned): main [3][TY][TX] rows
  // y0..y0+TY-1; top [3][TX] row y0-1; bot [3][TX] row y0+TY; pl8 [3][TY][4] columns x0-4..x0-1 of
  // rows y0..; plb [3][4] the same columns of row y0+TY; prt [3][4] columns x0+TX..x0+TX+3 of row
  // y0-1; pr8 [3][TY][4] those columns of rows y0...
  static constexpr unsigned E_MAIN = 0, E_TOP = r128(3u * TY * TX * SZ), E_BOT = E_TOP + r128(3u * TX * SZ);
  static constexpr unsigned E_PL8 = E_BOT + r128(3u * TX * SZ), E_PLB = E_PL8 + r128(3u * TY * 4 * SZ);
  static constexpr unsigned E_PRT = E_PLB + r128(12u * SZ), E_PR8 = E_PRT + r128(12u * SZ);
  static constexpr unsigned ES = E_PR8 + r128(3u * TY * 4 * SZ);
  // an H_in frame slot: main [3][TY][TX], top [3][TX] (row y0-1), pl8 [3][TY][4] (columns x0-4..x0-1)
  static constexpr unsigned H_MAIN = 0, H_TOP = r128(3u * TY * TX * SZ), H_PL8 = H_TOP + r128(3u * TX * SZ);
  static constexpr unsigned HS = H_PL8 + r128(3u * TY * 4 * SZ);
  // bytes of the boxes of one E frame and of one H_in frame
  static constexpr unsigned E_BYTES = (3u * TY * TX + 2 * 3u * TX + 2 * 3u * TY * 4 + 2 * 12u) * SZ;
  static constexpr unsigned H_BYTES = (3u * TY * TX + 3u * TX + 3u * TY * 4) * SZ;
  // H^n buffers [2][Hx, Hz][TY + 1][TX] (row 0: y0-1), then mbarriers [A], plane table [kMaxPlanes]
  static constexpr unsigned XS = 2u * (TY + 1) * TX * SZ;
  static constexpr unsigned OFF_E = 0, OFF_HIN = NE * ES, OFF_SH = OFF_HIN + NH * HS, OFF_MBAR = OFF_SH + 2 * XS;
  // mbarriers: one per frame stage, one for the bath state
  static constexpr unsigned OFF_INFO = OFF_MBAR + ((8 * NMBAR + 15) / 16) * 16;
  // bath-mode coefficient rows of every material ([modes][kCoefStride], at most kMaxMat NB rows)
  static constexpr unsigned OFF_COEF = OFF_INFO + plain::kMaxPlanes * 4;
  // (streamed: at most kStreamCoefRows rows in all, the host checks)
  static constexpr unsigned COEF_BYTES =
      NB > 0 ? (unsigned)(STREAM ? kStreamCoefRows : kMaxMat * NB) * kCoefStride * SZ : 0u;
  // bath state of one plane tile (bath form): per level (P^{n+1/2}, Y^n, then P^{n-1/2}, Y^{n-1})
  // the modes [3 nb][TY][TX] (box order), then P [3][TY][TX]
  static constexpr unsigned BT = TY * TX * SZ;   // one component / mode of the tile
  static constexpr unsigned B_P = 3u * (NB > 0 && !STREAM ? NB : 0) * BT, B_LVL = B_P + 3u * BT;
  static constexpr unsigned OFF_BATH = r128(OFF_COEF + COEF_BYTES);
  static constexpr unsigned BATH_BYTES = NB > 0 ? 2u * B_LVL : 0u;
  // the two halves' exchange (SPLIT = 2): E^{n+1/2} and the bath sums of each half, [9][TY][TX]
  static constexpr unsigned OFF_XCH = r128(OFF_BATH + BATH_BYTES);
  static constexpr unsigned XCH_BYTES = SPLIT > 1 ? 9u * BT : 0u;
  // the streamed modes' ring: R slots of [level a: MB][TY][TX], [level b: MB][TY][TX]
  static constexpr unsigned RING_SLOT = STREAM ? 2u * MB * BT : 0u;
  static constexpr unsigned OFF_RING = r128(OFF_XCH + XCH_BYTES);
  static constexpr unsigned bytes = OFF_RING + R * RING_SLOT + 128;   // + alignment slack
  // CTAs per SM that the shared memory admits (228 KB per SM, 1 KB reserved per CTA, static 128 B)
  static constexpr int per_sm = 233472 / (bytes + 1024 + 128) > 8 ? 8 : 233472 / (bytes + 1024 + 128);
  // CTAs per SM the registers are sized for: as the shared memory admits, or two with bath modes
  // (a cell's whole bath state is held in registers)
  static constexpr int min_blocks = NB > 0 ? (SPLIT > 1 ? 1 : 2) : per_sm;
  static_assert(NB == 0 || NB == 4 || NB == 8 || NB == 16 || NB == 128, "bath form: 4, 8, 16 or 128 modes");
  static_assert(ES % 128 == 0 && HS % 128 == 0 && XS % 128 == 0, "128-byte aligned frames");
  // the slot sums of the monitors / energy use the H^n buffer not in use (4 x TY x VX doubles)
  static_assert(4 * TY * VX * 8 <= XS, "reduction scratch fits an H buffer");
};

// NB = 0: the plain-plane kernel; NB > 0 (one cell per thread, FP32 increment form): the same
// kernel for z-chunks with Lorentz-Bath planes of at most NB bath modes per material, whose
// polarization and bath state (both levels) is loaded into registers at the start of the plane
//
// YB: bf16 bath storage -- one 32-bit word per mode, component and cell holding the value Y^n and
// the increment V = Y^n - Y^{n-1} as a bf16 pair, updated in place (the general kernel's layout);
// one level of words is staged instead of two.
//
// SIG: the simulation has a per-cell sigma(r) map (p.sig): each dispersive cell reads its sigma
// for the drive term and the energy weight (the Lorentz-Bath forms one plane ahead).  A separate
// instantiation, so that the kernels without a map carry none of it.
template <typename T, bool INC, int VX, int A, int NB = 0, bool YB = false, bool SIG = false>
__global__ void __launch_bounds__(Plain3DLayout<T, VX, A, NB>::threads, Plain3DLayout<T, VX, A, NB>::min_blocks)
plain3d_kernel(const Step3DParams<T> p, const __grid_constant__ PlainMaps maps, const __grid_constant__ BathMaps bm,
               int pcur, int ebuf, int hbuf) {
  using namespace plain;
  using L = Plain3DLayout<T, VX, A, NB>;
  static_assert(NB == 0 || (INC && VX == 1), "bath planes: FP32 increment form, one cell per thread");
  static_assert(!YB || (NB > 0 && sizeof(T) == 4), "bf16 bath storage: the FP32 bath form");
  using VV = Vec<T, VX>;
  constexpr int TY = L::TY, TX = L::TX, NE = L::NE, NH = L::NH;
  constexpr unsigned SZ = sizeof(T), ES = L::ES, HS = L::HS, XS = L::XS;
  constexpr unsigned RT = TX * SZ;              // a frame row (bytes)
  constexpr unsigned CM = TY * RT, CR = RT;     // component strides of main parts and of single rows
  constexpr unsigned CP8 = TY * 4 * SZ, CP1 = 4 * SZ;   // ... of the side columns
  constexpr unsigned CX = (TY + 1) * RT;        // H^n buffer: component stride
  extern __shared__ __align__(128) unsigned char smem_raw_[];
  // the dynamic shared memory, aligned to 128 bytes for the tensor copies
  unsigned char* smem_raw = smem_raw_ + ((128u - (smem_u32(smem_raw_) & 127u)) & 127u);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + L::OFF_MBAR);
  int* sInfo = reinterpret_cast<int*>(smem_raw + L::OFF_INFO);
  __shared__ int s_abort;
  auto at = [&](unsigned off) -> unsigned char* { return smem_raw + off; };
  auto ldf = [&](unsigned off) -> T { return *reinterpret_cast<const T*>(smem_raw + off); };

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  constexpr bool HELPER = L::HELPER;
  const bool helper = HELPER && w == TY;
  // the bath form's second thread of a cell (modes NBH.. of the cells of tile row w - TY)
  constexpr int SPLIT = L::SPLIT, NBH = L::NBH;
  const bool secondary = SPLIT > 1 && w >= TY;
  const int wrow = NB > 0 ? w % TY : w;   // the tile row of the thread's cells
  // the thread that issues the tensor copies: the helper's lane 0, else lane 0 of warp 0
  const bool issuer = (HELPER ? w == TY : w == 0) && lane == 0;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int i0 = x0 + VX * lane, j = y0 + wrow;
  // the host runs this kernel only when the tiles cover the grid exactly (nx % TX == 0, ny % 8 == 0)
  const bool own = !helper && !secondary;
  const int chunk = p.chunk_ids[blockIdx.z];
  const int zb = p.zstart[chunk], ze = p.zstart[chunk + 1];
  const int np = ze - zb;
  const int plane = (int)p.plane, ncell = (int)p.ncell;
  const int qxy = own || secondary ? j * p.nx + i0 : 0;
  const T dt = p.dt, S = p.S;
  const int nmc = (int)p.nmatcell;
  const int nbx32 = p.nx / 32;
  const int slot_row = blockIdx.y;   // 32 x 8 partial-sum slots: the tile's rows
  // frame byte offsets of a row's cells of this lane (relative to a slot): the row (main row w, or
  // the halo row y0-1), the row above it in y (+1), the column after the tile, the H_in row; their
  // component strides; the H^n buffer row (y - y0 + 1)
  struct RowOffs {
    unsigned oR, cR, oJ, cJ, oX, cXc, oH, cH, oS;
  };
  const unsigned cell = (unsigned)(VX * lane) * SZ;
  const RowOffs halo_row{L::E_TOP + cell, CR, L::E_MAIN + cell, CM, L::E_PRT, CP1, L::H_TOP + cell, CR, cell};
  const int wr = w < TY ? w : 0;
  const RowOffs main_row{L::E_MAIN + (unsigned)wr * RT + cell,
                         CM,
                         wr + 1 < TY ? L::E_MAIN + (unsigned)(wr + 1) * RT + cell : L::E_BOT + cell,
                         wr + 1 < TY ? CM : CR,
                         L::E_PR8 + (unsigned)wr * 4 * SZ,
                         CP8,
                         L::H_MAIN + (unsigned)wr * RT + cell,
                         CM,
                         (unsigned)(wr + 1) * RT + cell};
  const unsigned oS = main_row.oS;

  // ---- set-up: mbarriers, per-plane table ----
  if (tid == 0) {
    s_abort = 0;
    for (int a = 0; a <= A; ++a) plain::mbar_init(&mbar[a], 1);
    // streamed modes: per ring slot a "full" barrier (the copies) and an "empty" one (one arrival
    // per warp once it has read the slot)
    for (int r = 0; r < (L::STREAM ? L::R : 0); ++r) {
      plain::mbar_init(&mbar[A + 1 + r], 1);
      plain::mbar_init(&mbar[A + 1 + L::R + r], TY);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (np > kMaxPlanes) s_abort = 1;   // the host plans chunks of at most kMaxPlanes planes
  }
  for (int t = tid; t < np && t < kMaxPlanes; t += L::threads) {
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
    if (k < p.npml || k >= p.nz - p.npml) info |= kPmlE;
    if (p.npml > 0 && (k < p.npml || k >= p.nz - p.npml - 1)) info |= kPmlH;
    if (k + 1 >= p.nz) info |= kTop;
    if ((info & 0xF) && p.mat[(info & 0xF) - 1].kind == kLorentzBath && p.mat[(info & 0xF) - 1].nb > 0)
      info |= kBath;
    sInfo[t] = info;
  }
  T* sCoef = reinterpret_cast<T*>(smem_raw + L::OFF_COEF);   // [modes][kCoefStride]
  if (NB > 0)
    for (int q = tid; q < kCoefStride * p.nmodes; q += L::threads) sCoef[q] = p.coef[q];
  __syncthreads();
  if (s_abort) {
    if (tid == 0) atomicExch(p.err, 1);
    return;
  }

  // ---- staging (the issuer): stage g brings E_in(zb+g+1) (unless past the grid) and H_in(zb+g),
  // stage 0 also E_in(zb); the periodic neighbours are boxes of their own (wrapped coordinates) ----
  const int ym = y0 == 0 ? p.ny - 1 : y0 - 1, yp = y0 + TY == p.ny ? 0 : y0 + TY;
  const int xm = x0 == 0 ? p.nx - 4 : x0 - 4, xp = x0 + TX == p.nx ? 0 : x0 + TX;
  auto stage_bytes = [&](int g) -> unsigned {
    const int nE = (zb + g + 1 < p.nz ? 1 : 0) + (g == 0 ? 1 : 0);
    return nE * L::E_BYTES + L::H_BYTES;
  };
  auto load_e = [&](int kk, uint64_t* bar) {
    const unsigned d = smem_u32(smem_raw) + L::OFF_E + ((kk - zb) % NE) * ES;
    plain::tma_load5(d + L::E_MAIN, &maps.e_main, x0, y0, kk, 0, ebuf, bar);
    plain::tma_load5(d + L::E_TOP, &maps.e_row, x0, ym, kk, 0, ebuf, bar);
    plain::tma_load5(d + L::E_BOT, &maps.e_row, x0, yp, kk, 0, ebuf, bar);
    plain::tma_load5(d + L::E_PL8, &maps.e_pad8, xm, y0, kk, 0, ebuf, bar);
    plain::tma_load5(d + L::E_PLB, &maps.e_pad1, xm, yp, kk, 0, ebuf, bar);
    plain::tma_load5(d + L::E_PRT, &maps.e_pad1, xp, ym, kk, 0, ebuf, bar);
    plain::tma_load5(d + L::E_PR8, &maps.e_pad8, xp, y0, kk, 0, ebuf, bar);
  };
  auto issue_stage = [&](int g) {
    const int k = zb + g;
    uint64_t* bar = &mbar[g % A];
    if (k + 1 < p.nz) load_e(k + 1, bar);
    if (g == 0) load_e(zb, bar);
    const unsigned d = smem_u32(smem_raw) + L::OFF_HIN + (g % NH) * HS;
    plain::tma_load5(d + L::H_MAIN, &maps.h_main, x0, y0, k, 0, hbuf, bar);
    plain::tma_load5(d + L::H_TOP, &maps.h_row, x0, ym, k, 0, hbuf, bar);
    plain::tma_load5(d + L::H_PL8, &maps.h_pad8, xm, y0, k, 0, hbuf, bar);
  };
  // bath form: the bath state of plane zb+g (P^{n+1/2}, Y^n, P^{n-1/2}, Y^{n-1} of the tile) into the
  // bath buffer, completing on mbarrier A; issued after the barrier of the plane before, when the
  // buffer has been read into registers
  unsigned bpar = 0;           // parity of the next bath-state wait
  bool bath_pending = false;   // (issuer) a bath-state copy not yet waited for
  int bath_issued = 0;         // (issuer) bath-state copies issued
  auto issue_bath = [&](int g) {
    const int mi_ = (sInfo[g] & 0xF) - 1;
    const int i = bm.mat[0] == mi_ ? 0 : 1;
    const MatK<T>& M = p.mat[mi_];
    const int z = zb + g - M.zlo;
    uint64_t* bar = &mbar[A];
    // (bf16 pairs: the words have the size of T, one level in place; streamed modes: P only)
    plain::mbar_arrive_expect_tx(bar, ((L::STREAM ? 0u : (YB ? 1u : 2u) * 3u * M.nb) + 6u) * L::BT);
    const unsigned d = smem_u32(smem_raw) + L::OFF_BATH;
    if (!L::STREAM) plain::tma_load4(d, &bm.y[i][pcur], x0, y0, z, 0, bar);
    plain::tma_load4(d + L::B_P, &bm.pp[i][pcur], x0, y0, z, 0, bar);
    if (!YB && !L::STREAM) plain::tma_load4(d + L::B_LVL, &bm.y[i][1 - pcur], x0, y0, z, 0, bar);
    plain::tma_load4(d + L::B_LVL + L::B_P, &bm.pp[i][1 - pcur], x0, y0, z, 0, bar);
    bath_pending = true;
    ++bath_issued;
  };
  // ---- streamed modes (STREAM): batches of MB modes of one component, both levels, in the order
  // of use -- per bath plane of the chunk, per component, the bath-sum pass, then the update pass.
  // The issuer's cursor: bath plane sg (np: none left), component sc, pass sp, batch sb ----
  constexpr int MB = L::MB, R = L::R;
  uint64_t* rfull = mbar + A + 1;
  uint64_t* rempty = mbar + A + 1 + R;
  int sg = np, sc = 0, sp = 0, sb = 0;
  int q_issued = 0;   // (issuer) batches issued
  int q_used = 0;     // batches consumed
  int q_landed = 0;   // batches whose copies this thread saw complete (in order)
  auto next_bath_plane = [&](int g) {
    while (g < np && !(sInfo[g] & kBath)) ++g;
    return g;
  };
  auto issue_batch = [&]() {
    if (sg >= np) return;
    const int mi_ = (sInfo[sg] & 0xF) - 1;
    const int i = bm.mat[0] == mi_ ? 0 : 1;
    const int nbm_ = p.mat[mi_].nb;
    const int slot = q_issued % R;
    uint64_t* bar = &rfull[slot];
    plain::mbar_arrive_expect_tx(bar, 2u * MB * L::BT);
    const unsigned d = smem_u32(smem_raw) + L::OFF_RING + slot * L::RING_SLOT;
    // the box past the component's last mode reads the next component's (or, past the array, the
    // zero fill); those values go unused
    const int z = zb + sg - p.mat[mi_].zlo, m0 = sc * nbm_ + sb * MB;
    plain::tma_load4(d, &bm.y[i][pcur], x0, y0, z, m0, bar);
    plain::tma_load4(d + MB * L::BT, &bm.y[i][1 - pcur], x0, y0, z, m0, bar);
    ++q_issued;
    if (++sb * MB >= nbm_) {
      sb = 0;
      if (++sp == 2) {
        sp = 0;
        if (++sc == 3) {
          sc = 0;
          sg = next_bath_plane(sg + 1);
        }
      }
    }
  };
  if (issuer) {
    for (int g = 0; g < A && g < np; ++g) {
      plain::mbar_arrive_expect_tx(&mbar[g], stage_bytes(g));
      issue_stage(g);
    }
    if constexpr (NB > 0)
      if (np > 0 && (sInfo[0] & kBath)) issue_bath(0);
    if constexpr (L::STREAM) {
      sg = next_bath_plane(0);
      for (int r = 0; r < R; ++r) issue_batch();
    }
  }

  // ---- prologue: H^n of plane zb-1 at the own cells (z-difference of the E update at zb);
  // zb-1 is never inside the CPML (chunk starts are planned that way) ----
  T hxm[VX], hym[VX];
#pragma unroll
  for (int v = 0; v < VX; ++v) hxm[v] = hym[v] = T(0);
  if (zb > 0 && own) {
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      const int i = i0 + v;
      const int q = (zb - 1) * plane + j * p.nx + i;
      const int qj1 = (zb - 1) * plane + ((j + 1) % p.ny) * p.nx + i;
      const int qi1 = (zb - 1) * plane + j * p.nx + (i + 1) % p.nx;
      T hx = p.Hin[q], hy = p.Hin[ncell + q];
      const T dyEz = p.Ein[2 * ncell + qj1] - p.Ein[2 * ncell + q];
      const T dzEy = p.Ein[ncell + q + plane] - p.Ein[ncell + q];
      const T dzEx = p.Ein[q + plane] - p.Ein[q];
      const T dxEz = p.Ein[2 * ncell + qi1] - p.Ein[2 * ncell + q];
      hx = hx - S * (dyEz - dzEy);
      hy = hy - S * (dzEx - dxEz);
      hxm[v] = hx;
      hym[v] = hy;
    }
  }

  T uE = T(0), uP = T(0), uB = T(0), uH = T(0);
  const int pstrE = 2 * p.npml * plane, pstrH = (2 * p.npml + 1) * plane;
  int g_last = 0;        // the plane of the last wait
  bool wait_ok = true;   // that wait succeeded
  auto wait_stage = [&](int g) {
    g_last = g;
    wait_ok = plain::mbar_wait(&mbar[g % A], (unsigned)((g / A) & 1));
    if (!wait_ok) {
      s_abort = 1;
      atomicExch(p.err, 1);
    }
  };
  // H^n of plane k at the thread's VX cells from the staged frames (the own row of a compute warp,
  // the halo row y0-1 for the helper); writes H_x, H_z to the H^n buffer and returns the cells'
  // E_in(k) and H^n.  PML: the plane lies in the CPML of the H update.
  auto h_cells = [&](const RowOffs& o, bool PML, bool top, unsigned e0, unsigned e1, unsigned hin, unsigned xb,
                     T bH, T cH_, T* psHx, T* psHy, T* ex0, T* ey0, T* ez0, T* Hx, T* Hy, T* Hz) {
    const unsigned oR = o.oR, cR = o.cR, oJ = o.oJ, cJ = o.cJ, oX = o.oX, cXc = o.cXc, oH = o.oH, cH = o.cH;
    VV::ld(at(e0 + oR), ex0);
    VV::ld(at(e0 + cR + oR), ey0);
    VV::ld(at(e0 + 2 * cR + oR), ez0);
    T ex1[VX], ey1[VX], ez1[VX], exj[VX], ezj[VX];
    if (!top) {
      VV::ld(at(e1 + oR), ex1);
      VV::ld(at(e1 + cR + oR), ey1);
      VV::ld(at(e1 + 2 * cR + oR), ez1);
    } else {
#pragma unroll
      for (int v = 0; v < VX; ++v) ex1[v] = ey1[v] = ez1[v] = T(0);
    }
    VV::ld(at(e0 + oJ), exj);
    VV::ld(at(e0 + 2 * cJ + oJ), ezj);
    // E_y, E_z after the last cell: the next lane's first cell, or the column x0+TX
    T eyi = __shfl_down_sync(0xffffffffu, ey0[0], 1), ezi = __shfl_down_sync(0xffffffffu, ez0[0], 1);
    if (lane == 31) {
      eyi = ldf(e0 + oX + cXc);
      ezi = ldf(e0 + oX + 2 * cXc);
    }
    VV::ld(at(hin + oH), Hx);
    VV::ld(at(hin + cH + oH), Hy);
    VV::ld(at(hin + 2 * cH + oH), Hz);
#pragma unroll
    for (int v = 0; v < VX; ++v) {
      const T ey_i1 = v + 1 < VX ? ey0[v + 1 < VX ? v + 1 : 0] : eyi;
      const T ez_i1 = v + 1 < VX ? ez0[v + 1 < VX ? v + 1 : 0] : ezi;
      plain::h_cell(Hx[v], Hy[v], Hz[v], psHx[v], psHy[v], ezj[v] - ez0[v], ey1[v] - ey0[v], ex1[v] - ex0[v],
                    ez_i1 - ez0[v], ey_i1 - ey0[v], exj[v] - ex0[v], PML, bH, cH_, S);
    }
    VV::st(at(xb + o.oS), Hx);
    VV::st(at(xb + CX + o.oS), Hz);
  };

  // ---- bath form: a thread's modes [j0, j0 + NBH) of a cell's nbm modes ----
  const int cellx = wrow * TX + lane;   // the cell's index in the tile (bath form: VX = 1)
  // P^{n+1/2}, P^{n-1/2}, Y^n (into bY) and Y^{n-1} (into bV) from the staged bath buffer
  auto bath_read = [&](int j0, int nbm, T (&bPa)[3], T (&bPb)[3], T (&bY)[3][NBH], T (&bV)[3][NBH]) {
    const unsigned cofs = L::OFF_BATH + (unsigned)cellx * SZ;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bPa[c] = ldf(cofs + L::B_P + c * L::BT);
      bPb[c] = ldf(cofs + L::B_LVL + L::B_P + c * L::BT);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int jj = 0; jj < NBH; ++jj)
        if (j0 + jj < nbm) {
          if constexpr (YB) {
            const __nv_bfloat162 q =
                *reinterpret_cast<const __nv_bfloat162*>(at(cofs + (unsigned)(c * nbm + j0 + jj) * L::BT));
            bY[c][jj] = __low2float(q);    // Y^n
            bV[c][jj] = __high2float(q);   // V = Y^n - Y^{n-1}
          } else {
            bY[c][jj] = ldf(cofs + (unsigned)(c * nbm + j0 + jj) * L::BT);
            bV[c][jj] = ldf(cofs + L::B_LVL + (unsigned)(c * nbm + j0 + jj) * L::BT);
          }
        }
  };
  // Eq. Pz_update-LB's bath sum over the thread's modes, three components, modes outer (each
  // coefficient row {k(a+b), -k b, a+b, -(b+1), c, (w dt)^2} read once; ascending j); bV becomes
  // V = Y^n - Y^{n-1} (bf16 pairs: it holds V already)
  auto bath_sum = [&](const T* cfm, int j0, int nbm, T (&bY)[3][NBH], T (&bV)[3][NBH], T (&bsum)[3]) {
#pragma unroll
    for (int jj = 0; jj < NBH; ++jj) {
      if (j0 + jj < nbm) {
        const float4 ca = *reinterpret_cast<const float4*>(cfm + (j0 + jj) * kCoefStride);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (!YB) bV[c][jj] = bY[c][jj] - bV[c][jj];
          bsum[c] = bsum[c] + (ca.x * bY[c][jj] + ca.y * bV[c][jj]);
        }
      }
    }
  };
  // a cell's eps0 w0^2 dt^2 sigma(r) and rho(r)/dt^2 (Eq. EOM_Lorentz's per-cell sigma; the
  // layer's own values without a map)
  auto drive_of = [&](const MatK<T>& M, T sg) -> T {
    if constexpr (SIG) return M.dcE * sg;
    else return M.cE;
  };
  auto weight_of = [&](const MatK<T>& M, T sg) -> T {
    if constexpr (SIG) return sg > T(0) ? M.rho_s / sg : T(0);
    else return M.rho_idt2;
  };
  // Eq. Pz_update-LB (increment form): P^{n+3/2}, its increment, and P^{n+3/2} - P^{n-1/2}
  auto p_update = [&](const MatK<T>& M, T cEr, const T (&bPa)[3], const T (&bPb)[3], const T (&Ev)[3],
                      const T (&bsum)[3], T (&Pn)[3], T (&Vn)[3], T (&dP)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T V0 = bPa[c] - bPb[c];
      T num = cEr * Ev[c] - M.W * bPa[c] + M.c2 * V0;
      num = num - T(0.5) * dt * bsum[c];
      Vn[c] = num * M.inv_A;
      Pn[c] = bPa[c] + Vn[c];
      dP[c] = Vn[c] + V0;
    }
  };
  // Eq. Yzj_finite_difference (increment form) for the thread's modes; Y^{n+3/2} overwrites
  // Y^{n-1/2} (bf16 pairs: the pair (Y^{n+3/2}, its increment) overwrites the word); ub collects (Y^{n+3/2} - Y^{n+1/2})^2 + (w dt)^2 (Y^{n+3/2})^2 per component
  auto bath_modes = [&](const T* cfm, int j0, int nbm, int yB, int mstr, const T (&bY)[3][NBH],
                        const T (&bV)[3][NBH], const T (&dP)[3], T (&ub)[3]) {
#pragma unroll
    for (int jj = 0; jj < NBH; ++jj) {
      if (j0 + jj < nbm) {
        const float4 ca = *reinterpret_cast<const float4*>(cfm + (j0 + jj) * kCoefStride);
        const float2 cb = *reinterpret_cast<const float2*>(cfm + (j0 + jj) * kCoefStride + 4);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T y = bY[c][jj];
          const T Vy = ca.z * y + ca.w * bV[c][jj] + cb.x * dP[c];
          const T Ynew = y + Vy;
          const int q = yB + (c * nbm + j0 + jj) * mstr;
          if constexpr (YB)
            reinterpret_cast<__nv_bfloat162*>(p.Ya)[q] =
                __halves2bfloat162(__float2bfloat16_rn(Ynew), __float2bfloat16_rn(Vy));
          else
            p.Yb[q] = Ynew;
          if (p.eE_on) ub[c] += Vy * Vy + cb.y * Ynew * Ynew;
        }
      }
    }
  };
  // the two halves' exchange buffer: [0..2] E, [3..5] the first half's bath sums, [6..8] the second's
  T* sX = reinterpret_cast<T*>(smem_raw + L::OFF_XCH);
  constexpr int XT = TY * TX;

  if (helper) {
    // ======== helper warp: the halo row y0-1 of H^n, the staging of the planes ahead, and its part
    // in the barriers of the compute warps' reductions ========
    const int gxy = ym * p.nx + i0;   // grid column of the halo-row cells
    for (int g = 0; g < np; ++g) {
      const int k = zb + g;
      const int info = sInfo[g];
      const bool top = (info & kTop) != 0, pmlH = (info & kPmlH) != 0;
      const int ipH = k < p.npml ? k : k - p.nz + 1 + 2 * p.npml;
      const unsigned e0 = L::OFF_E + (g % NE) * ES, e1 = L::OFF_E + ((g + 1) % NE) * ES;
      const unsigned hin = L::OFF_HIN + (g % NH) * HS, xb = L::OFF_SH + (g & 1) * XS;
      double* red = reinterpret_cast<double*>(at(L::OFF_SH + ((g + 1) & 1) * XS));
      T psHx[VX], psHy[VX], ex0[VX], ey0[VX], ez0[VX], Hx[VX], Hy[VX], Hz[VX];
#pragma unroll
      for (int v = 0; v < VX; ++v) psHx[v] = psHy[v] = T(0);
      if (pmlH) {
        VV::ld(p.psiHin + ipH * plane + gxy, psHx);
        VV::ld(p.psiHin + pstrH + ipH * plane + gxy, psHy);
      }
      wait_stage(g);
      if (pmlH)
        h_cells(halo_row, true, top, e0, e1, hin, xb, p.pmlH[2 * k], p.pmlH[2 * k + 1], psHx, psHy, ex0, ey0, ez0,
                Hx, Hy, Hz);
      else
        h_cells(halo_row, false, top, e0, e1, hin, xb, T(1), T(0), psHx, psHy, ex0, ey0, ez0, Hx, Hy, Hz);
      // arm the mbarrier of stage g+A (the one of stage g) before the barrier, once stage g's phase
      // has completed: the new phase cannot complete before its copies, issued after the barrier
      if (lane == 0 && wait_ok && g + A < np) plain::mbar_arrive_expect_tx(&mbar[g % A], stage_bytes(g + A));
      __syncthreads();   // H^n(k) of the tile and its halo complete; E_in(k), H_in(k) slots free
      if (s_abort) break;
      if (lane == 0 && g + A < np) issue_stage(g + A);
      if constexpr (NB > 0)
        if (lane == 0 && g + 1 < np && (sInfo[g + 1] & kBath)) issue_bath(g + 1);
      if (info & kMonH) {
        for (int m = 0; m < p.nmon; ++m) {
          const int zm = p.mon_z[m];
          if (k == zm - 1 || k == zm) {
            double v2[2] = {0.0, 0.0};
            block_slot_sums<TY, VX>(v2, red, w, lane);
            __syncthreads();
          }
        }
      }
      if constexpr (L::STREAM) {
        // the ring: as the compute warps release each batch of this plane, the next one in order
        // of use goes into its slot
        if (lane == 0 && (info & kBath)) {
          const int nbat = (p.mat[(info & 0xF) - 1].nb + MB - 1) / MB;
          for (int t = 0; t < 6 * nbat && !s_abort; ++t) {
            const int slot = q_landed % R;
            if (plain::mbar_wait(&rempty[slot], (unsigned)((q_landed / R) & 1))) {
              ++q_landed;   // released by every compute warp, so landed
              issue_batch();
            } else {
              s_abort = 1;
              atomicExch(p.err, 1);
            }
          }
        }
        __syncwarp();
      }
      if (info & kMonE) {
        for (int m = 0; m < p.nmon; ++m)
          if (k == p.mon_z[m]) {
            double v2[2] = {0.0, 0.0};
            block_slot_sums<TY, VX>(v2, red, w, lane);
            __syncthreads();
          }
      }
    }
  } else if (secondary) {
    // ======== the bath form's second thread of each cell (SPLIT = 2): modes NBH.. of the cells of
    // tile row wrow; the same barriers as the first threads' planes ========
    T sg_ahead = T(0);   // sigma(r) one bath plane ahead, as the first threads load it
    int sg_ahead_k = -1;
    for (int g = 0; g < np; ++g) {
      const int k = zb + g;
      const int info = sInfo[g];
      const bool bathp = (info & kBath) != 0;
      double* red = reinterpret_cast<double*>(at(L::OFF_SH + ((g + 1) & 1) * XS));
      T bPa[3], bPb[3], bY[3][NBH], bV[3][NBH];
      const int mi2 = (info & 0xF) - 1;
      int nbm = 0, yB = 0, mstr = 0;
      T sg = T(0);
      if (bathp) {
        const MatK<T>& M = p.mat[mi2];
        nbm = M.nb;
        yB = (int)M.ybase + (k - M.zlo) * plane + qxy;
        mstr = (int)M.ncell;
        if constexpr (SIG) {
          const int rS = (int)M.base + (k - M.zlo) * plane + qxy;
          sg = sg_ahead_k == k ? sg_ahead : p.sig[rS];
          if (k + 1 < M.zhi) {
            sg_ahead = p.sig[rS + plane];
            sg_ahead_k = k + 1;
          }
        }
        if (!plain::mbar_wait(&mbar[A], bpar)) {
          s_abort = 1;
          atomicExch(p.err, 1);
        }
        bpar ^= 1u;
        bath_read(NBH, nbm, bPa, bPb, bY, bV);
      }
      __syncthreads();   // the plane's barrier
      if (s_abort) break;
      if (info & kMonH) {
        for (int m = 0; m < p.nmon; ++m) {
          const int zm = p.mon_z[m];
          if (k != zm - 1 && k != zm) continue;
          double v2[2] = {0.0, 0.0};
          block_slot_sums<TY, VX>(v2, red, w, lane);
          __syncthreads();
        }
      }
      if (bathp) {
        const MatK<T>& M = p.mat[mi2];
        const T* cfm = sCoef + M.coef_off * kCoefStride;
        T bsum[3] = {T(0), T(0), T(0)};
        bath_sum(cfm, NBH, nbm, bY, bV, bsum);
#pragma unroll
        for (int c = 0; c < 3; ++c) sX[(6 + c) * XT + cellx] = bsum[c];
        __syncthreads();   // E and both halves' bath sums exchanged
        T Ev[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Ev[c] = sX[c * XT + cellx];
          bsum[c] = sX[(3 + c) * XT + cellx] + bsum[c];   // the first half's sum first, as there
        }
        T Pn[3], Vn[3], dP[3];
        p_update(M, drive_of(M, sg), bPa, bPb, Ev, bsum, Pn, Vn, dP);
        T ub[3] = {T(0), T(0), T(0)};
        bath_modes(cfm, NBH, nbm, yB, mstr, bY, bV, dP, ub);
        if (p.eE_on && (info & kBox)) {
          const T wr = weight_of(M, sg);
#pragma unroll
          for (int c = 0; c < 3; ++c) uB += wr * ub[c];
        }
      }
      if (info & kMonE) {
        for (int m = 0; m < p.nmon; ++m) {
          if (k != p.mon_z[m]) continue;
          double v2[2] = {0.0, 0.0};
          block_slot_sums<TY, VX>(v2, red, w, lane);
          __syncthreads();
        }
      }
    }
  } else {
    // ======== compute warps: plane k of the own row.  GEN = false is a plain vacuum plane (no
    // layer, CPML, source, monitor or energy box, not the top plane) ========
    // frame offsets of the halo cell x0-1 of this row (and of the row above it in y)
    const unsigned oL = L::E_PL8 + (unsigned)(w * 4 + 3) * SZ;
    const unsigned oLJ = w + 1 < TY ? L::E_PL8 + (unsigned)((w + 1) * 4 + 3) * SZ : L::E_PLB + 3u * SZ;
    const unsigned cLJ = w + 1 < TY ? CP8 : CP1;
    const unsigned oLH = L::H_PL8 + (unsigned)(w * 4 + 3) * SZ;
    // sigma(r) of the cell one bath plane ahead (with a map): loaded at the start of a plane, used
    // by the next, so the load's latency is covered by a plane of work
    [[maybe_unused]] T sg_ahead = T(0);
    [[maybe_unused]] int sg_ahead_k = -1;
    auto body = [&](auto gen_t, auto bath_t, int g, int info) -> bool {
      constexpr bool GEN = decltype(gen_t)::value;
      constexpr bool BATH = NB > 0 && decltype(bath_t)::value;   // a Lorentz-Bath plane with modes
      const int k = zb + g;
      const int mi = GEN ? (info & 0xF) - 1 : -1;
      const bool in_box = GEN && (info & kBox) != 0;
      const bool top = GEN && (info & kTop) != 0;
      const bool pmlE = GEN && (info & kPmlE) != 0, pmlH = GEN && (info & kPmlH) != 0;
      const int ipE = k < p.npml ? k : k - p.nz + 2 * p.npml;
      const int ipH = k < p.npml ? k : k - p.nz + 1 + 2 * p.npml;
      const unsigned e0 = L::OFF_E + (g % NE) * ES, e1 = L::OFF_E + ((g + 1) % NE) * ES;
      const unsigned hin = L::OFF_HIN + (g % NH) * HS, xb = L::OFF_SH + (g & 1) * XS;
      double* red = reinterpret_cast<double*>(at(L::OFF_SH + ((g + 1) & 1) * XS));   // the other H^n buffer
      T psHx[VX], psHy[VX];
#pragma unroll
      for (int v = 0; v < VX; ++v) psHx[v] = psHy[v] = T(0);
      if (pmlH) {
        VV::ld(p.psiHin + ipH * plane + qxy, psHx);
        VV::ld(p.psiHin + pstrH + ipH * plane + qxy, psHy);
      }
      // bath planes: P^{n+1/2}, P^{n-1/2} and both levels of the bath modes of the cell, read from
      // the staged bath buffer before the plane's barrier (Y^n in bY; Y^{n-1} in bV, which becomes
      // V = Y^n - Y^{n-1} below)
      T bPa[3], bPb[3], bY[3][NBH], bV[3][NBH];
      int rB = 0, yB = 0, mstr = 0, nbm = 0;
      [[maybe_unused]] T sgB = T(0);   // sigma(r) of the cell (with a map)
      if constexpr (BATH) {
        const MatK<T>& M = p.mat[mi];
        const int rl = (k - M.zlo) * plane + qxy;
        rB = (int)M.base + rl;
        yB = (int)M.ybase + rl;
        mstr = (int)M.ncell;
        nbm = M.nb;
        if constexpr (SIG) {
          sgB = sg_ahead_k == k ? sg_ahead : p.sig[rB];
          if (k + 1 < M.zhi) {
            sg_ahead = p.sig[rB + plane];
            sg_ahead_k = k + 1;
          }
        }
      }
      // without the helper: warp 0 also computes the halo row y0-1 (its CPML memories loaded here)
      [[maybe_unused]] T hpsx[VX], hpsy[VX];
      if constexpr (!HELPER) {
#pragma unroll
        for (int v = 0; v < VX; ++v) hpsx[v] = hpsy[v] = T(0);
        if (pmlH && w == 0) {
          const int gxy = ym * p.nx + i0;
          VV::ld(p.psiHin + ipH * plane + gxy, hpsx);
          VV::ld(p.psiHin + pstrH + ipH * plane + gxy, hpsy);
        }
      }
      wait_stage(g);

      // ---- H^n of plane k at the own cells ----
      T ex0[VX], ey0[VX], ez0[VX], Hx[VX], Hy[VX], Hz[VX];
      const T bH = pmlH ? p.pmlH[2 * k] : T(1), cH_ = pmlH ? p.pmlH[2 * k + 1] : T(0);
      if (pmlH)
        h_cells(main_row, true, top, e0, e1, hin, xb, bH, cH_, psHx, psHy, ex0, ey0, ez0, Hx, Hy, Hz);
      else
        h_cells(main_row, false, top, e0, e1, hin, xb, bH, cH_, psHx, psHy, ex0, ey0, ez0, Hx, Hy, Hz);
      {
        const int q = k * plane + qxy;
        VV::st(p.Hout + q, Hx);
        VV::st(p.Hout + ncell + q, Hy);
        VV::st(p.Hout + 2 * ncell + q, Hz);
        if (pmlH) {
          VV::st(p.psiHout + ipH * plane + qxy, psHx);
          VV::st(p.psiHout + pstrH + ipH * plane + qxy, psHy);
        }
      }
      if constexpr (!HELPER) {
        if (w == 0) {
          T hx0[VX], hy0[VX], hz0[VX], hHx[VX], hHy[VX], hHz[VX];
          if (pmlH)
            h_cells(halo_row, true, top, e0, e1, hin, xb, bH, cH_, hpsx, hpsy, hx0, hy0, hz0, hHx, hHy, hHz);
          else
            h_cells(halo_row, false, top, e0, e1, hin, xb, bH, cH_, hpsx, hpsy, hx0, hy0, hz0, hHx, hHy, hHz);
        }
        // arm the mbarrier of stage g+A once stage g's phase has completed (as the helper does)
        if (issuer && wait_ok && g + A < np) plain::mbar_arrive_expect_tx(&mbar[g % A], stage_bytes(g + A));
      }
      // ---- H_y, H_z at x-1 of the thread's first cell: from the lane to the left, or on lane 0
      // recomputed for the halo cell x0-1 of this row ----
      T hyx0 = __shfl_up_sync(0xffffffffu, Hy[VX - 1], 1), hzx0 = __shfl_up_sync(0xffffffffu, Hz[VX - 1], 1);
      if (lane == 0) {
        const T ax = ldf(e0 + oL), ay = ldf(e0 + CP8 + oL), az = ldf(e0 + 2 * CP8 + oL);
        const T bx = top ? T(0) : ldf(e1 + oL), by = top ? T(0) : ldf(e1 + CP8 + oL);
        const T jx = ldf(e0 + oLJ), jz = ldf(e0 + 2 * cLJ + oLJ);
        T hx = ldf(hin + oLH), hy = ldf(hin + CP8 + oLH), hz = ldf(hin + 2 * CP8 + oLH);
        T qx = T(0), qy = T(0);
        if (pmlH) {
          const int gq = j * p.nx + (x0 == 0 ? p.nx - 1 : x0 - 1);
          qx = p.psiHin[ipH * plane + gq];
          qy = p.psiHin[pstrH + ipH * plane + gq];
        }
        // the cell's x+1 neighbour is this lane's first cell (ey0[0], ez0[0])
        plain::h_cell(hx, hy, hz, qx, qy, jz - az, by - ay, bx - ax, ez0[0] - az, ey0[0] - ay, jx - ax, pmlH, bH,
                      cH_, S);
        hyx0 = hy;
        hzx0 = hz;
      }
      if constexpr (BATH) {
        if (plain::mbar_wait(&mbar[A], bpar)) {
          if (issuer) bath_pending = false;
        } else {
          s_abort = 1;
          atomicExch(p.err, 1);
        }
        bpar ^= 1u;
        bath_read(0, L::STREAM ? 0 : nbm, bPa, bPb, bY, bV);   // streamed: P only
      }
      __syncthreads();   // H^n(k) of the tile and its halo complete; E_in(k), H_in(k) slots free
      if (s_abort) return false;
      if constexpr (!HELPER)
        if (issuer && g + A < np) issue_stage(g + A);
      if constexpr (NB > 0)
        if (issuer && g + 1 < np && (sInfo[g + 1] & kBath)) issue_bath(g + 1);

      // ---- E-side CPML memories ----
      T psEx[VX], psEy[VX];
#pragma unroll
      for (int v = 0; v < VX; ++v) psEx[v] = psEy[v] = T(0);
      if (pmlE) {
        VV::ld(p.psiE + ipE * plane + qxy, psEx);
        VV::ld(p.psiE + pstrE + ipE * plane + qxy, psEy);
      }
      // ---- H-side monitor partials (planes zm-1 and zm) and the H energy ----
      if (GEN && (info & kMonH)) {
        for (int m = 0; m < p.nmon; ++m) {
          const int zm = p.mon_z[m];
          if (k != zm - 1 && k != zm) continue;
          const int off = (k == zm) ? 1 : 0;
          double v2[2] = {0.0, 0.0};
#pragma unroll
          for (int v = 0; v < VX; ++v) {
            v2[0] += (double)Hx[v];
            v2[1] += (double)Hy[v];
          }
          block_slot_sums<TY, VX>(v2, red, w, lane);
          if (tid < 2 * VX && p.mon_partial_H) {
            const int qn = tid / VX, h = tid - qn * VX;
            p.mon_partial_H[(int64_t)(4 * m + 2 * qn + off) * p.nbxy + slot_row * nbx32 + blockIdx.x * VX + h] =
                slot_total<TY, VX>(red, qn, h);
          }
          __syncthreads();   // red read before it is rewritten
        }
      }
      if (GEN && p.eH_on && in_box) {
#pragma unroll
        for (int v = 0; v < VX; ++v) uH += Hx[v] * Hx[v] + Hy[v] * Hy[v] + Hz[v] * Hz[v];
      }

      // ---- D/E (Eq. 1a) and P (Eq. Pz_1D_Lorentz) of plane k at the own cells, one component at
      // a time (the material state of a component is loaded, used and stored before the next) ----
      double monE[2] = {0.0, 0.0};   // sums of E_x and E_y over the thread's cells (E monitors)
      T Ev[3];                       // bath planes: E^{n+1/2} of the cell
      {
        T hxy[VX], hzy[VX];   // H_x, H_z at y-1
        VV::ld(at(xb + oS - RT), hxy);
        VV::ld(at(xb + CX + oS - RT), hzy);
        const T bE = pmlE ? p.pmlE[2 * k] : T(1), cE_ = pmlE ? p.pmlE[2 * k + 1] : T(0);
        const int q = k * plane + qxy;
        const MatK<T>* M = mi >= 0 ? &p.mat[mi] : nullptr;
        const int r = mi >= 0 ? (int)M->base + (k - M->zlo) * plane + qxy : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          // the curl differences of component c (Eq. FDTD-1D form, CPML memory on the z term)
          T curl[VX];
#pragma unroll
          for (int v = 0; v < VX; ++v) {
            if (c == 0) {
              const T dyHz = Hz[v] - hzy[v];
              const T dzHy = Hy[v] - hym[v];
              if (pmlE) {
                psEx[v] = bE * psEx[v] + cE_ * dzHy;
                curl[v] = dyHz - (dzHy + psEx[v]);
              } else {
                curl[v] = dyHz - dzHy;
              }
            } else if (c == 1) {
              const T dzHx = Hx[v] - hxm[v];
              const T dxHz = Hz[v] - (v > 0 ? Hz[v > 0 ? v - 1 : 0] : hzx0);
              if (pmlE) {
                psEy[v] = bE * psEy[v] + cE_ * dzHx;
                curl[v] = (dzHx + psEy[v]) - dxHz;
              } else {
                curl[v] = dzHx - dxHz;
              }
            } else {
              const T dxHy = Hy[v] - (v > 0 ? Hy[v > 0 ? v - 1 : 0] : hyx0);
              const T dyHx = Hx[v] - hxy[v];
              curl[v] = dxHy - dyHx;
            }
          }
          const T* e0c = c == 0 ? ex0 : (c == 1 ? ey0 : ez0);
          T Ec[VX];
          if (mi < 0) {
            // outside the layers, with the soft sources of this plane on component c (the host runs
            // this kernel only for simulations whose source planes all lie outside the layers)
            T J[VX];
            bool hasJ = false;
#pragma unroll
            for (int v = 0; v < VX; ++v) J[v] = T(0);
            if (GEN && (info & kSrc)) {
              for (int s = 0; s < p.nsrc; ++s) {
                if (p.src_z[s] != k || p.src_comp[s] != c) continue;
                hasJ = true;
                if (p.src_cos[s]) {
                  T cs[VX], sn[VX];
                  VV::ld(p.src_cos[s] + qxy, cs);
                  VV::ld(p.src_sin[s] + qxy, sn);
#pragma unroll
                  for (int v = 0; v < VX; ++v) J[v] += p.src_a[s] * cs[v] + p.src_b[s] * sn[v];
                } else {
#pragma unroll
                  for (int v = 0; v < VX; ++v) J[v] += p.src_a[s];
                }
              }
            }
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              T e = e0c[v] + S * curl[v];
              if (hasJ) e = e + dt * J[v];
              Ec[v] = e;
            }
            if (GEN && p.eE_on && in_box)
#pragma unroll
              for (int v = 0; v < VX; ++v) uE += Ec[v] * Ec[v];
          } else if (BATH) {
            // D-free form as below, from the P levels in registers; P and the bath modes of the three
            // components are updated together after the loop
            Ec[0] = e0c[0] + (S * curl[0] - (bPa[c] - bPb[c])) * M->inv_eps;
            Ev[c] = Ec[0];
            if (p.eE_on && in_box) uE += M->eps * (Ec[0] * Ec[0]);
          } else {
            T Pa[VX], Pb[VX], D[VX];
            VV::ld(p.Pa + c * nmc + r, Pa);
            VV::ld(p.Pb + c * nmc + r, Pb);
            if (!INC) VV::ld(p.D + c * nmc + r, D);
#pragma unroll
            for (int v = 0; v < VX; ++v) {
              if (!INC) {
                // D^{n+1/2} = D^{n-1/2} + S [curl differences];  E = (1/eps_inf)(D - P^{n+1/2})
                D[v] = D[v] + S * curl[v];
                Ec[v] = M->inv_eps * (D[v] - Pa[v]);
              } else {
                // D-free: E += (dt curl H - (P^{n+1/2} - P^{n-1/2})) / eps_inf
                Ec[v] = e0c[v] + (S * curl[v] - (Pa[v] - Pb[v])) * M->inv_eps;
              }
            }
            if (!INC) VV::st(p.D + c * nmc + r, D);
            if (M->kind != kVacuum) {
              // Eq. Pz_1D_Lorentz (Drude: w0^2 dropped from the restoring term); the new level
              // overwrites P^{n-1}
              T Pn[VX], Sg[VX];
#pragma unroll
              for (int v = 0; v < VX; ++v) Sg[v] = T(0);
              if constexpr (SIG) VV::ld(p.sig + r, Sg);
#pragma unroll
              for (int v = 0; v < VX; ++v) {
                T Vn;
                const T cEr = drive_of(*M, Sg[v]);
                if (!INC) {
                  const T num = cEr * Ec[v] - M->c1m * Pa[v] - M->c2 * Pb[v];
                  Pn[v] = M->inv_A * num;
                  Vn = Pn[v] - Pa[v];
                } else {
                  const T V0 = Pa[v] - Pb[v];
                  const T num = cEr * Ec[v] - M->W * Pa[v] + M->c2 * V0;
                  Vn = num * M->inv_A;
                  Pn[v] = Pa[v] + Vn;
                }
                if (p.eE_on && in_box) uP += weight_of(*M, Sg[v]) * (Vn * Vn + M->w0r2dt2 * Pn[v] * Pn[v]);
              }
              VV::st(p.Pb + c * nmc + r, Pn);
            }
            if (p.eE_on && in_box)
#pragma unroll
              for (int v = 0; v < VX; ++v) uE += M->eps * (Ec[v] * Ec[v]);
          }
          VV::st(p.Eout + c * ncell + q, Ec);
          if (GEN && c < 2)
#pragma unroll
            for (int v = 0; v < VX; ++v) monE[c] += (double)Ec[v];
        }
        if (pmlE) {
          VV::st(p.psiE + ipE * plane + qxy, psEx);
          VV::st(p.psiE + pstrE + ipE * plane + qxy, psEy);
        }
      }
      if constexpr (BATH && L::STREAM) {
        // ---- streamed modes: per component, the bath sum of Eq. Pz_update-LB over the batches
        // as they arrive, P^{n+3/2}, then Eq. Yzj_finite_difference over the same batches again
        // (the general kernel's arithmetic and order, ascending j) ----
        const MatK<T>& M = p.mat[mi];
        const T* cfm = sCoef + M.coef_off * kCoefStride;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T bsum = T(0), ub = T(0), Pn = T(0), Vn = T(0), dP = T(0);
#pragma unroll 1
          for (int pass = 0; pass < 2; ++pass) {
#pragma unroll 1
            for (int j0 = 0; j0 < nbm; j0 += MB) {
              const int slot = q_used % R;
              const unsigned par = (unsigned)((q_used / R) & 1);
              if (!s_abort) {
                if (plain::mbar_wait(&rfull[slot], par)) {
                  ++q_landed;
                } else {
                  s_abort = 1;
                  atomicExch(p.err, 1);
                }
              }
              const unsigned so = L::OFF_RING + slot * L::RING_SLOT + (unsigned)cellx * SZ;
              T ys[MB], vs[MB];
#pragma unroll
              for (int u = 0; u < MB; ++u) {
                ys[u] = ldf(so + u * L::BT);
                vs[u] = ldf(so + (MB + u) * L::BT);
              }
              __syncwarp();
              if (lane == 0) plain::mbar_arrive(&rempty[slot]);   // this warp has read the slot
              if (pass == 0) {
#pragma unroll
                for (int u = 0; u < MB; ++u) {
                  if (j0 + u < nbm) {
                    const float2 ca = *reinterpret_cast<const float2*>(cfm + (j0 + u) * kCoefStride);
                    const T v = ys[u] - vs[u];
                    bsum = bsum + (ca.x * ys[u] + ca.y * v);
                  }
                }
              } else {
#pragma unroll
                for (int u = 0; u < MB; ++u) {
                  if (j0 + u < nbm) {
                    const float4 ca = *reinterpret_cast<const float4*>(cfm + (j0 + u) * kCoefStride);
                    const float2 cb = *reinterpret_cast<const float2*>(cfm + (j0 + u) * kCoefStride + 4);
                    const T y = ys[u], v = y - vs[u];
                    const T Vy = ca.z * y + ca.w * v + cb.x * dP;
                    const T Ynew = y + Vy;
                    p.Yb[yB + (c * nbm + j0 + u) * mstr] = Ynew;   // overwrites Y^{n-1}
                    if (p.eE_on) ub += Vy * Vy + cb.y * Ynew * Ynew;
                  }
                }
              }
              // without the helper, the issuer refills the slot once every warp has read it
              if (!HELPER && issuer && !s_abort) {
                if (plain::mbar_wait(&rempty[slot], par)) {
                  issue_batch();
                } else {
                  s_abort = 1;
                  atomicExch(p.err, 1);
                }
              }
              ++q_used;
            }
            if (pass == 0) {
              const T V0 = bPa[c] - bPb[c];
              T num = drive_of(M, sgB) * Ev[c] - M.W * bPa[c] + M.c2 * V0;
              num = num - T(0.5) * dt * bsum;
              Vn = num * M.inv_A;
              Pn = bPa[c] + Vn;
              p.Pb[c * nmc + rB] = Pn;   // overwrites P^{n-1/2}
              dP = Vn + V0;              // P^{n+3/2} - P^{n-1/2}
            }
          }
          if (p.eE_on && in_box) {
            const T wr = weight_of(M, sgB);
            uP += wr * (Vn * Vn + M.w0r2dt2 * Pn * Pn);
            uB += wr * ub;
          }
        }
      } else if constexpr (BATH) {
        // ---- Eq. Pz_update-LB and Eq. Yzj_finite_difference (increment form) for the three
        // components, modes outer (with SPLIT = 2 this thread's half of the modes; the halves
        // exchange their bath sums and both form the same P^{n+3/2}) ----
        const MatK<T>& M = p.mat[mi];
        const T* cfm = sCoef + M.coef_off * kCoefStride;
        T bsum[3] = {T(0), T(0), T(0)};
        bath_sum(cfm, 0, nbm, bY, bV, bsum);
        if constexpr (SPLIT > 1) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sX[c * XT + cellx] = Ev[c];
            sX[(3 + c) * XT + cellx] = bsum[c];
          }
          __syncthreads();   // E and both halves' bath sums exchanged
#pragma unroll
          for (int c = 0; c < 3; ++c) bsum[c] = bsum[c] + sX[(6 + c) * XT + cellx];
        }
        T Pn[3], Vn[3], dP[3];
        p_update(M, drive_of(M, sgB), bPa, bPb, Ev, bsum, Pn, Vn, dP);
#pragma unroll
        for (int c = 0; c < 3; ++c) p.Pb[c * nmc + rB] = Pn[c];   // overwrites P^{n-1/2}
        T ub[3] = {T(0), T(0), T(0)};
        bath_modes(cfm, 0, nbm, yB, mstr, bY, bV, dP, ub);
        if (p.eE_on && in_box) {
          const T wr = weight_of(M, sgB);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            uP += wr * (Vn[c] * Vn[c] + M.w0r2dt2 * Pn[c] * Pn[c]);
            uB += wr * ub[c];
          }
        }
      }
      // ---- E-side monitor partials ----
      if (GEN && (info & kMonE)) {
        for (int m = 0; m < p.nmon; ++m) {
          if (k != p.mon_z[m]) continue;
          double v2[2] = {monE[0], monE[1]};
          block_slot_sums<TY, VX>(v2, red, w, lane);
          if (tid < 2 * VX && p.mon_partial_E) {
            const int qn = tid / VX, h = tid - qn * VX;
            p.mon_partial_E[(int64_t)(2 * m + qn) * p.nbxy + slot_row * nbx32 + blockIdx.x * VX + h] =
                slot_total<TY, VX>(red, qn, h);
          }
          __syncthreads();   // red read before it is rewritten
        }
      }
      // ---- H^n(k) of the own cells: the next plane's z-difference ----
#pragma unroll
      for (int v = 0; v < VX; ++v) {
        hxm[v] = Hx[v];
        hym[v] = Hy[v];
      }
      return true;
    };
    for (int g = 0; g < np; ++g) {
      const int info = sInfo[g];
      bool ok;
      if (info == 0)
        ok = body(std::false_type{}, std::false_type{}, g, info);
      else if (NB > 0 && (info & kBath))
        ok = body(std::true_type{}, std::true_type{}, g, info);
      else
        ok = body(std::true_type{}, std::false_type{}, g, info);
      if (!ok) break;
    }
  }
  // after an abort: a bounded wait for the stage that ran out and those issued after it, so that no
  // copy is in flight into this CTA's shared memory when it exits (a stage armed but not issued
  // has no copies)
  if (s_abort && issuer) {
    for (int g = wait_ok ? g_last + 1 : g_last; g < np && g < g_last + A; ++g)
      plain::mbar_wait(&mbar[g % A], (unsigned)((g / A) & 1));
    if (NB > 0 && !HELPER && bath_pending) plain::mbar_wait(&mbar[A], bpar);
    if (NB > 0 && HELPER && bath_issued > 0) plain::mbar_wait(&mbar[A], (unsigned)((bath_issued - 1) & 1));
    // streamed modes issued whose completion this thread has not seen
    for (int q = q_landed; q < q_issued; ++q) plain::mbar_wait(&rfull[q % R], (unsigned)((q / R) & 1));
  }
  // ---- energy partials of this block, one per 32 x 8 slot (zero outside the box) ----
  if constexpr (SPLIT > 1) {
    // the second threads' bath energy joins the first threads' before the block sums
    if (p.eE_on) {
      __syncthreads();
      if (secondary) sX[cellx] = uB;
      __syncthreads();
      if (!secondary) uB += sX[cellx];
    }
  }
  if (p.eE_on || p.eH_on) {
    __syncthreads();
    double* red = reinterpret_cast<double*>(at(L::OFF_SH));
    T u4[4] = {uE, uP, uB, uH};
    block_slot_sums<TY, VX>(u4, red, w, lane);
    if (tid < 4 * VX) {
      const int qn = tid / VX, h = tid - qn * VX;
      const int64_t slot = (int64_t)chunk * p.nbxy + slot_row * nbx32 + blockIdx.x * VX + h;
      const double s = slot_total<TY, VX>(red, qn, h);
      if (qn < 3 && p.eE_on) p.en_partial_E[(int64_t)qn * p.nbxy * p.nchunks_total + slot] = s;
      if (qn == 3 && p.eH_on) p.en_partial_H[slot] = s;
    }
  }
}

}  // namespace fdtdbath
