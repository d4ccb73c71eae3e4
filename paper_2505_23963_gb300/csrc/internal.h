// internal.h -- data structures shared by the host planner (api.cpp) and the kernels.
//
// State layout in HBM (one simulation):
//   E, H        : two buffers each (ping-pong), [3][nz][ny][nx]; one launch reads the
//                 "in" buffer (halo neighbours included) and writes the "out" buffer.
//   psiE        : CPML memories of the E update, [2][2*npml][ny][nx], updated in place by the
//                 single-step kernels; a second buffer for the two-steps-per-pass kernel.
//   psiH        : CPML memories of the H update, two buffers, [2][2*npml+1][ny][nx].
//   D           : FP64 path only, [3][material cells] (material planes only).
//   Pa / Pb     : P^{n+1/2} and P^{n-1/2} slots; the new P^{n+3/2} overwrites the older
//                 slot and the host swaps the two pointers each step (both precisions).
//   Ya / Yb     : the same two slots for every bath mode, [3][nb][cells] per
//                 Lorentz-Bath material (material-only storage).
//   partial     : per-block FP64 partial sums of the monitor planes and of the energy box,
//                 reduced in a fixed order by reduce.cu.
#pragma once

#include <cuda.h>

#include <cstdint>

namespace fdtdbath {

constexpr int kMaxMat = 8;
constexpr int kMaxSrc = 4;
constexpr int kMaxMon = 4;
constexpr int kMaxBath = 32;       // bath modes per material: 1D cavity kernel, batch and adjoint
constexpr int kMaxBathStep = 128;  // bath modes per material: the 3D / 2D step kernel (streamed above 32)
constexpr int kTX = 32;
constexpr int kCoefStride = 8;  // coefficient row per bath mode
constexpr int kMaxChunk = 128;  // planes per z-chunk (the per-plane table in shared memory)

enum Kind { kVacuum = 0, kLorentz = 1, kDrude = 2, kLorentzBath = 3 };

#ifdef __CUDACC__
// The literal (FP64) form of the bath recursion with fused multiply-adds, the same sequence in
// every kernel that runs it (one rounding per FMA; the other FP64 arithmetic is uncontracted):
//   bath sum term   k_j (a_j Y^n + b_j Y^{n-1}),           Eq. Pz_update-LB
//   new mode        a_j Y^n + (b_j+1) Y^{n-1} + c_j dP,    Eq. Yzj_finite_difference
//   energy term     (Y^{n+1} - Y^n)^2 + (w_j dt)^2 (Y^{n+1})^2
template <typename T>
__device__ __forceinline__ T bath_sum_lit(T bsum, T k, T a, T b, T y, T ym) {
  return fma(k, fma(a, y, b * ym), bsum);
}
template <typename T>
__device__ __forceinline__ T bath_new_lit(T a, T b1, T c, T y, T ym, T dP) {
  return fma(c, dP, fma(a, y, b1 * ym));
}
template <typename T>
__device__ __forceinline__ T bath_energy_lit(T ub, T vy, T w2, T yn) {
  return fma(vy, vy, fma(w2 * yn, yn, ub));
}
#endif

template <typename T>
struct MatK {
  int zlo, zhi, kind, nb;
  int64_t base;   // first cell of this material in the pooled material arrays
  int64_t ybase;  // first element of this material's bath block in Ya / Yb
  int64_t ncell;  // cells of this material
  int coef_off;   // first row of this material's modes in coef[]
  T eps;          // eps_inf
  T cE;           // eps0 w0^2 dt^2 sigma
  T c1m;          // w0^2 dt^2 - 2 (Drude: -2)         [FP64 path]
  T W;            // w0^2 dt^2 (Drude: 0)                [FP32 increment path]
  T c2;           // 1 - gamma0 dt/2 - dt/2 sum_j k_j c_j
  T A;            // 1 + gamma0 dt/2 + dt/2 sum_j k_j c_j
  T inv_A;        // 1/A (1/(1 + gamma dt/2) without a bath)
  T inv_eps;      // 1/eps_inf
  T rho_idt2;     // rho/dt^2, rho = 1/(sigma w0^2) (0 when sigma = 0), energy density
  T w0r2dt2;      // (w0 dt)^2 in the potential term (Drude: 0)
  // with a per-cell oscillator strength sigma(r) (Eq. EOM_Lorentz): cE = dcE sigma(r),
  // rho/dt^2 = rho_s / sigma(r) (0 where sigma(r) = 0)
  T dcE;          // w0^2 dt^2 (0 for a vacuum layer)
  T rho_s;        // 1/(w0^2 dt^2)
};

// Per bath mode j (coefficient row of kCoefStride values):
//   FP64 path : {k_j, a_j, b_j, b_j + 1, c_j, (w_j dt)^2}
//   FP32 path : {k_j (a_j + b_j), -k_j b_j, a_j + b_j, -(b_j + 1), c_j, (w_j dt)^2}  (increment arithmetic)

template <typename T>
struct Step3DParams {
  int nx, ny, nz;
  int64_t plane, ncell;
  T dt, S;   // time step and Courant factor S = dt/dx
  const T* Ein;
  T* Eout;
  const T* Hin;
  T* Hout;
  int doH, doE;
  // CPML
  int npml;
  const T* pmlE;  // [nz][2] = (b, c) at integer z
  const T* pmlH;  // [nz][2] = (b, c) at z + 1/2
  T* psiE;        // [2][2*npml][plane]
  const T* psiHin;
  T* psiHout;     // [2][2*npml+1][plane]
  // materials
  int nmat;
  MatK<T> mat[kMaxMat];
  const T* coef;   // [nmodes][kCoefStride], staged into shared memory by every CTA
  int nmodes;
  T* D;
  T* Pa;
  T* Pb;
  T* Ya;
  T* Yb;
  int64_t nmatcell;
  const T* sig;   // sigma(r) per material cell (pooled like P), or null: every layer's own sigma
  // sources: J(x, y) = src_a * cos(phase) + src_b * sin(phase)   (src_b unused without phase)
  int nsrc;
  int src_comp[kMaxSrc];
  int src_z[kMaxSrc];
  T src_a[kMaxSrc];
  T src_b[kMaxSrc];
  const T* src_cos[kMaxSrc];
  const T* src_sin[kMaxSrc];
  // monitors and energy partial sums
  int nmon;
  int mon_z[kMaxMon];
  double* mon_partial_E;  // [2*nmon][nbxy] for this launch's E step (or null)
  double* mon_partial_H;  // [4*nmon][nbxy] for this launch's H step (or null)
  int eE_on, eH_on;       // energy of E / H parts recorded in this launch
  int ebox_lo, ebox_hi;
  double* en_partial_E;   // [3][nblocks]
  double* en_partial_H;   // [1][nblocks]
  double ew;              // dx / (nx ny)
  // z chunks (at most 128 planes each); block z of this launch works on chunk chunk_ids[z]
  const int* zstart;      // [nchunks_total + 1]
  const int* chunk_ids;
  int nchunks_total;
  int nbxy;               // partial-sum slots per z-chunk (the (x, y) tiles of the 32 x 8 tiling)
  int vec16;              // nx is a multiple of 16 bytes' worth of elements: 16-byte staging
  int* err;               // device flag set when a bounded wait for an asynchronous copy ran out
};

// Persistent 1D cavity kernel (nx = ny = 1, x polarization): all steps of a call in one launch,
// one cluster of up to 16 CTAs of kCav1DThreads threads per cavity, one cell per thread, the
// state in registers.
constexpr int kCav1DThreads = 512;
constexpr int kCav1DMaxCluster = 16;
template <typename T>
struct Cav1DParams {
  int nz, npml;
  int bounds[kCav1DMaxCluster + 1];   // cell range of CTA r: [bounds[r], bounds[r+1])
  T S, dt;
  T* E;                               // [3][nz]; only E_x (component 0) is used
  T* H;                               // [3][nz]; only H_y (component 1) is used
  T* D;
  T* Pslot[2];
  T* Yslot[2];
  int pcur0;                          // slot holding P^{n+1/2} at the first step of the launch
  const T* sig;                       // sigma(r) per material cell, or null (the layer's sigma)
  const T* coef;
  int nmat;
  MatK<T> mat[kMaxMat];
  const T* pmlE;
  const T* pmlH;
  T* psiE;
  T* psiH;
  int psiH_stride;
  int nsrc, src_z;
  const double* src_tab;              // source amplitude of each step of the launch
  int nmon, mon_z;
  int energy_on, every, ebox_lo, ebox_hi;
  double* partial;
  int ring_cap;
  int64_t ring_stride, monE_off, monH_off, enE_off, enH_off;
  int64_t step0;
  int nsteps;
};
int launch_cavity1d_f32(const Cav1DParams<float>& p, int nbmax, int cluster, void* stream);
int launch_cavity1d_f64(const Cav1DParams<double>& p, int nbmax, int cluster, void* stream);

// Launchers (defined in step3d_f32.cu / step3d_f64.cu).
// te = 1: the y-invariant TE form (ny = 1, sources on E_y only): E_x, E_z, H_y, P_x, P_z and the
// x / z bath modes are known to be zero and are neither read nor written.
int launch_step3d_f32(const Step3DParams<float>& p, int nbmax, int ty, int nbx, int nby,
                      int nchunks, int bath_bf16, int te, void* stream);
int launch_step3d_f64(const Step3DParams<double>& p, int nbmax, int ty, int nbx, int nby,
                      int nchunks, int te, void* stream);
// The plain-plane step (plain3d.cuh): chunks without bath modes of at most 64 planes, grids tiled
// exactly by its (32 VX) x 8 tiles, H and E half-steps together.  Its frames are staged by tensor
// copies described by these maps: the E and H arrays, each one allocation of two buffers, as 5-D
// tensors (x, y, z, component, buffer); boxes of (x, y) extent the tile's rows (TX x 8), one row
// (TX x 1) and the 4-cell side columns (4 x 8, 4 x 1), all three components at once.
struct PlainMaps {
  CUtensorMap e_main, e_row, e_pad8, e_pad1;
  CUtensorMap h_main, h_row, h_pad8;
};
// tile width: four FP32 or two FP64 cells per thread (16-byte vectors), 32 threads per row
constexpr int plain_tile_x(int prec) { return prec == 64 ? 64 : 128; }
int launch_plain3d_f32(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                       void* stream);
// The Lorentz-Bath chunks (FP32, one cell per thread -- two with more than 8 modes --, tiles
// 32 x 8 with maps of that box width, nb = the largest number of bath modes of a material: at
// most 16).  The polarization and bath
// modes of a plane (both levels) are staged by tensor copies too, from these maps: per
// Lorentz-Bath material with modes (at most 2) and per state slot (the two P / Y buffers, whose
// roles swap every step), P as a 4-D tensor (x, y, z in the layer, component) and the modes as
// (x, y, z in the layer, component * nb + mode), boxes of one 32 x 8 plane tile.
constexpr int kBathTileX = 32;
constexpr int kBathPlainMaxModes = 128;
constexpr int kBathPlainRegModes = 16;   // above: the streamed form (FP32 bath storage only)
constexpr int kStreamCoefRows = 256;     // the streamed form's coefficient rows (all materials)
constexpr int kStreamBatchModes = 8;     // modes of one component per streamed batch
constexpr int kBathPlainMaxMats = 2;
struct BathMaps {
  int nmat;                                   // materials with maps
  int mat[kBathPlainMaxMats];                 // their indices in Step3DParams::mat
  CUtensorMap y[kBathPlainMaxMats][2];        // [material][slot]
  CUtensorMap pp[kBathPlainMaxMats][2];       // [material][slot]
};
// ybf: bf16 bath storage (the modes as in-place (value, increment) pairs, maps y[i][0] = y[i][1]
// over them; at most 16 modes)
int launch_bath3d_f32(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur, int ebuf,
                      int hbuf, int nchunks, int nb, int ybf, void* stream);
// the same two launches with a per-cell sigma(r) map (p.sig), from their own translation unit
int launch_plain3d_sig_f32(const Step3DParams<float>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                           void* stream);
int launch_bath3d_sig_f32(const Step3DParams<float>& p, const PlainMaps& maps, const BathMaps& bmaps, int pcur,
                          int ebuf, int hbuf, int nchunks, int nb, int ybf, void* stream);
// The y-invariant TE form's z-chunks (te2d.cuh): FP32, nx a multiple of kTe2dTileX, both
// half-steps of a step; nb = 0 the chunks without bath modes, nb <= kTe2dMaxModes those with.
constexpr int kTe2dTileX = 256;
constexpr int kTe2dMaxModes = 8;
int launch_te2d_f32(const Step3DParams<float>& p, int nchunks, int nb, void* stream);
// both kinds in one launch: p.chunk_ids lists the nplain chunks without bath modes, then nbath
int launch_te2d_fused_f32(const Step3DParams<float>& p, int nplain, int nbath, int nb, void* stream);
int launch_plain3d_f64(const Step3DParams<double>& p, const PlainMaps& maps, int ebuf, int hbuf, int nchunks,
                       void* stream);

// Two steps per pass (tb2.cuh) over grids without polarizable material: 32 x 8 tiles, grids tiled
// exactly by them.  p describes step n (fields and CPML memories in / out, its sources and partial
// rows); the rest, step n+1.  Every output goes to the other buffer: E, H, psiH as p.Eout / p.Hout /
// p.psiHout, the E-side memories to psiEout.
constexpr int kTbTX = 32, kTbTY = 8;
template <typename T>
struct Tb2Params {
  Step3DParams<T> p;
  T* psiEout;
  T src_a2[kMaxSrc], src_b2[kMaxSrc];    // source amplitudes of step n+1
  double* mon_partial_E2;                // partial rows of step n+1
  double* mon_partial_H2;
  double* en_partial_E2;
  double* en_partial_H2;
  int eE_on2, eH_on2;
};
int launch_tb2_f32(const Tb2Params<float>& q, int nchunks, void* stream);
int launch_tb2_f64(const Tb2Params<double>& q, int nchunks, void* stream);

// ---- discrete adjoint (adjoint.cu) ----
// One reverse step of the exact transpose of the forward step (D-free form), applied to the
// adjoint state (Eb, Hb, psi memories, P / P_m and bath-mode adjoints); see adjoint.cu.
constexpr int kAdjMaxGrad = 2 + kMaxBath;   // dL/dsigma, dL/dgamma0, dL/dk_j

// Division of dividends n < 2^31 by a run-time invariant divisor 1 <= d < 2^31 with a
// multiply-high (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, and
// n / d = (mulhi(m, n) + n) >> l; the 33-bit multiplier 2^32 + m is split so that the sum
// stays below 2^32 for n < 2^31.
struct FastDiv {
  uint32_t m;
  int l;
};
inline FastDiv make_fastdiv(uint32_t d) {
  int l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
  return FastDiv{(uint32_t)m, l};
}
template <typename T>
struct AdjParams {
  int nx, ny, nz, npml;
  int64_t plane, ncell, nmatcell;
  T S, dt;
  const T* pmlE;            // [nz][2] (b, c) at integer z
  const T* pmlH;            // [nz][2] (b, c) at z + 1/2
  T* Eb;                    // [3][ncell] adjoint of E
  T* Hb;                    // [3][ncell] adjoint of H
  T* psiEb;                 // [2][2 npml][plane]   adjoint of the E-side CPML memories (in place)
  T* psiEb_out;             // [2][2 npml][plane]   b_E-scaled copy for the next reverse step
  const T* psiHb;           // [2][2 npml + 1][plane]
  T* psiHb_out;
  int nmat;
  MatK<T> mat[kMaxMat];
  const T* coefLit;         // [rows][kCoefStride] literal rows {k, a, b, b+1, c, (w dt)^2}
  T* Pb;                    // [3][nmatcell] adjoint of P^{n+3/2} on entry, of P^{n+1/2} on exit
  T* Pmb;                   // adjoint of P^{n+1/2} on entry, of P^{n-1/2} on exit
  T* Yb0;                   // bath modes, the same two roles as Pb / Pmb
  T* Yb1;
  // monitor sources of this reverse step (dL/d of the plane means, divided by the plane size)
  int zm;                   // monitor plane, -1 for none
  T gEx, gEy, gHx, gHy;
  // gradient of the material gm (-1: none) from the forward values recorded for this step
  int gm;
  const T* fE;              // E^{n+1/2}   [3][ncell_gm]
  const T* fPn;             // P^{n+3/2}
  const T* fPm;             // P^{n-1/2}
  const T* fY;              // Y^{n+1/2}   [3][nb][ncell_gm]
  const T* fYm;             // Y^{n-1/2}
  double dcE;               // d cE / d sigma = (w0 dt)^2
  double halfdt, invA;
  double ga[kMaxBath], gb[kMaxBath], gk[kMaxBath], gdc[kMaxBath], gds[kMaxBath];
  // the same factors rounded once to the state type on the host, as the kernel uses them
  T tsig, thA;              // (T)(dcE invA), (T)(halfdt invA)
  T ta[kMaxBath], tb[kMaxBath], tdc[kMaxBath], tds[kMaxBath];
  double* gpart;            // [gridDim][kAdjMaxGrad] per-block running sums (FP64)
  FastDiv fd_plane, fd_nx;  // division by plane = nx ny and by nx (cell index -> i, j, k)
  const signed char* zmat;  // [nz] material index of every plane, -1 for none
  // cells [ra, rb): the planes from the first material's to the last's (adjoint_k1 runs them and
  // the rest in two launches; set by the launcher)
  int64_t ra, rb;
};
// te = 1: the TE form (the forward run was the y-invariant TE form and the adjoint sources sit
// on E_y and H_x only): the adjoints of E_x, E_z, H_y, P_x, P_z and the x / z bath modes are zero
int launch_adjoint_f32(const AdjParams<float>& p, int nbmax, int te, void* stream);
int launch_adjoint_f64(const AdjParams<double>& p, int nbmax, int te, void* stream);
int64_t adjoint_blocks(int64_t ncell);

// reduce.cu: fixed-order reduction of the per-block partials into per-step series,
// running DFT accumulation and energy traces.
struct ReduceParams {
  const double* partial;  // ring of per-step partial blocks
  int64_t ring_stride;    // doubles per ring step
  int ring_cap;           // steps in the ring
  int nmon;
  int nbxy, nblocks;
  int64_t mon_E_off, mon_H_off, en_E_off, en_H_off;  // offsets inside one ring step
  int energy_on;
  int64_t step_lo, step_hi;  // global steps to reduce: [lo, hi)
  int every;                 // energy recorded on steps with step % every == 0
  double* series;            // [ring_cap][6*nmon + 4]
};
int launch_reduce_series(const ReduceParams& r, void* stream);

struct DftParams {
  const double* series;
  int ring_cap, series_stride;
  int nmon;
  int64_t step_lo, step_hi;
  double dt;
  const double* freqs[kMaxMon];
  int nfreq[kMaxMon];
  double* acc[kMaxMon];   // [nfreq][8]
  int energy_on, every;
  double* trace;          // [cap][4]
  int64_t trace_cap;
  double inv_plane;       // 1/(nx ny)
  double ew;              // dx/(nx ny)
};
int launch_dft_accumulate(const DftParams& d, void* stream);

// Read-only view of a simulation's current device state (after its pending H half-step has
// been flushed), for entry points defined outside api.cpp.
struct SimViewMat {
  int kind, nb;
  int64_t zlo, zhi, ncell, base, ybase;
  double eps, rho, w0r2;
  double wj2[kMaxBathStep];
};
struct SimView {
  int prec;                 // 32 or 64
  int inc;                  // 1: Pb/Yb hold increments X^{n+1/2} - X^{n-1/2}; 0: the older level
  int64_t nx, ny, nz, plane, ncell, nmatcell;
  double dx, dt;
  const void* E;            // [3][ncell], E^{n-1/2}
  const void* H;            // [3][ncell], H^n
  const void* Pa;           // P^{n+1/2}
  const void* Pb;           // P^{n-1/2}
  const void* Ya;
  const void* Yb;
  int nmat;
  SimViewMat mat[kMaxMat];
  void* stream;
  int device;
};

}  // namespace fdtdbath

struct fdtdbath_sim;
// Implemented in api.cpp: flush the pending H half-step and describe the state; record errors.
int fdtdbath_internal_view(fdtdbath_sim* s, fdtdbath::SimView* v);
int fdtdbath_internal_fail(fdtdbath_sim* s, int code, const char* msg);
