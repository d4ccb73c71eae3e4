// api.cpp -- host planner and C ABI of the FDTD-Bath library (see include/fdtdbath.h).
//
// The planner validates a problem, expands the per-material coefficients of the explicit
// ADE updates (Eq. Pz_1D_Lorentz, Pz_update-LB, Yzj_finite_difference), builds the CPML
// profiles, sizes and allocates the device state, plans the z-chunks of the fused step
// kernel and drives it: one launch per step, the H half-step of step n folded into the
// launch of step n+1 (an "H pending" flag carries it across calls), and a fixed-order
// reduction of the monitor / energy partial sums every few hundred steps.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fdtdbath.h"
#include "host_common.h"
#include "internal.h"

using namespace fdtdbath;

namespace {

thread_local std::string g_create_error;

struct HostSrc {
  int comp;
  int64_t z;
  double nu, fwidth, amp, t0;
  bool has_phase;
  void *dcos, *dsin;
  double phase1d;   // the phase of a 1D run (one transverse cell)
};

struct HostMon {
  int64_t z;
  int nfreq;
  void* dfreq;
  void* dacc;
};

}  // namespace

// Checkpoints of the adjoint driver: full states every `every` steps of the recorded forward run
// (plus the state at its end), and the buffers of the reverse sweep.
struct AdjState {
  bool recorded = false;
  int64_t n0 = 0, nsteps = 0;
  int every = 0;
  size_t cp_bytes = 0;
  std::vector<void*> cps;
  std::vector<int64_t> cp_n;
  std::vector<int> cp_pcur;
};

struct fdtdbath_sim {
  int prec = 64;
  size_t esz = 8;
  int64_t nx = 0, ny = 0, nz = 0, plane = 0, ncell = 0;
  double res = 0, courant = 0, dx = 0, dt = 0;
  int npml = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, void*) = nullptr;
  void* uctx = nullptr;
  std::vector<void*> allocs;
  size_t bytes_held = 0;
  // state
  void* E[2] = {nullptr, nullptr};
  void* H[2] = {nullptr, nullptr};
  int ecur = 0, hcur = 0;
  void* psiE = nullptr;
  void* psiH[2] = {nullptr, nullptr};
  int psicur = 0;
  void* pmlE = nullptr;
  void* pmlH = nullptr;
  void* D = nullptr;
  void* Pslot[2] = {nullptr, nullptr};
  void* Yslot[2] = {nullptr, nullptr};
  // bf16 bath storage (precision 32): Yslot[0] holds, per mode and cell, the pair (value Y^{n+1/2},
  // increment Y^{n+1/2} - Y^{n-1/2}) of bf16 in one 32-bit word, updated in place (no slot swap);
  // Yslot[1] is unused
  bool ybf = false;
  size_t yesz = 8;
  int pcur = 0;  // literal form: slot holding P^{n+1/2}
  void* coef = nullptr;
  int64_t nmatcell = 0, nybath = 0;
  std::vector<HostMat> mats;
  std::vector<HostSrc> srcs;
  std::vector<HostMon> mons;
  int64_t e_lo = 0, e_hi = 0, e_cap = 0;
  int e_every = 1;
  bool energy_on = false;
  void* trace = nullptr;
  // partial sums
  int ring_cap = 256;
  int64_t ring_stride = 0, monE_off = 0, monH_off = 0, enE_off = 0, enH_off = 0;
  void* partial = nullptr;
  void* series = nullptr;
  // progress
  int64_t n = 0;           // completed E half-steps (= completed steps)
  bool h_pending = false;  // H^n not yet computed
  int64_t reduced = 0;     // steps whose partials are folded into DFT / trace
  int64_t launches = 0;
  // launch plan
  int ty = 8, nbx = 1, nby = 1, nchunks = 1, nbmax = 0;
  void* zstart = nullptr;
  // chunk ids on the device: [all chunks..., chunks without bath planes..., chunks with them...]
  void* chunk_ids = nullptr;
  int nplain = 0, nbath = 0;
  // a bath-free kernel for the plain chunks runs beside the bath kernel on a forked stream
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // 1D simulations (nx = ny = 1, at most one source and one monitor) run the persistent
  // cavity kernel: one cluster of c1d CTAs, in place, all steps of a call per launch
  bool path1d = false;
  int c1d = 1;
  int ncomp1d = 3;          // 1 while only Ex, Hy, P_x and its bath can be nonzero
  std::vector<int> bounds1d;            // cell range of every CTA of the cluster
  void* src_tab = nullptr;              // per-step source amplitudes of one launch (device)
  int red_nbxy = 1, red_nblocks = 1;   // partial-sum layout seen by the reduction
  int nblk3d = 1;                       // energy partials per step of the 3D kernel
  // quiet: steps record no monitor or energy partials (the adjoint's recomputed segments)
  bool quiet = false;
  // y-invariant TE form: ny = 1 and every source on E_y, so E_x, E_z, H_y, P_x, P_z and the x / z
  // bath modes stay exactly zero and the single-row kernels skip them; cleared for good when a
  // write could make one of them nonzero
  bool te = false;
  bool adj_te = false;      // the last reverse sweep ran the TE form
  // plain-plane kernel (plain3d.cuh) for the chunks without bath planes: grids tiled exactly by
  // its TX x 8 tiles (TX = 128 FP32, 64 FP64 cells), every source plane outside the layers
  bool plain_ok = false;
  PlainMaps maps{};         // its tensor maps of the E and H arrays
  // its Lorentz-Bath form for the bath chunks: FP32, at most 16 bath modes per material in
  // registers (FP32 or bf16 bath storage) or up to 128 streamed (FP32 storage), 32 x 8 tiles;
  // chunks of at most 64 planes
  bool bath_plain = false;
  // the TE form's register-streaming kernel (te2d.cuh) for the chunks without bath planes and
  // (FP32 bath storage, at most 8 modes) those with, while the simulation runs the TE form: FP32,
  // ny = 1, nx a multiple of kTe2dTileX, no source plane inside a layer
  bool te2d_ok = false;
  // per-cell oscillator strength sigma(r) (Eq. EOM_Lorentz), pooled like P, allocated by the first
  // write of the map
  void* sig = nullptr;
  bool sigmap = false;
  bool te2d_ok0 = false;   // the TE kernel's availability at creation
  PlainMaps bmaps{};        // tensor maps of 32-cell-wide boxes
  BathMaps bath_maps{};     // tensor maps of its polarization and bath-mode arrays
  // the bath-free and bath launches of a step one after the other on the simulation's stream (the
  // plain-plane kernel beside the general kernel's bath instantiation: their CTAs lose more to
  // sharing SMs than they gain from overlapping), or concurrently on two streams (otherwise)
  bool serial_pair = false;
  void* errflag = nullptr;  // device int: a bounded wait of a kernel ran out (FDTDBATH_ERR_TIMEOUT)
  // two steps per pass (tb2.cuh): grids without polarizable material tiled exactly by 32 x 8
  // tiles run pairs of steps in one launch; its E-side CPML memories go to the second buffer,
  // and the two pointers swap after each such launch
  bool tb_ok = false;
  void* psiE_alt = nullptr;
  AdjState adj;
  std::string err;
};

namespace {

int fail(fdtdbath_sim* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(fdtdbath_sim* s, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(s, FDTDBATH_ERR_CUDA, m);
}

void* dalloc(fdtdbath_sim* s, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (s->ualloc) {
    p = s->ualloc(bytes, s->uctx);
  } else {
    if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  }
  if (p) {
    s->allocs.push_back(p);
    s->bytes_held += bytes;
    cudaMemsetAsync(p, 0, bytes, s->stream);
  }
  return p;
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double>& v) {
  std::vector<T> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
  return o;
}

int h2d(fdtdbath_sim* s, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaMemcpyAsync H2D");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamSynchronize");
  return 0;
}

int d2h(fdtdbath_sim* s, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaMemcpyAsync D2H");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamSynchronize");
  return 0;
}

// CPML profile of this simulation's z axis (see cpml_coeffs).
void cpml_bc(const fdtdbath_sim* s, double zpos, double* b, double* c) {
  cpml_coeffs(s->npml, s->nz, s->dx, s->dt, zpos, b, c);
}

// Does any Lorentz-Bath layer with bath modes overlap planes [lo, hi)?
bool chunk_has_bath(const fdtdbath_sim* s, int64_t lo, int64_t hi) {
  for (auto& m : s->mats)
    if (m.kind == FDTDBATH_LORENTZ_BATH && m.nb > 0 && m.zlo < hi && m.zhi > lo) return true;
  return false;
}

// z-chunks.  Chunk starts avoid the CPML planes (the chunk-start H recompute needs no CPML
// memory) and fall on every Lorentz-Bath layer boundary inside the allowed range, so that a chunk
// holds either no bath plane or only bath planes (plus whatever the boundary rule forces in).
// Between those cuts, a range of L planes is split into chunks of zc planes (uniform plan), or
// (balanced plan) into a head chunk of ceil(3L/4) planes and a tail chunk of the rest: dispatched
// longest first, the tail chunks of a launch fill its last partial wave of CTAs.
int plan_chunks(fdtdbath_sim* s, int zc, bool balanced, int plain_zc, int bath_zc, int bath_nmin,
                std::vector<int>& starts) {
  starts.clear();
  starts.push_back(0);
  const int64_t lo_ok = s->npml + 1, hi_ok = s->nz - 1 - s->npml;
  std::vector<int64_t> bounds{0, s->nz};
  for (auto& m : s->mats)
    if (m.kind == FDTDBATH_LORENTZ_BATH) {
      if (m.zlo >= lo_ok && m.zlo <= hi_ok) bounds.push_back(m.zlo);
      if (m.zhi >= lo_ok && m.zhi <= hi_ok) bounds.push_back(m.zhi);
    }
  std::sort(bounds.begin(), bounds.end());
  bounds.erase(std::unique(bounds.begin(), bounds.end()), bounds.end());
  int64_t z = 0;
  for (size_t b = 0; b + 1 < bounds.size(); ++b) {
    const int64_t a = bounds[b], e = bounds[b + 1];
    if (z >= e) continue;   // already covered by a chunk the boundary rule extended
    const bool bath = chunk_has_bath(s, z, e);
    const int nzc = bath ? bath_zc : plain_zc;
    if (nzc > 0) {
      // ranges of the plain-plane kernel (without bath planes): near-equal chunks of about nzc
      // planes; of its bath form: near-equal chunks of at most nzc planes, at least bath_nmin
      const int64_t z0 = z, L = e - z0;
      const int64_t n = bath ? std::max<int64_t>((L + nzc - 1) / nzc, std::min<int64_t>(L, bath_nmin))
                             : std::max<int64_t>(1, (L + nzc / 2) / nzc);
      for (int64_t i = 1; i <= n && z < e; ++i) {
        int64_t nx = z0 + (L * i) / n;
        if (nx < lo_ok) nx = lo_ok;
        if (nx > hi_ok) nx = s->nz;
        if (nx > s->nz) nx = s->nz;
        if (nx <= z) continue;
        starts.push_back((int)nx);
        z = nx;
      }
      continue;
    }
    const int64_t step = balanced ? std::max<int64_t>(1, (3 * (e - a) + 3) / 4) : zc;
    while (z < e) {
      int64_t nx = std::min(z + step, e);
      if (nx < lo_ok) nx = lo_ok;
      if (nx > hi_ok) nx = s->nz;
      if (nx > s->nz) nx = s->nz;
      starts.push_back((int)nx);
      z = nx;
    }
  }
  return (int)starts.size() - 1;
}

// Chunk length for the two-steps-per-pass kernel on a grid without polarizable material (one z
// range): the number of chunks n whose CTAs (tiles x n) fill the last wave of resident CTAs best,
// weighed against the three ghost planes each chunk recomputes: maximise
// (waves / ceil(waves)) * (L / (L + 3)), L = nz / n, n = 1 .. 16, chunks of at most 64 planes.
int tb_chunk_planes(const fdtdbath_sim* s) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess || sms <= 0) return 32;
  const double slots = (double)sms * (s->prec == 64 ? 1 : 3);   // resident CTAs (shared memory)
  const double tiles = (double)(s->nx / kTbTX) * (double)(s->ny / kTbTY);
  int best = 32;
  double best_eff = -1.0;
  for (int n = 1; n <= 16; ++n) {
    const double L = (double)s->nz / n;
    if (L > 64.0 || L < 4.0) continue;
    const double waves = tiles * n / slots;
    const double eff = waves / std::ceil(waves) * (L / (L + 3.0));
    if (eff > best_eff + 1e-12) {
      best_eff = eff;
      best = (int)std::ceil(L);
    }
  }
  return best;
}

// Source amplitude at t_n: A exp(-u^2/(2 tau^2)) sin(2 pi nu u), u = t_n - t0 (no phase), or
// the pair (A g sin(theta), A g cos(theta)) combined with cos/sin of the phase table.
void source_amp(const HostSrc& q, double t, double* a, double* b) {
  const double tau = 1.0 / (2.0 * M_PI * q.fwidth);
  const double u = t - q.t0;
  if (!q.has_phase) {
    *a = q.amp * std::exp(-u * u / (2.0 * tau * tau)) * std::sin(2.0 * M_PI * q.nu * u + 0.0);
    *b = 0.0;
  } else {
    const double g = q.amp * std::exp(-u * u / (2.0 * tau * tau));
    const double th = 2.0 * M_PI * q.nu * u;
    *a = g * std::sin(th);
    *b = g * std::cos(th);
  }
}

// Tensor maps of the plain-plane kernel (PlainMaps): the E and H blocks as 5-D tensors (x, y, z,
// component, buffer), boxes of the tile's rows, one row and the 4-cell side columns.  The encoder
// is the driver's cuTensorMapEncodeTiled, looked up through the runtime; false when unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
  }
  return fn;
}

bool encode_plain_maps(fdtdbath_sim* s, int tile_x, PlainMaps* out) {
  const EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t esz = s->esz;
  const cuuint64_t dims[5] = {(cuuint64_t)s->nx, (cuuint64_t)s->ny, (cuuint64_t)s->nz, 3, 2};
  const cuuint64_t strides[4] = {(cuuint64_t)s->nx * esz, (cuuint64_t)s->plane * esz, (cuuint64_t)s->ncell * esz,
                                 3 * (cuuint64_t)s->ncell * esz};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const cuuint32_t tx = (cuuint32_t)tile_x;
  const CUtensorMapDataType dt = s->prec == 64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  auto enc = [&](CUtensorMap* m, void* base, cuuint32_t bx, cuuint32_t by) {
    const cuuint32_t box[5] = {bx, by, 1, 3, 1};
    return fn(m, dt, 5, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  return enc(&out->e_main, s->E[0], tx, 8) && enc(&out->e_row, s->E[0], tx, 1) &&
         enc(&out->e_pad8, s->E[0], 4, 8) && enc(&out->e_pad1, s->E[0], 4, 1) &&
         enc(&out->h_main, s->H[0], tx, 8) && enc(&out->h_row, s->H[0], tx, 1) &&
         enc(&out->h_pad8, s->H[0], 4, 8);
}

// Tensor maps of the bath form's state staging (BathMaps): for each Lorentz-Bath material with
// modes (at most kBathPlainMaxMats) and each of the two state slots, P (x, y, z in the layer,
// component) and the bath modes (x, y, z in the layer, component * nb + mode), FP32, boxes of one
// kBathTileX x 8 tile of one plane.
bool encode_bath_maps(fdtdbath_sim* s, BathMaps* out) {
  const EncodeTiledFn fn = tensor_map_encoder();
  if (!fn || s->prec != 32) return false;
  *out = BathMaps{};
  for (size_t m = 0; m < s->mats.size(); ++m) {
    const HostMat& M = s->mats[m];
    if (M.kind != FDTDBATH_LORENTZ_BATH || M.nb == 0) continue;
    if (out->nmat == kBathPlainMaxMats) return false;
    const int i = out->nmat++;
    out->mat[i] = (int)m;
    const cuuint64_t nzm = (cuuint64_t)(M.zhi - M.zlo);
    const cuuint32_t es[4] = {1, 1, 1, 1};
    for (int b = 0; b < 2; ++b) {
      const cuuint64_t ydims[4] = {(cuuint64_t)s->nx, (cuuint64_t)s->ny, nzm, 3 * (cuuint64_t)M.nb};
      const cuuint64_t ystr[3] = {(cuuint64_t)s->nx * 4, (cuuint64_t)s->plane * 4, (cuuint64_t)M.ncell * 4};
      // boxes of the whole plane tile's modes, or (streamed form) of kStreamBatchModes modes
      const cuuint32_t bm_ = s->nbmax > kBathPlainRegModes ? (cuuint32_t)kStreamBatchModes : 3 * (cuuint32_t)M.nb;
      const cuuint32_t ybox[4] = {(cuuint32_t)kBathTileX, 8, 1, bm_};
      const cuuint64_t pdims[4] = {(cuuint64_t)s->nx, (cuuint64_t)s->ny, nzm, 3};
      const cuuint64_t pstr[3] = {(cuuint64_t)s->nx * 4, (cuuint64_t)s->plane * 4, (cuuint64_t)s->nmatcell * 4};
      const cuuint32_t pbox[4] = {(cuuint32_t)kBathTileX, 8, 1, 3};
      // (bf16 storage: one array of 4-byte (value, increment) pairs, the same for both slots)
      void* yb = (char*)s->Yslot[s->ybf ? 0 : b] + M.ybase * 4;
      void* pb = (char*)s->Pslot[b] + M.base * 4;
      if (fn(&out->y[i][b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, yb, ydims, ystr, ybox, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
      if (fn(&out->pp[i][b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pb, pdims, pstr, pbox, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    }
  }
  return out->nmat > 0;
}

template <typename T>
Step3DParams<T> make_params(fdtdbath_sim* s, int doH, int doE) {
  Step3DParams<T> p{};
  p.nx = (int)s->nx;
  p.ny = (int)s->ny;
  p.nz = (int)s->nz;
  p.plane = s->plane;
  p.ncell = s->ncell;
  p.dt = (T)s->dt;
  p.S = (T)(s->dt / s->dx);
  p.Ein = (const T*)s->E[s->ecur];
  p.Eout = (T*)s->E[1 - s->ecur];
  p.Hin = (const T*)s->H[s->hcur];
  p.Hout = (T*)s->H[1 - s->hcur];
  p.doH = doH;
  p.doE = doE;
  p.npml = s->npml;
  p.pmlE = (const T*)s->pmlE;
  p.pmlH = (const T*)s->pmlH;
  p.psiE = (T*)s->psiE;
  p.psiHin = (const T*)s->psiH[s->psicur];
  p.psiHout = (T*)s->psiH[1 - s->psicur];
  p.nmat = (int)s->mats.size();
  int off = 0;
  for (size_t m = 0; m < s->mats.size(); ++m) {
    p.mat[m] = mat_k<T>(s->mats[m], off, s->dt);
    off += s->mats[m].nb;
  }
  p.coef = (const T*)s->coef;
  p.nmodes = off;
  p.D = (T*)s->D;
  p.nmatcell = s->nmatcell;
  p.sig = s->sigmap ? (const T*)s->sig : nullptr;
  p.Pa = (T*)s->Pslot[s->pcur];
  p.Pb = (T*)s->Pslot[1 - s->pcur];
  p.Ya = (T*)s->Yslot[s->ybf ? 0 : s->pcur];
  p.Yb = (T*)s->Yslot[s->ybf ? 0 : 1 - s->pcur];   // bf16 pairs: one array
  p.nsrc = (int)s->srcs.size();
  const double t = (double)s->n * s->dt;
  for (size_t q = 0; q < s->srcs.size(); ++q) {
    double a, b;
    source_amp(s->srcs[q], t, &a, &b);
    p.src_comp[q] = s->srcs[q].comp;
    p.src_z[q] = (int)s->srcs[q].z;
    p.src_a[q] = (T)a;
    p.src_b[q] = (T)b;
    p.src_cos[q] = (const T*)s->srcs[q].dcos;
    p.src_sin[q] = (const T*)s->srcs[q].dsin;
  }
  p.nmon = s->quiet ? 0 : (int)s->mons.size();
  for (size_t m = 0; m < s->mons.size(); ++m) p.mon_z[m] = (int)s->mons[m].z;
  double* part = (double*)s->partial;
  const int64_t eslot = s->n % s->ring_cap;
  const int64_t hslot = (s->n - 1 + s->ring_cap) % s->ring_cap;
  p.mon_partial_E = doE ? part + eslot * s->ring_stride + s->monE_off : nullptr;
  p.mon_partial_H = doH ? part + hslot * s->ring_stride + s->monH_off : nullptr;
  p.eE_on = (!s->quiet && doE && s->energy_on && (s->n % s->e_every) == 0) ? 1 : 0;
  p.eH_on = (!s->quiet && doH && s->energy_on && ((s->n - 1) % s->e_every) == 0) ? 1 : 0;
  p.ebox_lo = (int)s->e_lo;
  p.ebox_hi = (int)s->e_hi;
  p.en_partial_E = part + eslot * s->ring_stride + s->enE_off;
  p.en_partial_H = part + hslot * s->ring_stride + s->enH_off;
  p.ew = s->dx / (double)s->plane;
  p.zstart = (const int*)s->zstart;
  p.chunk_ids = (const int*)s->chunk_ids;
  p.nchunks_total = s->nchunks;
  p.nbxy = s->nbx * s->nby;
  p.vec16 = (s->nx % (int64_t)(16 / sizeof(T)) == 0) ? 1 : 0;
  p.err = (int*)s->errflag;
  return p;
}

int launch_typed(const Step3DParams<float>& p, int nbmax, int ty, int nbx, int nby, int n, bool ybf,
                 bool te, cudaStream_t st) {
  return launch_step3d_f32(p, nbmax, ty, nbx, nby, n, ybf ? 1 : 0, te ? 1 : 0, st);
}
int launch_typed(const Step3DParams<double>& p, int nbmax, int ty, int nbx, int nby, int n, bool,
                 bool te, cudaStream_t st) {
  return launch_step3d_f64(p, nbmax, ty, nbx, nby, n, te ? 1 : 0, st);
}

template <typename T>
int launch_chunks(fdtdbath_sim* s, Step3DParams<T> p, int nbmax, int id_off, int n, cudaStream_t st) {
  p.chunk_ids = (const int*)s->chunk_ids + id_off;
  s->launches++;
  return launch_typed(p, nbmax, s->ty, s->nbx, s->nby, n, s->ybf, s->te && s->ty == 1, st);
}

int launch_plain_typed(const Step3DParams<float>& p, const fdtdbath_sim* s, int n, cudaStream_t st) {
  return launch_plain3d_f32(p, s->maps, s->ecur, s->hcur, n, st);
}
int launch_plain_typed(const Step3DParams<double>& p, const fdtdbath_sim* s, int n, cudaStream_t st) {
  return launch_plain3d_f64(p, s->maps, s->ecur, s->hcur, n, st);
}

int launch_bath_typed(const Step3DParams<float>& p, const fdtdbath_sim* s, int n, cudaStream_t st) {
  return launch_bath3d_f32(p, s->bmaps, s->bath_maps, s->pcur, s->ecur, s->hcur, n, s->nbmax, s->ybf ? 1 : 0, st);
}
int launch_bath_typed(const Step3DParams<double>&, const fdtdbath_sim*, int, cudaStream_t) {
  return (int)cudaErrorInvalidValue;   // FP64 runs the general kernel (bath_plain is never set)
}

int launch_te2d_typed(const Step3DParams<float>& p, int n, int nb, cudaStream_t st) {
  return launch_te2d_f32(p, n, nb, st);
}
int launch_te2d_typed(const Step3DParams<double>&, int, int, cudaStream_t) {
  return (int)cudaErrorInvalidValue;   // FP64 runs the general kernel (te2d_ok is never set)
}
int launch_te2d_fused_typed(const Step3DParams<float>& p, int nplain, int nbath, int nb, cudaStream_t st) {
  return launch_te2d_fused_f32(p, nplain, nbath, nb, st);
}
int launch_te2d_fused_typed(const Step3DParams<double>&, int, int, int, cudaStream_t) {
  return (int)cudaErrorInvalidValue;
}

// Chunks with bath planes: the plain-plane kernel's bath form when it applies (both half-steps of
// a step), otherwise the general kernel with the simulation's bath-mode bound.
template <typename T>
int launch_bath_chunks(fdtdbath_sim* s, Step3DParams<T> p, int id_off, int n, cudaStream_t st) {
  if (s->te2d_ok && s->te && s->ty == 1 && !s->ybf && s->nbmax <= kTe2dMaxModes && p.doH && p.doE) {
    p.chunk_ids = (const int*)s->chunk_ids + id_off;
    s->launches++;
    return launch_te2d_typed(p, n, s->nbmax, st);
  }
  if (!(s->bath_plain && p.doH && p.doE)) return launch_chunks<T>(s, p, s->nbmax, id_off, n, st);
  p.chunk_ids = (const int*)s->chunk_ids + id_off;
  s->launches++;
  return launch_bath_typed(p, s, n, st);
}

// Chunks without bath planes: the plain-plane kernel when it applies (both half-steps of a step),
// otherwise the general kernel's bath-free instantiation.

template <typename T>
int launch_plain_chunks(fdtdbath_sim* s, Step3DParams<T> p, int id_off, int n, cudaStream_t st) {
  if (s->te2d_ok && s->te && s->ty == 1 && p.doH && p.doE) {
    // the TE form's register-streaming kernel (te2d.cuh)
    p.chunk_ids = (const int*)s->chunk_ids + id_off;
    s->launches++;
    return launch_te2d_typed(p, n, 0, st);
  }
  if (!(s->plain_ok && p.doH && p.doE)) return launch_chunks<T>(s, p, 0, id_off, n, st);
  p.chunk_ids = (const int*)s->chunk_ids + id_off;
  s->launches++;
  return launch_plain_typed(p, s, n, st);
}

// One step's launches: without a pending E half-step, or without bath chunks, one launch over
// all chunks (the bath-free kernel when no bath update runs); otherwise the bath-free kernel
// over the plain chunks on the side stream, concurrently with the bath kernel over the bath
// chunks on the simulation's stream, joined before anything that follows.
template <typename T>
int launch_all(fdtdbath_sim* s, int doH, int doE) {
  Step3DParams<T> p = make_params<T>(s, doH, doE);
  if (!doE) return launch_chunks<T>(s, p, 0, 0, s->nchunks, s->stream);
  if (s->nbmax == 0) return launch_plain_chunks<T>(s, p, 0, s->nchunks, s->stream);
  if (sizeof(T) == 4 && s->te2d_ok && s->te && s->ty == 1 && !s->ybf && s->nbmax <= kTe2dMaxModes &&
      s->nplain > 0 && s->nbath > 0 && doH) {
    // the TE form: both kinds of chunks in one launch of its register-streaming kernel
    p.chunk_ids = (const int*)s->chunk_ids + s->nchunks;
    s->launches++;
    return launch_te2d_fused_typed(p, s->nplain, s->nbath, s->nbmax, s->stream);
  }
  if (s->nbath == 0) return launch_chunks<T>(s, p, s->nbmax, 0, s->nchunks, s->stream);
  if (s->nplain == 0) return launch_bath_chunks<T>(s, p, s->nchunks, s->nbath, s->stream);
  if (s->serial_pair) {
    const int rc = launch_plain_chunks<T>(s, p, s->nchunks, s->nplain, s->stream);
    return rc ? rc : launch_bath_chunks<T>(s, p, s->nchunks + s->nplain, s->nbath, s->stream);
  }
  cudaError_t e = cudaEventRecord(s->ev_fork, s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->ev_fork, 0);
  if (e != cudaSuccess) return (int)e;
  int rc = launch_plain_chunks<T>(s, p, s->nchunks, s->nplain, s->side);
  if (rc) return rc;
  rc = launch_bath_chunks<T>(s, p, s->nchunks + s->nplain, s->nbath, s->stream);
  if (rc) return rc;
  e = cudaEventRecord(s->ev_join, s->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_join, 0);
  return (int)e;
}

template <typename T>
Cav1DParams<T> make_params1d(fdtdbath_sim* s, int64_t nsteps) {
  Cav1DParams<T> p{};
  p.nz = (int)s->nz;
  p.npml = s->npml;
  for (int r = 0; r <= s->c1d; ++r) p.bounds[r] = s->bounds1d[(size_t)r];
  p.S = (T)(s->dt / s->dx);
  p.dt = (T)s->dt;
  p.E = (T*)s->E[s->ecur];
  p.H = (T*)s->H[s->hcur];
  p.D = (T*)s->D;
  p.Pslot[0] = (T*)s->Pslot[0];
  p.Pslot[1] = (T*)s->Pslot[1];
  p.Yslot[0] = (T*)s->Yslot[0];
  p.Yslot[1] = (T*)s->Yslot[1];
  p.pcur0 = s->pcur;
  p.sig = s->sigmap ? (const T*)s->sig : nullptr;
  p.coef = (const T*)s->coef;
  p.nmat = (int)s->mats.size();
  int off = 0;
  for (size_t m = 0; m < s->mats.size(); ++m) {
    p.mat[m] = mat_k<T>(s->mats[m], off, s->dt);
    off += s->mats[m].nb;
  }
  p.pmlE = (const T*)s->pmlE;
  p.pmlH = (const T*)s->pmlH;
  p.psiE = (T*)s->psiE;
  p.psiH = (T*)s->psiH[s->psicur];
  p.psiH_stride = 2 * s->npml + 1;
  p.nsrc = (int)s->srcs.size();
  p.src_z = p.nsrc ? (int)s->srcs[0].z : -1;
  p.src_tab = (const double*)s->src_tab;
  p.nmon = (int)s->mons.size();
  p.mon_z = p.nmon ? (int)s->mons[0].z : -1;
  p.energy_on = s->energy_on ? 1 : 0;
  p.every = s->e_every;
  p.ebox_lo = (int)s->e_lo;
  p.ebox_hi = (int)s->e_hi;
  p.partial = (double*)s->partial;
  p.ring_cap = s->ring_cap;
  p.ring_stride = s->ring_stride;
  p.monE_off = s->monE_off;
  p.monH_off = s->monH_off;
  p.enE_off = s->enE_off;
  p.enH_off = s->enH_off;
  p.step0 = s->n;
  p.nsteps = (int)nsteps;
  return p;
}

// Cell ranges of the cluster's CTAs: contiguous, at most kCav1DThreads cells each, balanced by
// work (vacuum 1, CPML 2, Lorentz / Drude 3, Lorentz-Bath 3 + N_b per cell).
std::vector<int> balance_cells(const fdtdbath_sim* s, int C) {
  std::vector<double> w((size_t)s->nz, 1.0);
  for (int64_t z = 0; z < s->nz; ++z)
    if (z < s->npml || z >= s->nz - s->npml) w[(size_t)z] = 2.0;
  for (auto& m : s->mats)
    for (int64_t z = m.zlo; z < m.zhi; ++z)
      w[(size_t)z] = m.kind == FDTDBATH_VACUUM ? 1.0 : 3.0 + (m.kind == FDTDBATH_LORENTZ_BATH ? m.nb : 0);
  double total = 0.0;
  for (double v : w) total += v;
  std::vector<int> b(1, 0);
  double acc = 0.0;
  int64_t z = 0;
  for (int r = 0; r < C; ++r) {
    const double target = total * (r + 1) / C;
    const int64_t left_ctas = C - r - 1;
    int64_t end = z;
    while (end < s->nz && (end - z) < kCav1DThreads &&
           (end == z || acc + w[(size_t)end] <= target + 1e-9 || s->nz - end > left_ctas * kCav1DThreads)) {
      acc += w[(size_t)end];
      ++end;
    }
    if (r == C - 1) end = s->nz;
    b.push_back((int)end);
    z = end;
  }
  return b;
}

int launch_1d(fdtdbath_sim* s, int64_t nsteps) {
  // per-step source amplitudes, evaluated on the host exactly as for the 3D kernel
  if (!s->srcs.empty()) {
    std::vector<double> tab((size_t)nsteps);
    const HostSrc& q = s->srcs[0];
    const double tau = 1.0 / (2.0 * M_PI * q.fwidth);
    for (int64_t i = 0; i < nsteps; ++i) {
      const double t = (double)(s->n + i) * s->dt;   // host code is built without FP contraction
      const double u = t - q.t0;
      tab[(size_t)i] = q.amp * std::exp(-u * u / (2.0 * tau * tau)) * std::sin(2.0 * M_PI * q.nu * u + q.phase1d);
    }
    cudaError_t e = cudaMemcpyAsync(s->src_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "source table copy");
  }
  int rc;
  if (s->prec == 64) rc = launch_cavity1d_f64(make_params1d<double>(s, nsteps), s->nbmax, s->c1d, s->stream);
  else rc = launch_cavity1d_f32(make_params1d<float>(s, nsteps), s->nbmax, s->c1d, s->stream);
  s->launches++;
  if (rc) return cuda_fail(s, (cudaError_t)rc, "1D cavity kernel launch");
  return 0;
}

int launch_tb2_any(const Tb2Params<float>& q, int n, cudaStream_t st) { return launch_tb2_f32(q, n, st); }
int launch_tb2_any(const Tb2Params<double>& q, int n, cudaStream_t st) { return launch_tb2_f64(q, n, st); }

// Steps n and n+1 in one launch of the two-steps-per-pass kernel (the pending H half-step of step
// n included): step n's parameters as for a single step, then step n+1's sources and partial rows.
template <typename T>
int launch_tb2_typed(fdtdbath_sim* s) {
  Tb2Params<T> q{};
  q.p = make_params<T>(s, 1, 1);
  q.psiEout = (T*)s->psiE_alt;
  const int64_t n1 = s->n + 1;
  const double t1 = (double)n1 * s->dt;
  for (size_t k = 0; k < s->srcs.size(); ++k) {
    double a, b;
    source_amp(s->srcs[k], t1, &a, &b);
    q.src_a2[k] = (T)a;
    q.src_b2[k] = (T)b;
  }
  double* part = (double*)s->partial;
  const int64_t eslot = n1 % s->ring_cap, hslot = s->n % s->ring_cap;
  q.mon_partial_E2 = part + eslot * s->ring_stride + s->monE_off;
  q.mon_partial_H2 = part + hslot * s->ring_stride + s->monH_off;
  q.en_partial_E2 = part + eslot * s->ring_stride + s->enE_off;
  q.en_partial_H2 = part + hslot * s->ring_stride + s->enH_off;
  q.eE_on2 = (!s->quiet && s->energy_on && (n1 % s->e_every) == 0) ? 1 : 0;
  q.eH_on2 = (!s->quiet && s->energy_on && (s->n % s->e_every) == 0) ? 1 : 0;
  s->launches++;
  return launch_tb2_any(q, s->nchunks, s->stream);
}

int launch_pair(fdtdbath_sim* s) {
  const int rc = s->prec == 64 ? launch_tb2_typed<double>(s) : launch_tb2_typed<float>(s);
  if (rc) return cuda_fail(s, (cudaError_t)rc, "two-step kernel launch");
  s->ecur = 1 - s->ecur;
  s->hcur = 1 - s->hcur;
  s->psicur = 1 - s->psicur;
  std::swap(s->psiE, s->psiE_alt);
  return 0;
}

int launch_step(fdtdbath_sim* s, int doH, int doE) {
  const int rc = s->prec == 64 ? launch_all<double>(s, doH, doE) : launch_all<float>(s, doH, doE);
  if (rc) return cuda_fail(s, (cudaError_t)rc, "step kernel launch");
  if (doE) s->ecur = 1 - s->ecur;
  if (doH) {
    s->hcur = 1 - s->hcur;
    s->psicur = 1 - s->psicur;
  }
  return 0;
}

// Fold the partial sums of complete steps [reduced, upto) into the DFT accumulators / trace.
int reduce_upto(fdtdbath_sim* s, int64_t upto) {
  if (upto <= s->reduced) return 0;
  if ((s->mons.empty() && !s->energy_on) || s->quiet) {
    s->reduced = upto;
    return 0;
  }
  const int nbxy = s->red_nbxy, nblocks = s->red_nblocks;
  ReduceParams r{};
  r.partial = (const double*)s->partial;
  r.ring_stride = s->ring_stride;
  r.ring_cap = s->ring_cap;
  r.nmon = (int)s->mons.size();
  r.nbxy = nbxy;
  r.nblocks = nblocks;
  r.mon_E_off = s->monE_off;
  r.mon_H_off = s->monH_off;
  r.en_E_off = s->enE_off;
  r.en_H_off = s->enH_off;
  r.energy_on = s->energy_on ? 1 : 0;
  r.step_lo = s->reduced;
  r.step_hi = upto;
  r.every = s->e_every;
  r.series = (double*)s->series;
  int rc = launch_reduce_series(r, s->stream);
  s->launches++;
  if (rc) return cuda_fail(s, (cudaError_t)rc, "reduce kernel launch");
  DftParams d{};
  d.series = (const double*)s->series;
  d.ring_cap = s->ring_cap;
  d.series_stride = 6 * (int)s->mons.size() + 4;
  d.nmon = (int)s->mons.size();
  d.step_lo = s->reduced;
  d.step_hi = upto;
  d.dt = s->dt;
  for (size_t m = 0; m < s->mons.size(); ++m) {
    d.freqs[m] = (const double*)s->mons[m].dfreq;
    d.nfreq[m] = s->mons[m].nfreq;
    d.acc[m] = (double*)s->mons[m].dacc;
  }
  d.energy_on = s->energy_on ? 1 : 0;
  d.every = s->e_every;
  d.trace = (double*)s->trace;
  d.trace_cap = s->e_cap;
  d.inv_plane = 1.0 / (double)s->plane;
  d.ew = s->dx / (double)s->plane;
  rc = launch_dft_accumulate(d, s->stream);
  s->launches++;
  if (rc) return cuda_fail(s, (cudaError_t)rc, "dft kernel launch");
  s->reduced = upto;
  return 0;
}

int flush_h(fdtdbath_sim* s) {
  if (!s->h_pending) return 0;
  int rc = launch_step(s, 1, 0);
  if (rc) return rc;
  s->h_pending = false;
  return 0;
}

int flush_all(fdtdbath_sim* s) {
  int rc = flush_h(s);
  if (rc) return rc;
  return reduce_upto(s, s->n);
}

// A 1D simulation leaves the persistent 1D kernel for the 3D one (for good): the partials the
// 1D kernel left are reduced in its layout first, later ones use the 3D kernel's block count.
int switch_to_3d(fdtdbath_sim* s) {
  if (!(s->path1d && s->ncomp1d == 1)) return 0;
  int rc = reduce_upto(s, s->n);
  if (rc) return rc;
  s->ncomp1d = 3;
  s->red_nblocks = s->nblk3d;
  return 0;
}

// ---- field access ------------------------------------------------------------------
struct FieldRef {
  int kind;  // 0 full grid, 1 material P / PM, 2 bath mode, 3 sigma(r)
  int comp, mode, level;
};

bool parse_field(int32_t f, FieldRef* r) {
  if (f >= 0 && f < 6) {
    *r = {0, f, 0, 0};
    return true;
  }
  if (f >= 6 && f < 12) {
    *r = {1, (f - 6) % 3, 0, f >= 9 ? 1 : 0};
    return true;
  }
  if (f == FDTDBATH_FIELD_SIGMA) {
    *r = {3, 0, 0, 0};
    return true;
  }
  if (f >= 1024 && f < 1024 + 6 * 256) {
    const int q = f - 1024;
    const int cl = q / 256;
    *r = {2, cl / 2, q % 256, cl % 2};
    return r->mode < kMaxBathStep;
  }
  return false;
}

// Host copies of canonical state pieces as double.
int fetch(fdtdbath_sim* s, const void* dptr, int64_t count, std::vector<double>& out) {
  out.assign((size_t)count, 0.0);
  if (s->prec == 64) return d2h(s, out.data(), dptr, (size_t)count * 8);
  std::vector<float> tmp((size_t)count);
  int rc = d2h(s, tmp.data(), dptr, (size_t)count * 4);
  for (int64_t i = 0; i < count; ++i) out[(size_t)i] = tmp[(size_t)i];
  return rc;
}

int store(fdtdbath_sim* s, void* dptr, const std::vector<double>& in) {
  if (s->prec == 64) return h2d(s, dptr, in.data(), in.size() * 8);
  std::vector<float> tmp(in.size());
  for (size_t i = 0; i < in.size(); ++i) tmp[i] = (float)in[i];
  return h2d(s, dptr, tmp.data(), tmp.size() * 4);
}

char* elem_ptr(void* base, int64_t idx, size_t esz) { return (char*)base + idx * (int64_t)esz; }

// ---- per-cell oscillator strength sigma(r) (Eq. EOM_Lorentz / EOM_LorentzBath-1) ------------
// The full-grid sigma(r): the map where one is set, else every dispersive layer's own sigma; zero
// outside the dispersive layers.
int sigma_full(fdtdbath_sim* s, std::vector<double>& full) {
  full.assign((size_t)s->ncell, 0.0);
  for (auto& m : s->mats) {
    if (m.kind == FDTDBATH_VACUUM) continue;
    double* o = full.data() + m.zlo * s->plane;
    if (!s->sigmap) {
      std::fill(o, o + m.ncell, m.sigma);
      continue;
    }
    std::vector<double> a;
    const int rc = fetch(s, elem_ptr(s->sig, m.base, s->esz), m.ncell, a);
    if (rc) return rc;
    std::copy(a.begin(), a.end(), o);
  }
  return 0;
}

// The TE form's register-streaming kernel reads each layer's own sigma only: while a map is set
// its chunks go to the general kernel; without one the choice made at creation returns.  (The
// general, plain-plane and 1D kernels read the map.)
void sigma_mode(fdtdbath_sim* s, bool on) {
  s->sigmap = on;
  s->te2d_ok = on ? false : s->te2d_ok0;
}

// Validate a full-grid sigma(r) (finite, >= 0 in the dispersive layers, each layer stable at its
// largest value; values elsewhere ignored) and make it the simulation's map.
int set_sigma_map(fdtdbath_sim* s, const std::vector<double>& full) {
  const int dims = (s->nx > 1) + (s->ny > 1) + (s->nz > 1);
  for (auto& m : s->mats) {
    if (m.kind == FDTDBATH_VACUUM) continue;
    const double* v = full.data() + m.zlo * s->plane;
    double mx = 0.0;
    for (int64_t r = 0; r < m.ncell; ++r) {
      if (!(v[r] >= 0.0) || !std::isfinite(v[r]))
        return fail(s, FDTDBATH_ERR_ARG, "sigma(r) must be finite and non-negative");
      mx = std::max(mx, v[r]);
    }
    if (!oscillator_stable(m, mx, s->dt, s->courant, dims))
      return fail(s, FDTDBATH_ERR_CFL, "field-oscillator update unstable at the largest sigma(r) of a layer");
  }
  if (!s->sig) {
    s->sig = dalloc(s, (size_t)s->nmatcell * s->esz);
    if (!s->sig) return fail(s, FDTDBATH_ERR_OOM, "device allocation failed");
  }
  for (auto& m : s->mats) {
    std::vector<double> v((size_t)m.ncell, 0.0);
    if (m.kind != FDTDBATH_VACUUM) {
      const double* src = full.data() + m.zlo * s->plane;
      std::copy(src, src + m.ncell, v.begin());
    }
    const int rc = store(s, elem_ptr(s->sig, m.base, s->esz), v);
    if (rc) return rc;
  }
  sigma_mode(s, true);
  return 0;
}

// bf16 <-> float on the host (round to nearest even; no NaN payloads are produced by the kernels)
float bf16_to_float(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
uint16_t float_to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Both levels of one bf16-stored bath mode block of `count` cells: Y^{n+1/2} = value,
// Y^{n-1/2} = value - increment (FP32 arithmetic, as the kernel forms them).
int fetch_bf16_levels(fdtdbath_sim* s, int64_t off, int64_t count, std::vector<float>& y0, std::vector<float>& y1) {
  std::vector<uint16_t> ab(2 * (size_t)count);   // (value, increment) per cell
  int rc = d2h(s, ab.data(), elem_ptr(s->Yslot[0], off, 4), (size_t)count * 4);
  if (rc) return rc;
  y0.resize((size_t)count);
  y1.resize((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    y0[(size_t)i] = bf16_to_float(ab[2 * (size_t)i]);
    y1[(size_t)i] = y0[(size_t)i] - bf16_to_float(ab[2 * (size_t)i + 1]);
  }
  return 0;
}

int store_bf16_levels(fdtdbath_sim* s, int64_t off, const std::vector<float>& y0, const std::vector<float>& y1) {
  std::vector<uint16_t> ab(2 * y0.size());
  for (size_t i = 0; i < y0.size(); ++i) {
    ab[2 * i] = float_to_bf16(y0[i]);
    ab[2 * i + 1] = float_to_bf16(y0[i] - y1[i]);
  }
  return h2d(s, elem_ptr(s->Yslot[0], off, 4), ab.data(), ab.size() * 2);
}

// FDTDBATH_ERR_NONFINITE when any of the n values copied out is a NaN or an Inf.
int check_finite(fdtdbath_sim* s, const double* v, size_t n, const char* what) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i]))
      return fail(s, FDTDBATH_ERR_NONFINITE,
                  std::string(what) + " holds NaN or Inf: the state diverged or was given non-finite values");
  return FDTDBATH_OK;
}

// FDTDBATH_ERR_TIMEOUT when a kernel's bounded wait for staged data ran out since the simulation
// was created (its results are then not valid).  Call after the stream has been synchronized.
int check_timeout(fdtdbath_sim* s) {
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, s->errflag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(s, e, "error flag");
  if (flag)
    return fail(s, FDTDBATH_ERR_TIMEOUT,
                "a step kernel's bounded wait for its staged planes ran out (the results are not valid)");
  return FDTDBATH_OK;
}

}  // namespace

int fdtdbath_internal_view(fdtdbath_sim* s, SimView* v) {
  if (!s || !v) return FDTDBATH_ERR_ARG;
  cudaSetDevice(s->device);
  int rc = flush_h(s);
  if (rc) return rc;
  *v = SimView{};
  v->prec = s->prec;
  v->inc = 0;
  v->nx = s->nx;
  v->ny = s->ny;
  v->nz = s->nz;
  v->plane = s->plane;
  v->ncell = s->ncell;
  v->nmatcell = s->nmatcell;
  v->dx = s->dx;
  v->dt = s->dt;
  v->E = s->E[s->ecur];
  v->H = s->H[s->hcur];
  v->Pa = s->Pslot[s->pcur];
  v->Pb = s->Pslot[1 - s->pcur];
  if (s->ybf) return fail(s, FDTDBATH_ERR_UNSUPPORTED, "this entry point does not read bf16 bath storage");
  if (s->sigmap) return fail(s, FDTDBATH_ERR_UNSUPPORTED, "this entry point uses each layer's own sigma, not a sigma(r) map");
  v->Ya = s->Yslot[s->pcur];
  v->Yb = s->Yslot[1 - s->pcur];
  v->nmat = (int)s->mats.size();
  for (size_t m = 0; m < s->mats.size(); ++m) {
    const HostMat& h = s->mats[m];
    SimViewMat& o = v->mat[m];
    o.kind = h.kind;
    o.nb = h.nb;
    o.zlo = h.zlo;
    o.zhi = h.zhi;
    o.ncell = h.ncell;
    o.base = h.base;
    o.ybase = h.ybase;
    o.eps = h.eps;
    o.rho = h.rho;
    o.w0r2 = h.w0r2;
    for (int j = 0; j < h.nb; ++j) o.wj2[j] = h.wj[j] * h.wj[j];
  }
  v->stream = s->stream;
  v->device = s->device;
  return 0;
}

int fdtdbath_internal_fail(fdtdbath_sim* s, int code, const char* msg) { return fail(s, code, msg); }

// ======================================================================================
extern "C" {

int fdtdbath_create(const fdtdbath_grid* grid, double resolution, double courant,
                    const fdtdbath_material* materials, int32_t nmat,
                    const fdtdbath_source* sources, int32_t nsrc,
                    const fdtdbath_monitor* monitors, int32_t nmon,
                    const fdtdbath_options* opt, fdtdbath_sim** out) {
  if (!out) return fail(nullptr, FDTDBATH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !opt) return fail(nullptr, FDTDBATH_ERR_ARG, "grid/options is NULL");
  if (grid->n[0] < 1 || grid->n[1] < 1 || grid->n[2] < 4)
    return fail(nullptr, FDTDBATH_ERR_ARG, "grid needs nx, ny >= 1 and nz >= 4");
  if (grid->n[0] > (1 << 20) || grid->n[1] > (1 << 20) || grid->n[2] > (1 << 20))
    return fail(nullptr, FDTDBATH_ERR_ARG, "grid dimension too large");
  if (!(resolution > 0) || !(courant > 0))
    return fail(nullptr, FDTDBATH_ERR_ARG, "resolution and courant must be positive");
  if (opt->precision != 32 && opt->precision != 64)
    return fail(nullptr, FDTDBATH_ERR_ARG, "precision must be 32 or 64");
  if (opt->bath_storage != 0 && opt->bath_storage != 1) return fail(nullptr, FDTDBATH_ERR_ARG, "bath_storage must be 0 or 1");
  if (opt->bath_storage == 1 && opt->precision != 32)
    return fail(nullptr, FDTDBATH_ERR_ARG, "bf16 bath storage needs precision 32");
  if (nmat < 0 || nmat > kMaxMat || (nmat && !materials))
    return fail(nullptr, FDTDBATH_ERR_ARG, "0 <= nmat <= 8");
  if (nsrc < 0 || nsrc > kMaxSrc || (nsrc && !sources))
    return fail(nullptr, FDTDBATH_ERR_ARG, "0 <= nsrc <= 4");
  if (nmon < 0 || nmon > kMaxMon || (nmon && !monitors))
    return fail(nullptr, FDTDBATH_ERR_ARG, "0 <= nmon <= 4");
  const int64_t nx = grid->n[0], ny = grid->n[1], nz = grid->n[2];
  if (grid->pml_cells < 0 || 2 * (int64_t)grid->pml_cells + 2 > nz)
    return fail(nullptr, FDTDBATH_ERR_ARG, "pml_cells out of range");
  int dims = (nx > 1) + (ny > 1) + (nz > 1);
  if (courant > 1.0 / std::sqrt((double)dims) + 1e-12)
    return fail(nullptr, FDTDBATH_ERR_CFL, "Courant number above 1/sqrt(dims)");

  fdtdbath_sim* s = new fdtdbath_sim();
  s->prec = opt->precision;
  s->esz = s->prec == 64 ? 8 : 4;
  s->ybf = opt->bath_storage == 1;
  s->yesz = s->ybf ? 2 : s->esz;
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->plane = nx * ny;
  s->ncell = nx * ny * nz;
  s->res = resolution;
  s->courant = courant;
  s->dx = 1.0 / resolution;
  s->dt = courant * s->dx;
  s->npml = grid->pml_cells;
  s->stream = (cudaStream_t)opt->cuda_stream;
  s->device = opt->device;
  s->ualloc = opt->alloc;
  s->ufree = opt->free;
  s->uctx = opt->alloc_ctx;
  auto bail = [&](int code, const std::string& msg) {
    g_create_error = msg;
    fdtdbath_destroy(s);
    return code;
  };
  if ((s->ualloc == nullptr) != (s->ufree == nullptr))
    return bail(FDTDBATH_ERR_ARG, "alloc and free must both be set or both NULL");
  // ---- materials ----
  std::vector<int> order(nmat);
  for (int m = 0; m < nmat; ++m) order[m] = m;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return materials[a].z_lo < materials[b].z_lo; });
  int64_t prev_hi = 0;
  for (int oi = 0; oi < nmat; ++oi) {
    const fdtdbath_material& M = materials[order[oi]];
    if (M.z_lo < 0 || M.z_hi > nz || M.z_lo >= M.z_hi) return bail(FDTDBATH_ERR_ARG, "material z-range outside the grid");
    if (M.z_lo < prev_hi) return bail(FDTDBATH_ERR_ARG, "material layers overlap");
    prev_hi = M.z_hi;
    HostMat h{};
    std::string why;
    const int rc = build_material(M, s->plane, s->dt, courant, dims, h, why);
    if (rc) return bail(rc, why);
    h.user_index = order[oi];
    expand_material(h, s->dt);
    s->mats.push_back(h);
  }
  int64_t base = 0, ybase = 0;
  for (auto& m : s->mats) {
    m.base = base;
    base += m.ncell;
    m.ybase = ybase;
    ybase += (int64_t)3 * m.nb * m.ncell;
    s->nbmax = std::max(s->nbmax, m.nb);
  }
  s->nmatcell = base;
  s->nybath = ybase;
  // the kernels index every array with 32-bit offsets
  const int64_t lim = ((int64_t)1 << 31) - 1;
  if (3 * s->ncell > lim || 3 * s->nmatcell > lim || s->nybath > lim ||
      2 * (2 * (int64_t)s->npml + 1) * s->plane > lim)
    return bail(FDTDBATH_ERR_ARG, "state arrays above 2^31 elements are not supported");
  if (s->nbmax > 0) s->nbmax = s->nbmax <= 4 ? 4 : s->nbmax <= 8 ? 8 : s->nbmax <= 16 ? 16 : s->nbmax <= 32 ? 32 : 128;

  // ---- sources / monitors / energy box ----
  for (int q = 0; q < nsrc; ++q) {
    const fdtdbath_source& S = sources[q];
    if (S.component < 0 || S.component > 2 || S.z < 0 || S.z >= nz)
      return bail(FDTDBATH_ERR_ARG, "source component or plane out of range");
    if (!(S.fwidth > 0)) return bail(FDTDBATH_ERR_ARG, "source fwidth must be positive");
    HostSrc h{S.component, S.z, S.center, S.fwidth, S.amplitude, S.t0, S.phase != nullptr, nullptr, nullptr,
              S.phase ? S.phase[0] : 0.0};
    s->srcs.push_back(h);
  }
  for (int q = 0; q < nmon; ++q) {
    const fdtdbath_monitor& M = monitors[q];
    if (M.z < 1 || M.z >= nz || M.nfreq < 1 || !M.freqs) return bail(FDTDBATH_ERR_ARG, "monitor out of range");
    s->mons.push_back(HostMon{M.z, M.nfreq, nullptr, nullptr});
  }
  s->energy_on = opt->energy_hi > opt->energy_lo;
  if (s->energy_on) {
    if (opt->energy_lo < 0 || opt->energy_hi > nz) return bail(FDTDBATH_ERR_ARG, "energy box outside the grid");
    s->e_lo = opt->energy_lo;
    s->e_hi = opt->energy_hi;
    s->e_cap = opt->energy_capacity > 0 ? opt->energy_capacity : 65536;
    s->e_every = 1;
  }

  // ---- launch plan ----
  // tile height: 8 rows, or single-row tiles for grids with fewer than 8 rows
  s->ty = ny >= 8 ? 8 : 1;
  s->nbx = (int)((nx + kTX - 1) / kTX);
  s->nby = (int)((ny + s->ty - 1) / s->ty);
  // balanced chunks when every launch still gets at least a full wave of CTAs (4 bath-free or 2
  // bath CTAs per SM), otherwise uniform 32-plane chunks; FDTDBATH_ZCHUNK forces a uniform plan
  int zc = 32;
  bool balanced = true;
  if (const char* e = std::getenv("FDTDBATH_ZCHUNK")) {
    zc = std::min(64, std::max(1, std::atoi(e)));
    balanced = false;
  }
  // the plain-plane kernel takes the chunks without bath planes (plain3d.cuh) on grids tiled exactly
  // by its (TX x 8) tiles whose source planes lie outside the layers, when the tensor maps can be
  // encoded (FDTDBATH_PLAIN=0 keeps the general kernel); those ranges are then cut into near-equal
  // chunks of about plain_zc planes (FDTDBATH_PLAIN_ZCHUNK, at most 64)
  // Its bath form (FP32; at most 16 modes per material held in registers, with FP32 or bf16 bath
  // storage, or up to 128 streamed, with FP32 storage; at most two Lorentz-Bath materials; 32 x 8
  // tiles) takes the Lorentz-Bath ranges, cut into near-equal
  // chunks of about bath_zc planes (FDTDBATH_BATH_ZCHUNK, at most 64; FDTDBATH_BATHPLAIN=0 keeps
  // the general kernel there).  One chunk per layer of up to 64 planes measured fastest on the
  // 256^3 slab: each chunk start pays the prologue and the first stages' latency.
  {
    bool src_in_layer = false;
    for (auto& q : s->srcs)
      for (auto& m : s->mats)
        if (q.z >= m.zlo && q.z < m.zhi) src_in_layer = true;
    const int tx = plain_tile_x(s->prec);
    const char* e = std::getenv("FDTDBATH_PLAIN");
    s->plain_ok = !(e && std::atoi(e) == 0) && s->ty == 8 && nx % tx == 0 && ny % 8 == 0 && !src_in_layer;
    const char* et = std::getenv("FDTDBATH_TE2D");
    s->te2d_ok = !(et && std::atoi(et) == 0) && s->prec == 32 && ny == 1 && nx % kTe2dTileX == 0 && !src_in_layer;
    const char* eb = std::getenv("FDTDBATH_BATHPLAIN");
    int nmodes_all = 0;
    for (auto& m : s->mats) nmodes_all += m.nb;
    s->bath_plain = !(eb && std::atoi(eb) == 0) && s->prec == 32 && s->nbmax > 0 &&
                    s->nbmax <= kBathPlainMaxModes && s->ty == 8 && nx % kBathTileX == 0 && ny % 8 == 0 &&
                    !src_in_layer &&
                    // the streamed form (more than 16 modes): FP32 bath storage, its coefficient table
                    (s->nbmax <= kBathPlainRegModes || (!s->ybf && nmodes_all <= kStreamCoefRows));
  }
  // two steps per pass (FDTDBATH_TB=1): grids without polarizable material, at least 8 rows, tiled
  // exactly by its 32 x 8 tiles; its ghost planes favour longer chunks.  Off by default: it halves
  // the DRAM traffic but issues more instructions per cell than two single steps take time for.
  {
    const char* e = std::getenv("FDTDBATH_TB");
    s->tb_ok = e && std::atoi(e) == 1 && s->mats.empty() && s->ty == 8 && nx % kTbTX == 0 && ny % kTbTY == 0;
  }
  int plain_zc = 0, bath_zc = 0, bath_nmin = 1;
  if (s->plain_ok) {
    plain_zc = s->tb_ok ? tb_chunk_planes(s) : 16;
    if (const char* e = std::getenv("FDTDBATH_PLAIN_ZCHUNK")) plain_zc = std::min(64, std::max(1, std::atoi(e)));
  }
  if (s->bath_plain) {
    // chunks of at most 64 planes, and enough of them for a CTA on every SM
    bath_zc = 64;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess && sms > 0) {
      const int64_t tiles = (nx / kBathTileX) * (ny / 8);
      bath_nmin = (int)((sms + tiles - 1) / tiles);
    }
    if (const char* e = std::getenv("FDTDBATH_BATH_ZCHUNK")) {
      bath_zc = std::min(64, std::max(1, std::atoi(e)));
      bath_nmin = 1;
    }
  }
  std::vector<int> starts;
  if (balanced) {
    int sms = 0;
    balanced = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess && sms > 0;
    if (balanced) {
      const int n = plan_chunks(s, zc, true, plain_zc, bath_zc, bath_nmin, starts);
      int64_t nplain = 0, nbath = 0;
      for (int c = 0; c < n; ++c) {
        if (starts[c + 1] - starts[c] > 128) balanced = false;
        (chunk_has_bath(s, starts[c], starts[c + 1]) ? nbath : nplain) += 1;
      }
      const int64_t tiles = (int64_t)s->nbx * s->nby;
      if ((!s->plain_ok && nplain > 0 && nplain * tiles < 4LL * sms) || (nbath > 0 && nbath * tiles < 2LL * sms))
        balanced = false;
    }
  }
  // uniform plan on grids with few tiles per plane (the 2D cavities: one row of 32-wide tiles, or
  // 128-wide tiles in the TE form): 16-plane chunks, so that each launch still has CTAs for
  // every SM
  if (!balanced && !std::getenv("FDTDBATH_ZCHUNK")) {
    const bool te0 = s->ty == 1 && ny == 1 && std::all_of(s->srcs.begin(), s->srcs.end(),
                                                             [](const HostSrc& q) { return q.comp == 1; });
    const int64_t ktiles = te0 ? (nx + 4 * kTX - 1) / (4 * kTX) : (int64_t)s->nbx * s->nby;
    if (ktiles < 64) zc = 16;
  }
  s->nchunks = plan_chunks(s, zc, balanced, plain_zc, bath_zc, bath_nmin, starts);
  for (int c = 0; c < s->nchunks; ++c)   // the plain-plane kernel takes chunks of at most 64 planes
    if (starts[c + 1] - starts[c] > 64) (chunk_has_bath(s, starts[c], starts[c + 1]) ? s->bath_plain : s->plain_ok) = false;
  for (size_t c = 0; c + 1 < starts.size(); ++c)
    if (starts[c + 1] - starts[c] > 128) return bail(FDTDBATH_ERR_ARG, "z-chunk longer than 128 planes");
  if ((int64_t)s->nbx * s->nby > 65535 * 64) return bail(FDTDBATH_ERR_ARG, "grid too large for the launch plan");

  cudaError_t ce = cudaSetDevice(s->device);
  if (ce != cudaSuccess) return bail(FDTDBATH_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(ce));

  // ---- device state ----
  const size_t esz = s->esz;
  // E and H: one allocation of two buffers each (the tensor maps of the plain-plane kernel span both)
  s->E[0] = dalloc(s, 2 * 3 * s->ncell * esz);
  s->H[0] = dalloc(s, 2 * 3 * s->ncell * esz);
  if (!s->E[0] || !s->H[0]) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  s->E[1] = (char*)s->E[0] + 3 * s->ncell * esz;
  s->H[1] = (char*)s->H[0] + 3 * s->ncell * esz;
  for (int b = 0; b < 2; ++b) {
    s->psiH[b] = dalloc(s, 2 * (size_t)(2 * s->npml + 1) * s->plane * esz);
    s->Pslot[b] = dalloc(s, 3 * (size_t)s->nmatcell * esz);
    s->Yslot[b] = dalloc(s, s->ybf ? (b == 0 ? (size_t)s->nybath * 4 : 16) : (size_t)s->nybath * s->yesz);
    if (!s->psiH[b] || !s->Pslot[b] || !s->Yslot[b])
      return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  }
  // no tensor-map encoder: the general kernel
  if (s->plain_ok && !encode_plain_maps(s, plain_tile_x(s->prec), &s->maps)) s->plain_ok = false;
  if (s->bath_plain && !(encode_plain_maps(s, kBathTileX, &s->bmaps) && encode_bath_maps(s, &s->bath_maps)))
    s->bath_plain = false;
  // the plain-plane kernel beside the general kernel's bath form: one after the other; beside its
  // own bath form: concurrently (the two kinds of CTAs fit on one SM together)
  s->serial_pair = s->plain_ok && !s->bath_plain;
  s->psiE = dalloc(s, 2 * (size_t)(2 * s->npml) * s->plane * esz);
  if (s->tb_ok) {
    s->psiE_alt = dalloc(s, 2 * (size_t)(2 * s->npml) * s->plane * esz);
    if (!s->psiE_alt) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  }
  s->pmlE = dalloc(s, 2 * (size_t)nz * esz);
  s->pmlH = dalloc(s, 2 * (size_t)nz * esz);
  s->D = dalloc(s, s->prec == 64 ? 3 * (size_t)s->nmatcell * esz : 16);
  int nmodes = 0;
  for (auto& m : s->mats) nmodes += m.nb;
  s->coef = dalloc(s, (size_t)std::max(1, nmodes) * kCoefStride * esz);
  s->zstart = dalloc(s, starts.size() * sizeof(int));
  s->errflag = dalloc(s, 16);
  s->chunk_ids = dalloc(s, 2 * (size_t)s->nchunks * sizeof(int));
  if (!s->psiE || !s->pmlE || !s->pmlH || !s->D || !s->coef || !s->zstart || !s->chunk_ids || !s->errflag)
    return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  std::vector<int> ids;
  for (int c = 0; c < s->nchunks; ++c) ids.push_back(c);
  std::vector<int> plain, bathc;
  for (int c = 0; c < s->nchunks; ++c) (chunk_has_bath(s, starts[c], starts[c + 1]) ? bathc : plain).push_back(c);
  // each launch dispatches its longest chunks first (blocks go out in grid order, chunk-major)
  auto clen = [&](int c) { return starts[c + 1] - starts[c]; };
  std::stable_sort(plain.begin(), plain.end(), [&](int a, int b) { return clen(a) > clen(b); });
  std::stable_sort(bathc.begin(), bathc.end(), [&](int a, int b) { return clen(a) > clen(b); });
  s->nplain = (int)plain.size();
  s->nbath = (int)bathc.size();
  ids.insert(ids.end(), plain.begin(), plain.end());
  ids.insert(ids.end(), bathc.begin(), bathc.end());
  if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(FDTDBATH_ERR_CUDA, "stream/event creation failed");
  // 1D path: one cluster of up to 8 CTAs of 256 threads
  s->te = ny == 1;
  for (auto& q : s->srcs)
    if (q.comp != 1) s->te = false;
  s->path1d = (nx == 1 && ny == 1 && nsrc <= 1 && nmon <= 1 && !s->ybf && s->nbmax <= kMaxBath &&
                nz <= (int64_t)kCav1DMaxCluster * kCav1DThreads);
  if (s->path1d) {
    // FP64 bath arithmetic is slow on this part: spread the cavity over the largest cluster
    int want = s->prec == 64 ? kCav1DMaxCluster : 8;
    if (const char* e = std::getenv("FDTDBATH_C1D")) want = std::max(1, std::min(kCav1DMaxCluster, std::atoi(e)));
    s->c1d = (int)std::max<int64_t>(want, (nz + kCav1DThreads - 1) / kCav1DThreads);
    s->c1d = std::min(s->c1d, kCav1DMaxCluster);
    s->bounds1d = balance_cells(s, s->c1d);
    for (int r = 0; r < s->c1d; ++r)
      if (s->bounds1d[(size_t)r + 1] - s->bounds1d[(size_t)r] > kCav1DThreads) s->path1d = false;
    s->ncomp1d = 1;
    for (auto& q : s->srcs)
      if (q.comp != 0) s->ncomp1d = 3;
    s->ring_cap = 4096;
  }
  // partial-sum ring: the 3D kernel's layout (nbxy per monitor quantity, nblk3d per energy
  // quantity), or the 1D kernel's (one per warp of its cluster); space for the larger of the two,
  // since a 1D simulation moves to the 3D kernel once a y/z component is set (switch_to_3d)
  s->nblk3d = s->nbx * s->nby * s->nchunks;
  s->red_nbxy = s->nbx * s->nby;
  const int nblk1d = s->c1d * (kCav1DThreads / 32);
  s->red_nblocks = (s->path1d && s->ncomp1d == 1) ? nblk1d : s->nblk3d;
  const int64_t nbxy = s->red_nbxy, nblocks = std::max(s->nblk3d, s->path1d ? nblk1d : 1);
  s->monE_off = 0;
  s->monH_off = 2 * (int64_t)s->mons.size() * nbxy;
  s->enE_off = s->monH_off + 4 * (int64_t)s->mons.size() * nbxy;
  s->enH_off = s->enE_off + 3 * nblocks;
  s->ring_stride = s->enH_off + nblocks;
  s->partial = dalloc(s, (size_t)s->ring_cap * s->ring_stride * 8);
  s->series = dalloc(s, (size_t)s->ring_cap * (6 * s->mons.size() + 4) * 8);
  if (!s->partial || !s->series) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  if (s->path1d) {
    s->src_tab = dalloc(s, (size_t)s->ring_cap * 8);
    if (!s->src_tab) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  }
  if (s->energy_on) {
    s->trace = dalloc(s, (size_t)s->e_cap * 4 * 8);
    if (!s->trace) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  }

  // ---- tables ----
  std::vector<double> pe(2 * nz), ph(2 * nz);
  for (int64_t k = 0; k < nz; ++k) {
    cpml_bc(s, (double)k, &pe[2 * k], &pe[2 * k + 1]);
    cpml_bc(s, (double)k + 0.5, &ph[2 * k], &ph[2 * k + 1]);
  }
  std::vector<double> rows;
  for (auto& m : s->mats) {
    const auto& src = (s->prec == 64) ? m.rowsLit : m.rowsInc;
    rows.insert(rows.end(), src.begin(), src.end());
  }
  if (rows.empty()) rows.assign(kCoefStride, 0.0);
  int rc = 0;
  if (s->prec == 64) {
    rc = rc ? rc : h2d(s, s->pmlE, pe.data(), pe.size() * 8);
    rc = rc ? rc : h2d(s, s->pmlH, ph.data(), ph.size() * 8);
    rc = rc ? rc : h2d(s, s->coef, rows.data(), rows.size() * 8);
  } else {
    auto pef = cast_vec<float>(pe), phf = cast_vec<float>(ph), rf = cast_vec<float>(rows);
    rc = rc ? rc : h2d(s, s->pmlE, pef.data(), pef.size() * 4);
    rc = rc ? rc : h2d(s, s->pmlH, phf.data(), phf.size() * 4);
    rc = rc ? rc : h2d(s, s->coef, rf.data(), rf.size() * 4);
  }
  rc = rc ? rc : h2d(s, s->zstart, starts.data(), starts.size() * sizeof(int));
  rc = rc ? rc : h2d(s, s->chunk_ids, ids.data(), ids.size() * sizeof(int));
  if (rc) return bail(rc, s->err);
  for (int q = 0; q < nsrc; ++q) {
    if (!sources[q].phase) continue;
    std::vector<double> c((size_t)s->plane), sn((size_t)s->plane);
    for (int64_t p = 0; p < s->plane; ++p) {
      c[(size_t)p] = std::cos(sources[q].phase[p]);
      sn[(size_t)p] = std::sin(sources[q].phase[p]);
    }
    s->srcs[q].dcos = dalloc(s, (size_t)s->plane * esz);
    s->srcs[q].dsin = dalloc(s, (size_t)s->plane * esz);
    if (!s->srcs[q].dcos || !s->srcs[q].dsin) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
    rc = store(s, s->srcs[q].dcos, c);
    rc = rc ? rc : store(s, s->srcs[q].dsin, sn);
    if (rc) return bail(rc, s->err);
  }
  for (int q = 0; q < nmon; ++q) {
    s->mons[q].dfreq = dalloc(s, (size_t)monitors[q].nfreq * 8);
    s->mons[q].dacc = dalloc(s, (size_t)monitors[q].nfreq * 8 * 8);
    if (!s->mons[q].dfreq || !s->mons[q].dacc) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
    rc = h2d(s, s->mons[q].dfreq, monitors[q].freqs, (size_t)monitors[q].nfreq * 8);
    if (rc) return bail(rc, s->err);
  }
  ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return bail(FDTDBATH_ERR_CUDA, std::string("create: ") + cudaGetErrorString(ce));
  s->te2d_ok0 = s->te2d_ok;
  *out = s;
  return FDTDBATH_OK;
}

int fdtdbath_step(fdtdbath_sim* s, int64_t nsteps) {
  if (!s || nsteps < 0) return fail(s, FDTDBATH_ERR_ARG, "bad arguments to fdtdbath_step");
  cudaSetDevice(s->device);
  if (s->path1d && s->ncomp1d == 1) {
    int64_t left = nsteps;
    while (left > 0) {
      if (s->n - s->reduced >= s->ring_cap / 2) {
        int rc = reduce_upto(s, s->n);
        if (rc) return rc;
      }
      const int64_t m = std::min<int64_t>(left, s->ring_cap - (s->n - s->reduced));
      int rc = launch_1d(s, m);
      if (rc) return rc;
      s->n += m;
      s->pcur ^= (int)(m & 1);
      left -= m;
    }
    return FDTDBATH_OK;
  }
  for (int64_t it = 0; it < nsteps; ++it) {
    if (s->tb_ok && s->h_pending && nsteps - it >= 2) {
      // two steps in one launch: its partials go to ring slots n-1 .. n+1
      if (s->n + 2 - s->reduced > s->ring_cap) {
        int rc = reduce_upto(s, s->n - 1);
        if (rc) return rc;
      }
      int rc = launch_pair(s);
      if (rc) return rc;
      s->n += 2;   // P slots: no polarizable material
      ++it;
      continue;
    }
    // keep the ring from overwriting partials not yet reduced
    if (s->n + 1 - s->reduced > s->ring_cap) {
      const int64_t complete = s->h_pending ? s->n - 1 : s->n;
      int rc = reduce_upto(s, complete);
      if (rc) return rc;
    }
    int rc = launch_step(s, s->h_pending ? 1 : 0, 1);
    if (rc) return rc;
    s->pcur = 1 - s->pcur;
    s->n += 1;
    s->h_pending = true;
  }
  return FDTDBATH_OK;
}

int fdtdbath_sync(fdtdbath_sim* s) {
  if (!s) return fail(s, FDTDBATH_ERR_ARG, "sim is NULL");
  cudaSetDevice(s->device);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(s, e, "deferred");
  return check_timeout(s);
}

int fdtdbath_read_fields(fdtdbath_sim* s, int32_t field, void* dst, size_t dst_bytes, int32_t dst_on_device) {
  if (!s || !dst) return fail(s, FDTDBATH_ERR_ARG, "NULL argument");
  FieldRef f;
  if (!parse_field(field, &f)) return fail(s, FDTDBATH_ERR_ARG, "unknown field id");
  if (dst_bytes < (size_t)s->ncell * s->esz) return fail(s, FDTDBATH_ERR_ARG, "destination too small");
  cudaSetDevice(s->device);
  int rc = flush_all(s);
  if (rc) return rc;
  std::vector<double> full((size_t)s->ncell, 0.0);
  if (f.kind == 0) {
    const void* src = f.comp < 3 ? elem_ptr(s->E[s->ecur], f.comp * s->ncell, s->esz)
                                 : elem_ptr(s->H[s->hcur], (f.comp - 3) * s->ncell, s->esz);
    rc = fetch(s, src, s->ncell, full);
    if (rc) return rc;
  } else if (f.kind == 3) {
    rc = sigma_full(s, full);
    if (rc) return rc;
  } else {
    for (auto& m : s->mats) {
      std::vector<double> a;
      const void* pa;
      if (f.kind == 1) {
        if (m.kind == FDTDBATH_VACUUM) continue;
        const int64_t off = f.comp * s->nmatcell + m.base;
        pa = elem_ptr(s->Pslot[f.level == 0 ? s->pcur : 1 - s->pcur], off, s->esz);
      } else {
        if (f.mode >= m.nb) continue;
        const int64_t off = m.ybase + ((int64_t)f.comp * m.nb + f.mode) * m.ncell;
        if (s->ybf) {
          std::vector<float> y0, y1;
          rc = fetch_bf16_levels(s, off, m.ncell, y0, y1);
          if (rc) return rc;
          const std::vector<float>& y = f.level == 0 ? y0 : y1;
          for (int64_t r = 0; r < m.ncell; ++r) full[(size_t)(m.zlo * s->plane + r)] = y[(size_t)r];
          continue;
        }
        pa = elem_ptr(s->Yslot[f.level == 0 ? s->pcur : 1 - s->pcur], off, s->esz);
      }
      rc = fetch(s, pa, m.ncell, a);
      if (rc) return rc;
      for (int64_t r = 0; r < m.ncell; ++r) full[(size_t)(m.zlo * s->plane + r)] = a[(size_t)r];
    }
  }
  // convert to the element type and deliver
  if (s->prec == 64) {
    if (dst_on_device) return h2d(s, dst, full.data(), full.size() * 8);
    std::memcpy(dst, full.data(), full.size() * 8);
  } else {
    std::vector<float> tmp(full.size());
    for (size_t i = 0; i < full.size(); ++i) tmp[i] = (float)full[i];
    if (dst_on_device) return h2d(s, dst, tmp.data(), tmp.size() * 4);
    std::memcpy(dst, tmp.data(), tmp.size() * 4);
  }
  return FDTDBATH_OK;
}

int fdtdbath_write_fields(fdtdbath_sim* s, int32_t field, const void* src, size_t src_bytes, int32_t src_on_device) {
  if (!s || !src) return fail(s, FDTDBATH_ERR_ARG, "NULL argument");
  FieldRef f;
  if (!parse_field(field, &f)) return fail(s, FDTDBATH_ERR_ARG, "unknown field id");
  if (src_bytes < (size_t)s->ncell * s->esz) return fail(s, FDTDBATH_ERR_ARG, "source too small");
  // the TE form carries only E_y, H_x, H_z and the y polarization / bath modes
  if ((f.kind == 0 && f.comp != 1 && f.comp != 3 && f.comp != 5) || ((f.kind == 1 || f.kind == 2) && f.comp != 1))
    s->te = false;
  if (f.kind != 3) {
    // the 1D kernel skips the y/z polarization while it provably stays zero
    const bool xpol = (f.kind == 0 && (f.comp == 0 || f.comp == 4)) || (f.kind != 0 && f.comp == 0);
    cudaSetDevice(s->device);
    if (!xpol) {
      const int rc0 = switch_to_3d(s);
      if (rc0) return rc0;
    }
  }
  cudaSetDevice(s->device);
  int rc = flush_all(s);
  if (rc) return rc;
  std::vector<double> in((size_t)s->ncell);
  {
    std::vector<unsigned char> raw((size_t)s->ncell * s->esz);
    if (src_on_device) {
      rc = d2h(s, raw.data(), src, raw.size());
      if (rc) return rc;
    } else {
      std::memcpy(raw.data(), src, raw.size());
    }
    for (int64_t i = 0; i < s->ncell; ++i)
      in[(size_t)i] = s->prec == 64 ? ((const double*)raw.data())[i] : (double)((const float*)raw.data())[i];
  }
  if (f.kind == 3) return set_sigma_map(s, in);
  auto refresh_D = [&](void) -> int {
    // FP64 path: D = eps_inf E + P^{n-1/2} in material cells (the relation E = (D - P)/eps_inf
    // holds between D^{n-1/2}, E^{n-1/2} and P^{n-1/2})
    if (s->prec != 64) return 0;
    for (auto& m : s->mats) {
      for (int c = 0; c < 3; ++c) {
        std::vector<double> e, pm;
        int r = fetch(s, elem_ptr(s->E[s->ecur], c * s->ncell + m.zlo * s->plane, 8), m.ncell, e);
        if (!r) r = fetch(s, elem_ptr(s->Pslot[1 - s->pcur], c * s->nmatcell + m.base, 8), m.ncell, pm);
        if (r) return r;
        std::vector<double> d((size_t)m.ncell);
        for (int64_t q = 0; q < m.ncell; ++q) d[(size_t)q] = m.eps * e[(size_t)q] + pm[(size_t)q];
        r = store(s, elem_ptr(s->D, c * s->nmatcell + m.base, 8), d);
        if (r) return r;
      }
    }
    return 0;
  };
  if (f.kind == 0) {
    void* dstp = f.comp < 3 ? elem_ptr(s->E[s->ecur], f.comp * s->ncell, s->esz)
                            : elem_ptr(s->H[s->hcur], (f.comp - 3) * s->ncell, s->esz);
    rc = store(s, dstp, in);
    if (!rc && f.comp < 3) rc = refresh_D();
    return rc;
  }
  for (auto& m : s->mats) {
    void* pa;
    if (f.kind == 1) {
      if (m.kind == FDTDBATH_VACUUM) continue;
      const int64_t off = f.comp * s->nmatcell + m.base;
      pa = elem_ptr(s->Pslot[f.level == 0 ? s->pcur : 1 - s->pcur], off, s->esz);
    } else {
      if (f.mode >= m.nb) continue;
      const int64_t off = m.ybase + ((int64_t)f.comp * m.nb + f.mode) * m.ncell;
      if (s->ybf) {
        // replace one level, keep the other, store the (value, increment) pair again
        std::vector<float> y0, y1;
        rc = fetch_bf16_levels(s, off, m.ncell, y0, y1);
        if (rc) return rc;
        std::vector<float>& y = f.level == 0 ? y0 : y1;
        for (int64_t r = 0; r < m.ncell; ++r) y[(size_t)r] = (float)in[(size_t)(m.zlo * s->plane + r)];
        rc = store_bf16_levels(s, off, y0, y1);
        if (rc) return rc;
        continue;
      }
      pa = elem_ptr(s->Yslot[f.level == 0 ? s->pcur : 1 - s->pcur], off, s->esz);
    }
    std::vector<double> v(in.begin() + m.zlo * s->plane, in.begin() + m.zlo * s->plane + m.ncell);
    rc = store(s, pa, v);
    if (rc) return rc;
  }
  if (f.kind == 1 && f.level == 1) rc = refresh_D();
  return rc;
}

int fdtdbath_sigma_box(fdtdbath_sim* s, const double lo[3], const double hi[3], double sigma) {
  if (!s || !lo || !hi) return fail(s, FDTDBATH_ERR_ARG, "NULL argument");
  if (!std::isfinite(sigma) || sigma < 0) return fail(s, FDTDBATH_ERR_ARG, "sigma must be finite and non-negative");
  const int64_t n[3] = {s->nx, s->ny, s->nz};
  for (int a = 0; a < 3; ++a)
    if (!(lo[a] >= 0.0 && lo[a] < hi[a] && hi[a] <= (double)n[a]))
      return fail(s, FDTDBATH_ERR_ARG, "the box must satisfy 0 <= lo < hi <= n on every axis");
  cudaSetDevice(s->device);
  int rc = flush_all(s);
  if (rc) return rc;
  std::vector<double> full;
  rc = sigma_full(s, full);
  if (rc) return rc;
  // covered fraction of cell (i, j, k) = [i, i+1) x [j, j+1) x [k, k+1): the product of the
  // overlap lengths of the box with the cell along the three axes
  std::vector<double> ov[3];
  for (int a = 0; a < 3; ++a) {
    ov[a].resize((size_t)n[a]);
    for (int64_t i = 0; i < n[a]; ++i) {
      const double t = std::min(hi[a], (double)(i + 1)) - std::max(lo[a], (double)i);
      ov[a][(size_t)i] = t > 0.0 ? t : 0.0;
    }
  }
  for (int64_t k = (int64_t)lo[2]; k < n[2] && (double)k < hi[2]; ++k)
    for (int64_t j = (int64_t)lo[1]; j < n[1] && (double)j < hi[1]; ++j)
      for (int64_t i = (int64_t)lo[0]; i < n[0] && (double)i < hi[0]; ++i) {
        const double f = ov[0][(size_t)i] * ov[1][(size_t)j] * ov[2][(size_t)k];
        double& v = full[(size_t)((k * n[1] + j) * n[0] + i)];
        v = f * sigma + (1.0 - f) * v;
      }
  return set_sigma_map(s, full);
}

int fdtdbath_dft(fdtdbath_sim* s, int32_t monitor, double* out) {
  if (!s || !out || monitor < 0 || monitor >= (int)s->mons.size()) return fail(s, FDTDBATH_ERR_ARG, "bad monitor");
  cudaSetDevice(s->device);
  int rc = flush_all(s);
  if (rc) return rc;
  const size_t nval = (size_t)s->mons[monitor].nfreq * 8;
  rc = d2h(s, out, s->mons[monitor].dacc, nval * 8);
  if (rc) return rc;
  rc = check_timeout(s);
  if (rc) return rc;
  return check_finite(s, out, nval, "the spectrum");
}

int fdtdbath_energy(fdtdbath_sim* s, double* trace, int64_t maxlen, int64_t* len) {
  if (!s || !len || (maxlen > 0 && !trace)) return fail(s, FDTDBATH_ERR_ARG, "bad arguments");
  *len = 0;
  if (!s->energy_on) return FDTDBATH_OK;
  cudaSetDevice(s->device);
  int rc = flush_all(s);
  if (rc) return rc;
  int64_t n = (s->n + s->e_every - 1) / s->e_every;
  if (n > s->e_cap) n = s->e_cap;
  if (n > maxlen) n = maxlen;
  if (n > 0) rc = d2h(s, trace, s->trace, (size_t)n * 4 * 8);
  *len = n;
  if (!rc) rc = check_timeout(s);
  if (!rc && n > 0) rc = check_finite(s, trace, (size_t)n * 4, "the energy trace");
  return rc;
}

int64_t fdtdbath_steps_done(const fdtdbath_sim* s) { return s ? s->n : -1; }

const char* fdtdbath_last_error(const fdtdbath_sim* s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

void fdtdbath_destroy(fdtdbath_sim* s) {
  if (!s) return;
  if (!s->allocs.empty()) {
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
  }
  for (void* p : s->allocs) {
    if (s->ufree) s->ufree(p, s->uctx);
    else cudaFree(p);
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->side) cudaStreamDestroy(s->side);
  delete s;
}

int fdtdbath_bath_form(int32_t shape, double frequency, double gamma, int32_t num_bath, double width,
                       double bath_gamma, double dephasing, double* frequencies, double* gammas,
                       double* couplings) {
  if (num_bath < 2 || !frequencies || !gammas || !couplings || !(width > 0) || dephasing < 0)
    return fail(nullptr, FDTDBATH_ERR_ARG, "bath_form needs num_bath >= 2, width > 0, dephasing >= 0");
  if (shape < 0 || shape > 2) return fail(nullptr, FDTDBATH_ERR_ARG, "unknown bath shape");
  const double dw = width / (double)(num_bath - 1);
  const double kb = std::sqrt(2.0 * dw / M_PI * dephasing);
  const double G = gamma + dephasing;
  for (int j = 0; j < num_bath; ++j) {
    const double f = (frequency - 0.5 * width) + dw * (double)j;
    frequencies[j] = f;
    gammas[j] = bath_gamma;
    const double d = f - frequency;
    if (shape == FDTDBATH_BATH_UNIFORM) couplings[j] = kb;
    else if (shape == FDTDBATH_BATH_LORENTZIAN) couplings[j] = kb * std::sqrt(G * G / (G * G + d * d));
    else couplings[j] = kb * std::exp(-d * d / (4.0 * G * G));
  }
  return FDTDBATH_OK;
}

int64_t fdtdbath_query(const fdtdbath_sim* s, int32_t key) {
  if (!s) return -1;
  switch (key) {
    case 0: return (int64_t)s->esz;
    case 1: return s->launches;
    case 2: return (int64_t)s->bytes_held;
    case 3: return (int64_t)s->nbx * s->nby * s->nchunks;
    case 4: return s->nchunks;
    case 5: return s->te && s->ty == 1 ? 1 : 0;
    case 6: return s->adj_te ? 1 : 0;
    case 7: return s->plain_ok ? 1 : 0;
    case 8: return s->path1d && s->ncomp1d == 1 ? 1 : 0;
    case 9: return s->bath_plain ? 1 : 0;
    case 10: return s->te2d_ok && s->te && s->ty == 1 ? 1 : 0;
    case 11: return s->sigmap ? 1 : 0;
    case 12: return s->tb_ok ? 1 : 0;
    default: return -1;
  }
}

}  // extern "C"

// ---- discrete adjoint driver ---------------------------------------------------------
namespace {

void dfree(fdtdbath_sim* s, void* p) {
  if (!p) return;
  for (size_t i = 0; i < s->allocs.size(); ++i)
    if (s->allocs[i] == p) {
      s->allocs.erase(s->allocs.begin() + (long)i);
      break;
    }
  if (s->ufree) s->ufree(p, s->uctx);
  else cudaFree(p);
}

struct StateRef {
  void* p;
  size_t bytes;
};

// The buffers that make up the state after a flushed step (the order of a checkpoint).
std::vector<StateRef> state_refs(fdtdbath_sim* s) {
  const size_t e = s->esz;
  std::vector<StateRef> v;
  v.push_back({s->E[s->ecur], 3 * (size_t)s->ncell * e});
  v.push_back({s->H[s->hcur], 3 * (size_t)s->ncell * e});
  v.push_back({s->psiE, 2 * (size_t)(2 * s->npml) * s->plane * e});
  v.push_back({s->psiH[s->psicur], 2 * (size_t)(2 * s->npml + 1) * s->plane * e});
  if (s->prec == 64) v.push_back({s->D, 3 * (size_t)s->nmatcell * e});
  for (int b = 0; b < 2; ++b) v.push_back({s->Pslot[b], 3 * (size_t)s->nmatcell * e});
  for (int b = 0; b < 2; ++b)
    v.push_back({s->Yslot[b], s->ybf ? (b == 0 ? (size_t)s->nybath * 4 : 16) : (size_t)s->nybath * s->yesz});
  return v;
}

int checkpoint_io(fdtdbath_sim* s, void* buf, bool save) {
  size_t off = 0;
  for (const StateRef& r : state_refs(s)) {
    if (r.bytes) {
      char* c = (char*)buf + off;
      cudaError_t e = save ? cudaMemcpyAsync(c, r.p, r.bytes, cudaMemcpyDeviceToDevice, s->stream)
                           : cudaMemcpyAsync(r.p, c, r.bytes, cudaMemcpyDeviceToDevice, s->stream);
      if (e != cudaSuccess) return cuda_fail(s, e, "checkpoint copy");
    }
    off += (r.bytes + 255) & ~size_t(255);
  }
  return 0;
}

size_t checkpoint_bytes(fdtdbath_sim* s) {
  size_t n = 0;
  for (const StateRef& r : state_refs(s)) n += (r.bytes + 255) & ~size_t(255);
  return n;
}

int save_checkpoint(fdtdbath_sim* s, size_t idx) {
  int rc = flush_h(s);
  if (rc) return rc;
  AdjState& a = s->adj;
  if (idx >= a.cps.size()) {
    void* p = dalloc(s, a.cp_bytes);
    if (!p) return fail(s, FDTDBATH_ERR_OOM, "checkpoint allocation failed");
    a.cps.push_back(p);
    a.cp_n.push_back(0);
    a.cp_pcur.push_back(0);
  }
  a.cp_n[idx] = s->n;
  a.cp_pcur[idx] = s->pcur;
  return checkpoint_io(s, a.cps[idx], true);
}

int restore_checkpoint(fdtdbath_sim* s, size_t idx) {
  AdjState& a = s->adj;
  s->h_pending = false;
  int rc = checkpoint_io(s, a.cps[idx], false);
  if (rc) return rc;
  s->n = a.cp_n[idx];
  s->pcur = a.cp_pcur[idx];
  s->reduced = s->n;
  return 0;
}

int launch_adjoint(const AdjParams<float>& p, int nbmax, bool te, cudaStream_t st) {
  return launch_adjoint_f32(p, nbmax, te ? 1 : 0, st);
}
int launch_adjoint(const AdjParams<double>& p, int nbmax, bool te, cudaStream_t st) {
  return launch_adjoint_f64(p, nbmax, te ? 1 : 0, st);
}

template <typename T>
int adjoint_sweep(fdtdbath_sim* s, const HostMon& mon, const std::vector<double>& freqs, const double* dLdF,
                  int gm, std::vector<double>& grad) {
  AdjState& A = s->adj;
  const int64_t N = s->ncell, plane = s->plane;
  const size_t e = s->esz;
  const HostMat& G = s->mats[(size_t)gm];
  const int64_t ncm = G.ncell;
  const int nb = G.nb;
  const int L = A.every;
  // ---- buffers ----
  std::vector<void*> bufs;
  bool oom = false;
  auto get = [&](size_t bytes) -> void* {
    void* p = dalloc(s, bytes);
    if (p) bufs.push_back(p);
    else oom = true;
    return p;
  };
  T* Eb = (T*)get(3 * (size_t)N * e);
  T* Hb = (T*)get(3 * (size_t)N * e);
  T* psE[2] = {(T*)get(2 * (size_t)(2 * s->npml) * plane * e), (T*)get(2 * (size_t)(2 * s->npml) * plane * e)};
  T* psH[2] = {(T*)get(2 * (size_t)(2 * s->npml + 1) * plane * e), (T*)get(2 * (size_t)(2 * s->npml + 1) * plane * e)};
  T* Pb = (T*)get(3 * (size_t)s->nmatcell * e);
  T* Pmb = (T*)get(3 * (size_t)s->nmatcell * e);
  T* Yb0 = (T*)get((size_t)s->nybath * e);
  T* Yb1 = (T*)get((size_t)s->nybath * e);
  T* snapE = (T*)get((size_t)L * 3 * ncm * e);
  T* snapP = (T*)get((size_t)(L + 2) * 3 * ncm * e);
  T* snapY = (T*)get((size_t)(L + 2) * 3 * std::max(1, nb) * ncm * e);
  const int64_t nblk = adjoint_blocks(N);
  double* gpart = (double*)get((size_t)nblk * kAdjMaxGrad * sizeof(double));
  int nrows = 0;
  for (auto& m : s->mats) nrows += m.nb;
  T* coefLit = (T*)get((size_t)std::max(1, nrows) * kCoefStride * e);
  signed char* zmat = (signed char*)get((size_t)s->nz);
  auto release = [&]() {
    for (void* p : bufs) dfree(s, p);
  };
  if (oom) {
    release();
    return fail(s, FDTDBATH_ERR_OOM, "adjoint buffer allocation failed");
  }
  // material index of every plane
  {
    std::vector<signed char> zm((size_t)s->nz, (signed char)-1);
    for (size_t m = 0; m < s->mats.size(); ++m)
      for (int64_t z = s->mats[m].zlo; z < s->mats[m].zhi; ++z) zm[(size_t)z] = (signed char)m;
    const int rc = h2d(s, zmat, zm.data(), zm.size());
    if (rc) {
      release();
      return rc;
    }
  }
  // literal coefficient rows in the state precision
  {
    std::vector<T> rows;
    for (auto& m : s->mats)
      for (double v : m.rowsLit) rows.push_back((T)v);
    if (rows.empty()) rows.assign(kCoefStride, T(0));
    int rc = h2d(s, coefLit, rows.data(), rows.size() * e);
    if (rc) {
      release();
      return rc;
    }
  }
  // ---- monitor adjoint sources per step: dL/d(plane mean) / plane ----
  const int64_t n0 = A.n0, NS = A.nsteps;
  std::vector<double> gE((size_t)NS * 2, 0.0), gH((size_t)NS * 2, 0.0);
  for (int64_t m = 0; m < NS; ++m) {
    const double tE = ((double)(n0 + m) + 0.5) * s->dt, tH = ((double)(n0 + m) + 1.0) * s->dt;
    for (int f = 0; f < mon.nfreq; ++f) {
      const double aE = 2.0 * M_PI * freqs[(size_t)f] * tE, aH = 2.0 * M_PI * freqs[(size_t)f] * tH;
      const double cE = std::cos(aE), sE = std::sin(aE), cH = std::cos(aH), sH = std::sin(aH);
      const double* d = dLdF + (size_t)f * 8;
      gE[(size_t)m * 2 + 0] += (d[0] * cE + d[1] * sE) * s->dt;
      gE[(size_t)m * 2 + 1] += (d[2] * cE + d[3] * sE) * s->dt;
      gH[(size_t)m * 2 + 0] += (d[4] * cH + d[5] * sH) * s->dt;
      gH[(size_t)m * 2 + 1] += (d[6] * cH + d[7] * sH) * s->dt;
    }
  }
  // TE form of the reverse sweep: the forward run was the TE form and nothing drives the
  // adjoints of E_x or H_y, so those (and E_z, P_x, P_z, the x / z bath modes) stay zero
  bool te = s->te && s->ty == 1;
  for (int64_t m = 0; m < NS && te; ++m)
    if (gE[(size_t)m * 2] != 0.0 || gH[(size_t)m * 2 + 1] != 0.0) te = false;
  s->adj_te = te;
  // ---- constant part of the kernel parameters ----
  AdjParams<T> p{};
  p.nx = (int)s->nx;
  p.ny = (int)s->ny;
  p.nz = (int)s->nz;
  p.npml = s->npml;
  p.plane = plane;
  p.ncell = N;
  p.nmatcell = s->nmatcell;
  p.S = (T)(s->dt / s->dx);
  p.dt = (T)s->dt;
  p.pmlE = (const T*)s->pmlE;
  p.pmlH = (const T*)s->pmlH;
  p.Eb = Eb;
  p.Hb = Hb;
  p.Pb = Pb;
  p.Pmb = Pmb;
  p.Yb0 = Yb0;
  p.Yb1 = Yb1;
  p.coefLit = coefLit;
  p.nmat = (int)s->mats.size();
  int off = 0;
  for (size_t m = 0; m < s->mats.size(); ++m) {
    p.mat[m] = mat_k<T>(s->mats[m], off, s->dt);
    off += s->mats[m].nb;
  }
  p.zm = (int)mon.z;
  p.gm = gm;
  const double dt = s->dt;
  p.dcE = G.w0 * G.w0 * dt * dt;
  p.halfdt = 0.5 * dt;
  p.invA = 1.0 / G.A;
  for (int j = 0; j < nb; ++j) {
    const double den = 1.0 + 0.5 * G.gj[(size_t)j] * dt;
    p.ga[j] = (2.0 - G.wj[(size_t)j] * G.wj[(size_t)j] * dt * dt) / den;
    p.gb[j] = -2.0 / den;
    p.gk[j] = G.kj[(size_t)j];
    p.gdc[j] = dt / (2.0 * den);
    p.gds[j] = G.kj[(size_t)j] * dt / den;
    p.ta[j] = (T)p.ga[j];
    p.tb[j] = (T)p.gb[j];
    p.tdc[j] = (T)p.gdc[j];
    p.tds[j] = (T)p.gds[j];
  }
  p.tsig = (T)(p.dcE * p.invA);
  p.thA = (T)(p.halfdt * p.invA);
  p.gpart = gpart;
  p.fd_plane = make_fastdiv((uint32_t)plane);
  p.fd_nx = make_fastdiv((uint32_t)s->nx);
  p.zmat = zmat;
  // every adjoint buffer starts at zero (dalloc zeroes them)
  const bool save_quiet = s->quiet;
  s->quiet = true;
  int ps = 0;   // current psi adjoint buffers
  int rc = 0;
  auto snap = [&](T* dst, const void* src, size_t count) -> int {
    cudaError_t ce = cudaMemcpyAsync(dst, src, count * e, cudaMemcpyDeviceToDevice, s->stream);
    return ce == cudaSuccess ? 0 : cuda_fail(s, ce, "adjoint snapshot");
  };
  const int64_t ncp = (NS + L - 1) / L;
  // a TE forward run keeps the x / z components of E, P and the bath modes at zero: only the
  // y component is recorded (the record buffers start at zero and the others stay so)
  const bool te_rec = s->te && s->ty == 1;
  auto live = [&](int cc) { return !te_rec || cc == 1; };
  const size_t yoff = te_rec ? (size_t)nb * ncm : 0, ycount = (te_rec ? 1 : 3) * (size_t)nb * ncm;
  for (int64_t c = ncp - 1; c >= 0 && !rc; --c) {
    rc = restore_checkpoint(s, (size_t)c);
    if (rc) break;
    const int64_t s0 = c * L;
    const int Lc = (int)std::min<int64_t>(L, NS - s0);
    // levels n-1/2 and n+1/2 of the material at the segment start
    for (int lv = 0; lv < 2 && !rc; ++lv) {
      const int slot = lv == 0 ? 1 - s->pcur : s->pcur;
      for (int cc = 0; cc < 3 && !rc; ++cc)
        if (live(cc))
          rc = snap(snapP + ((size_t)lv * 3 + cc) * ncm, elem_ptr(s->Pslot[slot], cc * s->nmatcell + G.base, e), (size_t)ncm);
      if (!rc && nb)
        rc = snap(snapY + (size_t)lv * 3 * nb * ncm + yoff, elem_ptr(s->Yslot[slot], G.ybase + (int64_t)yoff, e), ycount);
    }
    // recompute the segment, recording the material's E, P and Y after every step
    for (int m = 0; m < Lc && !rc; ++m) {
      rc = launch_step(s, s->h_pending ? 1 : 0, 1);
      if (rc) break;
      s->pcur = 1 - s->pcur;
      s->n += 1;
      s->h_pending = true;
      s->reduced = s->n;
      for (int cc = 0; cc < 3 && !rc; ++cc) {
        if (!live(cc)) continue;
        rc = snap(snapE + ((size_t)m * 3 + cc) * ncm, elem_ptr(s->E[s->ecur], cc * N + G.zlo * plane, e), (size_t)ncm);
        if (!rc)
          rc = snap(snapP + ((size_t)(m + 2) * 3 + cc) * ncm, elem_ptr(s->Pslot[s->pcur], cc * s->nmatcell + G.base, e),
                    (size_t)ncm);
      }
      if (!rc && nb)
        rc = snap(snapY + (size_t)(m + 2) * 3 * nb * ncm + yoff, elem_ptr(s->Yslot[s->pcur], G.ybase + (int64_t)yoff, e),
                  ycount);
    }
    // reverse sweep over the segment
    for (int m = Lc - 1; m >= 0 && !rc; --m) {
      const int64_t ng = s0 + m;
      p.fE = snapE + (size_t)m * 3 * ncm;
      p.fPn = snapP + (size_t)(m + 2) * 3 * ncm;
      p.fPm = snapP + (size_t)m * 3 * ncm;
      p.fY = snapY + (size_t)(m + 1) * 3 * std::max(1, nb) * ncm;
      p.fYm = snapY + (size_t)m * 3 * std::max(1, nb) * ncm;
      const double ip = 1.0 / (double)plane;
      p.gEx = (T)(gE[(size_t)ng * 2] * ip);
      p.gEy = (T)(gE[(size_t)ng * 2 + 1] * ip);
      p.gHx = (T)(gH[(size_t)ng * 2] * ip);
      p.gHy = (T)(gH[(size_t)ng * 2 + 1] * ip);
      p.psiEb = psE[ps];
      p.psiEb_out = psE[1 - ps];
      p.psiHb = psH[ps];
      p.psiHb_out = psH[1 - ps];
      const int lr = launch_adjoint(p, s->nbmax, te, s->stream);
      s->launches += 2;
      if (lr) rc = cuda_fail(s, (cudaError_t)lr, "adjoint kernel launch");
      ps = 1 - ps;
    }
  }
  // gradient: fixed-order sum of the per-block partials
  if (!rc) {
    std::vector<double> h((size_t)nblk * kAdjMaxGrad);
    rc = d2h(s, h.data(), gpart, h.size() * sizeof(double));
    grad.assign((size_t)(2 + nb), 0.0);
    for (int64_t b = 0; b < nblk && !rc; ++b)
      for (int t = 0; t < 2 + nb; ++t) grad[(size_t)t] += h[(size_t)b * kAdjMaxGrad + t];
  }
  s->quiet = save_quiet;
  release();
  return rc;
}

}  // namespace

int fdtdbath_adjoint_forward(fdtdbath_sim* s, int64_t nsteps, int32_t checkpoint_every) {
  if (!s || nsteps < 1 || checkpoint_every < 1) return fail(s, FDTDBATH_ERR_ARG, "bad arguments to fdtdbath_adjoint_forward");
  if (s->ybf) return fail(s, FDTDBATH_ERR_UNSUPPORTED, "the adjoint does not run on bf16 bath storage");
  if (s->sigmap) return fail(s, FDTDBATH_ERR_UNSUPPORTED, "the adjoint does not run with a per-cell sigma(r) map");
  if (s->nbmax > kMaxBath) return fail(s, FDTDBATH_ERR_UNSUPPORTED, "the adjoint handles at most 32 bath modes per material");
  cudaSetDevice(s->device);
  AdjState& a = s->adj;
  {
    const int rc0 = switch_to_3d(s);   // single-step launches: the persistent 1D kernel is not used
    if (rc0) return rc0;
  }
  a.recorded = false;
  a.n0 = s->n;
  a.nsteps = nsteps;
  a.every = checkpoint_every;
  a.cp_bytes = checkpoint_bytes(s);
  const int64_t ncp = (nsteps + checkpoint_every - 1) / checkpoint_every;
  for (int64_t c = 0; c < ncp; ++c) {
    int rc = save_checkpoint(s, (size_t)c);
    if (rc) return rc;
    rc = fdtdbath_step(s, std::min<int64_t>(checkpoint_every, nsteps - c * checkpoint_every));
    if (rc) return rc;
  }
  int rc = flush_all(s);
  if (rc) return rc;
  rc = save_checkpoint(s, (size_t)ncp);   // the state at the end, put back after the reverse sweep
  if (rc) return rc;
  a.recorded = true;
  return FDTDBATH_OK;
}

int fdtdbath_adjoint_backward(fdtdbath_sim* s, int32_t monitor, const double* dL_dF, int32_t material, double* grad) {
  if (!s || !dL_dF || !grad) return fail(s, FDTDBATH_ERR_ARG, "NULL argument");
  AdjState& a = s->adj;
  if (!a.recorded) return fail(s, FDTDBATH_ERR_ARG, "no recorded forward run: call fdtdbath_adjoint_forward first");
  if (monitor < 0 || monitor >= (int)s->mons.size()) return fail(s, FDTDBATH_ERR_ARG, "bad monitor");
  int gm = -1;
  for (size_t m = 0; m < s->mats.size(); ++m)
    if (s->mats[m].user_index == material) gm = (int)m;
  if (gm < 0) return fail(s, FDTDBATH_ERR_ARG, "bad material index");
  if (s->mats[(size_t)gm].kind == FDTDBATH_VACUUM) return fail(s, FDTDBATH_ERR_ARG, "a vacuum layer has no oscillator parameters");
  if (s->n != a.n0 + a.nsteps) return fail(s, FDTDBATH_ERR_ARG, "the simulation has moved since the recorded forward run");
  cudaSetDevice(s->device);
  const HostMon& mon = s->mons[(size_t)monitor];
  std::vector<double> freqs((size_t)mon.nfreq);
  int rc = d2h(s, freqs.data(), mon.dfreq, freqs.size() * sizeof(double));
  if (rc) return rc;
  std::vector<double> g;
  rc = s->prec == 64 ? adjoint_sweep<double>(s, mon, freqs, dL_dF, gm, g) : adjoint_sweep<float>(s, mon, freqs, dL_dF, gm, g);
  // put the recorded end state back in every case
  const int rc2 = restore_checkpoint(s, a.cps.size() - 1);
  if (rc) return rc;
  if (rc2) return rc2;
  // the caller's parameters are in nu-units: gamma0 = 2 pi gamma, k_j = 2 pi coupling_j
  grad[0] = g[0];
  grad[1] = 2.0 * M_PI * g[1];
  for (size_t j = 2; j < g.size(); ++j) grad[j] = 2.0 * M_PI * g[j];
  return FDTDBATH_OK;
}

// ---- snapshot / restore of the whole state -------------------------------------------
namespace {

// Header of a snapshot: the layout it was taken from (checked on restore) and the progress.
struct SnapHeader {
  char magic[8];
  int32_t version, prec, ybf, nmon;
  int64_t nx, ny, nz, npml, nmatcell, nybath, e_cap;
  int32_t nfreq[kMaxMon];
  int64_t n;
  int32_t pcur, te, ncomp1d, hpend;
  int64_t state_bytes, dft_bytes, trace_bytes, ring_bytes;
  int32_t sigmap;   // a per-cell sigma(r) map follows the pending step's partial sums
};
constexpr char kSnapMagic[8] = {'F', 'D', 'T', 'D', 'B', 'S', 'N', '1'};
constexpr size_t kSnapHead = 256;
static_assert(sizeof(SnapHeader) <= kSnapHead, "snapshot header");

SnapHeader snap_header(const fdtdbath_sim* s) {
  SnapHeader h{};
  std::memcpy(h.magic, kSnapMagic, 8);
  h.version = 2;
  h.prec = s->prec;
  h.ybf = s->ybf ? 1 : 0;
  h.nmon = (int32_t)s->mons.size();
  h.nx = s->nx;
  h.ny = s->ny;
  h.nz = s->nz;
  h.npml = s->npml;
  h.nmatcell = s->nmatcell;
  h.nybath = s->nybath;
  h.e_cap = s->energy_on ? s->e_cap : 0;
  for (size_t m = 0; m < s->mons.size(); ++m) h.nfreq[m] = s->mons[m].nfreq;
  h.n = s->n;
  h.pcur = s->pcur;
  h.te = s->te ? 1 : 0;
  h.ncomp1d = s->ncomp1d;
  h.state_bytes = (int64_t)checkpoint_bytes(const_cast<fdtdbath_sim*>(s));
  for (auto& mo : s->mons) h.dft_bytes += (int64_t)mo.nfreq * 8 * 8;
  h.trace_bytes = h.e_cap * 4 * 8;
  h.hpend = s->h_pending ? 1 : 0;
  h.ring_bytes = s->ring_stride * 8;
  h.sigmap = s->sigmap ? 1 : 0;
  return h;
}

// Copy every piece of a snapshot between the simulation and buf (host or device), in order:
// header, device state (the checkpoint layout), DFT accumulators, energy trace, and -- while the
// H half-step of the last step is pending -- the partial sums of that step (its E half).
int snap_io(fdtdbath_sim* s, char* buf, bool save, bool on_device, bool hpend, bool smap) {
  const cudaMemcpyKind to_buf = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const cudaMemcpyKind from_buf = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  size_t off = kSnapHead;
  auto piece = [&](void* dev, size_t bytes) -> int {
    if (bytes) {
      cudaError_t e = save ? cudaMemcpyAsync(buf + off, dev, bytes, to_buf, s->stream)
                           : cudaMemcpyAsync(dev, buf + off, bytes, from_buf, s->stream);
      if (e != cudaSuccess) return cuda_fail(s, e, save ? "snapshot copy" : "restore copy");
    }
    off += (bytes + 255) & ~size_t(255);
    return 0;
  };
  for (const StateRef& r : state_refs(s)) {
    const int rc = piece(r.p, r.bytes);
    if (rc) return rc;
  }
  for (auto& mo : s->mons) {
    const int rc = piece(mo.dacc, (size_t)mo.nfreq * 8 * 8);
    if (rc) return rc;
  }
  if (s->energy_on) {
    const int rc = piece(s->trace, (size_t)s->e_cap * 4 * 8);
    if (rc) return rc;
  }
  if (hpend) {
    const int64_t slot = (s->n - 1) % s->ring_cap;
    const int rc = piece((double*)s->partial + slot * s->ring_stride, (size_t)s->ring_stride * 8);
    if (rc) return rc;
  } else {
    off += ((size_t)s->ring_stride * 8 + 255) & ~size_t(255);
  }
  if (smap) {
    const int rc = piece(s->sig, (size_t)s->nmatcell * s->esz);
    if (rc) return rc;
  }
  const cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "snapshot stream");
  return 0;
}

// Bytes of a snapshot (with room for the pending step's partial sums, whether pending or not).
size_t snap_bytes(fdtdbath_sim* s) {
  size_t n = kSnapHead + checkpoint_bytes(s);
  for (auto& mo : s->mons) n += ((size_t)mo.nfreq * 64 + 255) & ~size_t(255);
  if (s->energy_on) n += ((size_t)s->e_cap * 32 + 255) & ~size_t(255);
  n += ((size_t)s->ring_stride * 8 + 255) & ~size_t(255);
  n += ((size_t)s->nmatcell * s->esz + 255) & ~size_t(255);   // a sigma(r) map, whether set or not
  return n;
}

}  // namespace

extern "C" {

int fdtdbath_snapshot_size(fdtdbath_sim* s, size_t* bytes) {
  if (!s || !bytes) return fail(s, FDTDBATH_ERR_ARG, "NULL argument");
  *bytes = snap_bytes(s);
  return FDTDBATH_OK;
}

int fdtdbath_snapshot(fdtdbath_sim* s, void* dst, size_t dst_bytes, int32_t dst_on_device) {
  if (!s || !dst) return fail(s, FDTDBATH_ERR_ARG, "NULL argument");
  if (dst_bytes < snap_bytes(s)) return fail(s, FDTDBATH_ERR_ARG, "snapshot buffer smaller than fdtdbath_snapshot_size");
  cudaSetDevice(s->device);
  // the partial sums of every complete step folded into the spectra and the trace; a pending H
  // half-step stays pending (the resumed run computes it in the launch the original would have)
  int rc = reduce_upto(s, s->h_pending ? s->n - 1 : s->n);
  if (rc) return rc;
  const SnapHeader h = snap_header(s);
  if (dst_on_device) {
    cudaError_t e = cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "snapshot header");
  } else {
    std::memcpy(dst, &h, sizeof(h));
  }
  return snap_io(s, (char*)dst, true, dst_on_device != 0, h.hpend != 0, h.sigmap != 0);
}

int fdtdbath_restore(fdtdbath_sim* s, const void* src, size_t src_bytes, int32_t src_on_device) {
  if (!s || !src) return fail(s, FDTDBATH_ERR_ARG, "NULL argument");
  cudaSetDevice(s->device);
  if (src_bytes < snap_bytes(s)) return fail(s, FDTDBATH_ERR_ARG, "snapshot smaller than this simulation's state");
  SnapHeader h{};
  if (src_on_device) {
    cudaError_t e = cudaMemcpy(&h, src, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "restore header");
  } else {
    std::memcpy(&h, src, sizeof(h));
  }
  SnapHeader mine = snap_header(s);
  const bool same = std::memcmp(h.magic, kSnapMagic, 8) == 0 && h.version == 2 && h.prec == mine.prec &&
                    h.ybf == mine.ybf && h.nmon == mine.nmon && h.nx == mine.nx && h.ny == mine.ny &&
                    h.nz == mine.nz && h.npml == mine.npml && h.nmatcell == mine.nmatcell &&
                    h.nybath == mine.nybath && h.e_cap == mine.e_cap &&
                    std::memcmp(h.nfreq, mine.nfreq, sizeof(h.nfreq)) == 0 && h.state_bytes == mine.state_bytes &&
                    h.ring_bytes == mine.ring_bytes && h.n >= 0 && (h.pcur == 0 || h.pcur == 1) &&
                    (h.ncomp1d == 1 || h.ncomp1d == 3) && (h.hpend == 0 || (h.hpend == 1 && h.n > 0)) &&
                    (h.sigmap == 0 || h.sigmap == 1);
  if (!same) return fail(s, FDTDBATH_ERR_ARG, "the snapshot was taken from a simulation of another layout");
  int rc = flush_all(s);   // nothing of this simulation's own queue may land after the restore
  if (rc) return rc;
  if (s->ncomp1d == 1 && h.ncomp1d == 3) {
    rc = switch_to_3d(s);   // the snapshot's 1D simulation had left the persistent 1D kernel
    if (rc) return rc;
  }
  s->n = h.n;   // the ring slot of a pending step is addressed through n
  if (h.sigmap && !s->sig) {
    s->sig = dalloc(s, (size_t)s->nmatcell * s->esz);
    if (!s->sig) return fail(s, FDTDBATH_ERR_OOM, "device allocation failed");
  }
  rc = snap_io(s, (char*)const_cast<void*>(src), false, src_on_device != 0, h.hpend != 0, h.sigmap != 0);
  if (rc) return rc;
  sigma_mode(s, h.sigmap != 0);   // the snapshot's sigma(r) map, or the layers' own sigma
  s->h_pending = h.hpend != 0;
  s->reduced = s->h_pending ? h.n - 1 : h.n;
  s->pcur = h.pcur;
  if (!h.te) s->te = false;
  s->adj.recorded = false;
  return FDTDBATH_OK;
}

}  // extern "C"
