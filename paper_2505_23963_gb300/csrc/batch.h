// batch.h -- data structures of the batched 1D form: many independent x-polarized 1D
// cavities of uneven length advanced by ONE persistent launch (batch1d.cuh), planned by the
// host packer in batch.cpp.
//
// Canonical device state of a batch (one allocation, type T = float or double):
//   E, H, P, PM, D, psiE, psiH : [ncell_total], cavity i at cells [cav_off[i], cav_off[i]+nz_i);
//                                E_x, H_y, P_x^{n+1/2}, P_x^{n-1/2}, D_x (FP64 form), CPML memories
//   bE, cE, bH, cH             : [ncell_total] CPML coefficients (b = 1, c = 0 outside the slabs)
//   Y0, Y1                     : bath modes Y_j^{n+1/2} / Y_j^{n-1/2}, per Lorentz-Bath material
//                                m a block [nb_m][ncell_m] starting at MatK::ybase
// During a launch every CTA holds its cells in shared memory; the canonical arrays are read at
// the start of the launch and written back at its end.
//
// Packing: the cavities are distributed over the clusters of the launch; the cavities of one
// cluster are laid end to end and cut into one contiguous cell range per CTA.  A CTA's range is
// a list of segments (a contiguous z-range of one cavity), each a list of runs (cells with one
// update kind, material, CPML and energy-box status).  A cavity cut between two CTAs of a
// cluster exchanges its boundary fields through distributed shared memory.
#pragma once

#include <cstdint>

#include "internal.h"

namespace fdtdbath {

constexpr int kBatchMaxSeg = 8;      // segments per CTA
constexpr int kBatchMaxRun = 64;     // runs per CTA
constexpr int kBatchMaxMat = 16;     // material slots per CTA
constexpr int kBatchMaxThreads = 1024;
constexpr int kBatchMaxWarps = kBatchMaxThreads / 32;
constexpr int kBatchMaxCluster = 16;
constexpr int kBatchChunk = 32;     // steps between the kernel's global-memory exchanges
constexpr int kBatchMaxCellsPerThread = 16;   // cells of one Lorentz-Bath run per thread

enum BatchRunKind { kRunVacuum = 0, kRunOsc = 1, kRunBath = 2 };

struct BatchRun {
  int l0, l1;      // local cells [l0, l1) of the CTA
  int kind;        // BatchRunKind
  int mslot;       // material slot of the CTA (kind > 0)
  int seg;         // segment of the CTA holding the run
  int inbox;       // 1: the cells are inside the cavity's energy box
  int psiE, psiH;  // 1: the cells carry a CPML memory of the E / H update
  int psi0;        // psi slot of the run's first cell (when psiE or psiH)
  int p0;          // kind > 0: shared-memory element offset of [P level 0 | P level 1 | D] blocks
  int y0;          // kind 2: shared-memory element offset of the bath block [2][nb][len]
  int nb;          // kind 2: bath modes
};

struct BatchSeg {
  int cav;         // cavity
  int z0, z1;      // cavity cells [z0, z1) held by the CTA
  int l0, l1;      // their local cells
  int link_left;   // 1: cell z0-1 is the last cell of the previous CTA of the cluster
  int link_right;  // 1: cell z1 is the first cell of the next CTA of the cluster
  int src_l;       // local cell of the cavity's soft source, -1 when not in this segment
  int slot;        // energy record slot of this segment
  int64_t g0;      // canonical index of cell z0
  int64_t src_off; // first entry of the cavity's source-amplitude table
  int src_len;     // entries of that table (the amplitude is exactly 0 after it)
  int pad;
};

struct BatchCta {
  int ncell, nseg, nrun, nmat, npsi;
  int seg0, run0, mat0;   // first entries of this CTA in the global seg / run / mat-slot lists
  int prev_ncell;         // cells of the previous CTA of the cluster (left link)
  int prev_off_H;         // byte offset of that CTA's H_y array (off_E is 0 in every CTA)
  int coef_rows;          // bath-mode coefficient rows of the CTA's material slots
  // dynamic shared-memory layout, byte offsets
  int off_E, off_H, off_psi, off_P, off_coef;
  int smem_bytes;
};

template <typename T>
struct BatchParams {
  const long long* ctr;    // completed steps before this launch (device counter)
  int nsteps;
  T S, dt;
  const BatchCta* ctas;
  const BatchSeg* segs;
  const BatchRun* runs;
  const int* matslot;      // global material id of every CTA material slot
  const MatK<T>* mats;
  const T* coef;           // [rows][kCoefStride]
  T *E, *H, *P, *PM, *D, *psiE, *psiH;
  const T *bE, *cE, *bH, *cH;
  T *Y0, *Y1;
  const double* src_tab;
  int energy_on, every, ring_cap;
  int64_t ring_stride;     // doubles per record = 4 * slots
  double* partial;         // [ring_cap][slots][4]: (sum eps E^2, P energy, bath energy, sum H^2)
};

struct BatchReduceParams {
  const long long* ctr;
  int nsteps, every, ring_cap;
  int64_t ring_stride;
  const double* partial;
  const int* slot_ptr;     // [ncav + 1] CSR over slot_idx
  const int* slot_idx;     // energy record slots of each cavity, in CTA order
  int ncav;
  double* trace;           // [ncav][trace_cap][4]
  int64_t trace_cap;
  double ew;               // dx (1D)
};

int launch_batch1d_f32(const BatchParams<float>& p, int nctas, int cluster, int threads, int smem,
                       void* stream);
int launch_batch1d_f64(const BatchParams<double>& p, int nctas, int cluster, int threads, int smem,
                       void* stream);
// Co-resident clusters of a launch shape (0 when it cannot launch) and the kernel's static
// shared memory; prepares the kernel attributes for that shape.
int batch1d_occupancy(int prec, int cluster, int threads, int smem, int* max_clusters,
                      int* static_smem);
int launch_batch_reduce(const BatchReduceParams& r, void* stream);
int launch_batch_advance(long long* ctr, int nsteps, void* stream);

}  // namespace fdtdbath
