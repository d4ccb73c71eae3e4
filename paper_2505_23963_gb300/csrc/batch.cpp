// batch.cpp -- host side of the batched 1D form (include/fdtdbath.h, "Batched 1D cavities"):
// validation, the packer that lays the cavities out over the clusters and CTAs of one persistent
// launch, the launch-shape autotuner, the CUDA-graph step driver and the C ABI.
//
// Packer.  A cavity is cut into pieces: maximal z-ranges whose cells share one update kind,
// material, CPML status and energy-box status, so every cell of a piece has the same cost in work
// units and shared-memory bytes.  Cavities are assigned to clusters longest-processing-time first
// (each to the least-loaded cluster with shared memory to spare); the cavities of a cluster are
// laid end to end and cut into at most C contiguous CTA ranges by a greedy fill under a bound on
// the work of one thread (the kernel deals a CTA's cells round-robin over its threads, so a
// Lorentz-Bath run's remainder falls on some threads only), the smallest feasible bound being
// found by bisection.  A fill also respects the shared-memory budget and the descriptor limits
// of a CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/fdtdbath.h"
#include "batch.h"
#include "host_common.h"

using namespace fdtdbath;

namespace {

thread_local std::string g_batch_create_error;

// work units per cell and step (calibrated on the device: a bath mode costs about one vacuum
// cell's E and H half-steps)
constexpr int64_t kWorkVac = 4, kWorkPsi = 2, kWorkOsc = 8, kWorkBathBase = 8, kWorkMode = 4;

struct Piece {
  int64_t z0, z1;
  int kind;         // BatchRunKind
  int mat;          // global material index, -1 for vacuum
  int nb;
  int psiE, psiH, inbox;
  int64_t work;     // per cell
  int64_t bytes;    // shared memory per cell
};

struct BCav {
  int64_t nz, off;
  int npml;
  std::vector<int> mats;   // global material indices, by z
  int64_t elo, ehi;
  int64_t src_z;           // -1: no source
  double amp, nu, fwidth, t0, phase;
  int64_t src_off;
  int src_len;
  std::vector<Piece> pieces;
  int64_t work, bytes;
};

struct PlanCta {
  std::vector<BatchSeg> segs;
  std::vector<BatchRun> runs;
  std::vector<int> mslots;   // global material ids
  BatchCta d{};
  int64_t work = 0;
};

struct Plan {
  int C = 0, T = 0, nclusters = 0, smem = 0;
  std::vector<PlanCta> ctas;            // nclusters * C, cluster-major
  std::vector<int> cav_cluster;
  std::vector<int> slot_ptr, slot_idx;
  int nslots = 0;
};

int64_t align16(int64_t b) { return (b + 15) & ~int64_t(15); }

}  // namespace

struct fdtdbath_batch {
  int prec = 32;
  size_t esz = 4;
  double res = 0, courant = 0, dx = 0, dt = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;   // private stream for graph capture
  int device = 0;
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, void*) = nullptr;
  void* uctx = nullptr;
  std::vector<void*> allocs;
  size_t bytes_held = 0;
  std::vector<BCav> cavs;
  std::vector<HostMat> mats;
  int64_t ncell = 0, nyall = 0;
  // device state
  void* state = nullptr;       // E H P PM D psiE psiH bE cE bH cH (ncell each), Y0 Y1 (nyall each)
  size_t state_bytes = 0;
  void* snap = nullptr;        // autotuner snapshot of the state
  void* mats_d = nullptr;
  void* coef_d = nullptr;
  void* src_d = nullptr;
  long long* ctr = nullptr;
  // plan on the device
  Plan plan;
  bool planned = false;
  void *ctas_d = nullptr, *segs_d = nullptr, *runs_d = nullptr, *mslot_d = nullptr;
  void *slot_ptr_d = nullptr, *slot_idx_d = nullptr;
  size_t plan_cap[6] = {0, 0, 0, 0, 0, 0};
  int fixed_C = 0, fixed_T = 0;
  // energy
  bool energy_on = false;
  int every = 1;
  int64_t cap_rec = 0;
  int ring_cap = 1024;
  void* partial = nullptr;
  size_t partial_cap = 0;
  void* trace = nullptr;
  // driver
  bool use_graph = true;
  std::map<int, cudaGraphExec_t> graphs;
  int64_t n = 0, launches = 0, replays = 0;
  float tuned_ms = 0.f;
  std::string err;
};

namespace {

int bfail(fdtdbath_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  else g_batch_create_error = msg;
  return code;
}

int bcuda(fdtdbath_batch* b, cudaError_t e, const char* what) {
  return bfail(b, FDTDBATH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* balloc(fdtdbath_batch* b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (b->ualloc) p = b->ualloc(bytes, b->uctx);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (p) {
    b->allocs.push_back(p);
    b->bytes_held += bytes;
    cudaMemsetAsync(p, 0, bytes, b->stream);
  }
  return p;
}

void bfree(fdtdbath_batch* b, void* p) {
  if (!p) return;
  for (size_t i = 0; i < b->allocs.size(); ++i)
    if (b->allocs[i] == p) {
      b->allocs.erase(b->allocs.begin() + (long)i);
      break;
    }
  if (b->ufree) b->ufree(p, b->uctx);
  else cudaFree(p);
}

// Cut a cavity into pieces of uniform per-cell cost.
void make_pieces(const std::vector<HostMat>& mats, BCav& c, size_t esz, bool inc) {
  std::vector<int64_t> cuts = {0, c.nz};
  for (int m : c.mats) {
    cuts.push_back(mats[(size_t)m].zlo);
    cuts.push_back(mats[(size_t)m].zhi);
  }
  if (c.npml > 0) {
    cuts.push_back(c.npml);
    cuts.push_back(c.nz - c.npml);
    cuts.push_back(c.nz - c.npml - 1);
  }
  if (c.ehi > c.elo) {
    cuts.push_back(c.elo);
    cuts.push_back(c.ehi);
  }
  std::sort(cuts.begin(), cuts.end());
  cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
  c.pieces.clear();
  c.work = c.bytes = 0;
  for (size_t i = 0; i + 1 < cuts.size(); ++i) {
    const int64_t z0 = cuts[i], z1 = cuts[i + 1];
    if (z0 < 0 || z1 > c.nz || z0 >= z1) continue;
    Piece p{};
    p.z0 = z0;
    p.z1 = z1;
    p.mat = -1;
    for (int m : c.mats)
      if (z0 >= mats[(size_t)m].zlo && z0 < mats[(size_t)m].zhi) p.mat = m;
    const HostMat* M = p.mat >= 0 ? &mats[(size_t)p.mat] : nullptr;
    // cells outside every layer take the plain vacuum update; any layer (a vacuum-kind layer
    // still has its eps_inf) takes the D/E update with 1/eps_inf and its polarization
    p.kind = !M ? kRunVacuum : (M->kind == FDTDBATH_LORENTZ_BATH && M->nb > 0 ? kRunBath : kRunOsc);
    p.nb = p.kind == kRunBath ? M->nb : 0;
    p.psiE = c.npml > 0 && (z0 < c.npml || z0 >= c.nz - c.npml);
    p.psiH = c.npml > 0 && (z0 < c.npml || z0 >= c.nz - c.npml - 1);
    p.inbox = c.ehi > c.elo && z0 >= c.elo && z0 < c.ehi;
    p.work = kWorkVac + (p.psiE + p.psiH) * kWorkPsi + (p.kind == kRunOsc ? kWorkOsc : 0) +
             (p.kind == kRunBath ? kWorkBathBase + kWorkMode * p.nb : 0);
    p.bytes = (int64_t)esz * (2 + ((p.psiE || p.psiH) ? 6 : 0) + (p.kind != kRunVacuum ? (inc ? 2 : 3) : 0) +
                              2 * p.nb);
    c.work += p.work * (z1 - z0);
    c.bytes += p.bytes * (z1 - z0);
    c.pieces.push_back(p);
  }
}

struct FillState {
  int64_t work = 0, bytes = 0;
  int nseg = 0, nrun = 0, nmat = 0;
  int mats[kBatchMaxMat];
  int last_cav = -1;
  // per-thread work: cell l of a CTA belongs to thread l mod T (every phase deals the cells
  // round-robin and continues the deal across runs), so thread t carries the work of its cells;
  // stored as base + rel[t], the common part added in whole rounds of T cells
  int64_t ncell = 0, base = 0, relmax = 0;
  std::vector<int64_t> rel;
};

// Shared-memory bytes a CTA needs beyond its per-cell costs: alignment of its arrays and runs
// and the coefficient rows of its bath materials.
int64_t cta_fixed_bytes() { return 6 * 16; }
int64_t run_fixed_bytes() { return 2 * 32; }

// Places the largest k <= kmax of the next cells, each of work w, that keeps every thread of the
// CTA at or below W, and returns k.
int64_t thread_fit(FillState& f, int T, int64_t w, int64_t kmax, int64_t W) {
  if (kmax <= 0) return 0;
  const int64_t curmax = f.base + f.relmax;
  if (w == 0) {
    f.ncell += kmax;
    return kmax;
  }
  // whole rounds: every thread gets q cells; the q-th round must keep the fullest thread in bounds
  const int64_t qfit = W >= curmax ? (W - curmax) / w : 0;
  const int64_t q = std::min<int64_t>(qfit, kmax / T);
  // the partial round: the next r threads of the deal, while each stays in bounds
  const int64_t rlim = std::min<int64_t>(kmax - q * T, T - 1);
  const int s = (int)(f.ncell % T);
  int64_t r = 0;
  while (r < rlim && f.base + f.rel[(size_t)((s + r) % T)] + (q + 1) * w <= W) ++r;
  const int64_t k = q * T + r;
  if (k > 0) {
    f.base += q * w;
    for (int64_t i = 0; i < r; ++i) {
      int64_t& v = f.rel[(size_t)((s + i) % T)];
      v += w;
      f.relmax = std::max(f.relmax, v);
    }
    f.ncell += k;
  }
  return k;
}

// Greedy fill of the cavities `ids` (in order) into CTAs of T threads under a per-thread work
// bound W and byte budget cap.  Returns the number of CTAs used (> maxc: infeasible) and, if
// out != null, the cut list (cavity index in ids, z) where each CTA starts.  T = 1 bounds the
// whole CTA's work.
int greedy_fill(const std::vector<BCav>& cavs, const std::vector<HostMat>& mats, const std::vector<int>& ids,
                int64_t W, int64_t cap, size_t esz, int T, int maxc, std::vector<std::pair<int, int64_t>>* out) {
  FillState f;
  int used = 1;
  f.bytes = cta_fixed_bytes();
  f.rel.assign((size_t)T, 0);
  if (out) {
    out->clear();
    if (!ids.empty()) out->push_back({0, 0});
  }
  auto new_cta = [&](int ci, int64_t z) {
    ++used;
    std::vector<int64_t> rel;
    rel.swap(f.rel);
    f = FillState();
    f.rel.swap(rel);
    std::fill(f.rel.begin(), f.rel.end(), 0);
    f.bytes = cta_fixed_bytes();
    if (out) out->push_back({ci, z});
  };
  for (int ci = 0; ci < (int)ids.size(); ++ci) {
    const BCav& c = cavs[(size_t)ids[(size_t)ci]];
    for (const Piece& p : c.pieces) {
      int64_t z = p.z0;
      while (z < p.z1) {
        if (used > maxc) return used;
        // descriptor costs of placing cells of this piece in the current CTA
        const bool newseg = f.last_cav != ci;
        bool newmat = false;
        int64_t extra = run_fixed_bytes();
        if (p.mat >= 0 && p.kind != kRunVacuum) {
          newmat = true;
          for (int k = 0; k < f.nmat; ++k)
            if (f.mats[k] == p.mat) newmat = false;
          if (newmat) extra += (int64_t)esz * kCoefStride * mats[(size_t)p.mat].nb;
        }
        const bool room = f.nseg + (newseg ? 1 : 0) <= kBatchMaxSeg && f.nrun + 1 <= kBatchMaxRun &&
                          f.nmat + (newmat ? 1 : 0) <= kBatchMaxMat;
        int64_t k = p.z1 - z;
        if (room) {
          if (p.bytes > 0) k = std::min(k, (cap - f.bytes - extra) / p.bytes);
          k = thread_fit(f, T, p.work, k, W);
        } else {
          k = 0;
        }
        if (k <= 0) {
          if (f.ncell == 0 && f.nseg == 0) return maxc + 1;   // one cell does not fit an empty CTA
          new_cta(ci, z);
          continue;
        }
        f.work += k * p.work;
        f.bytes += k * p.bytes + extra;
        if (newseg) {
          ++f.nseg;
          f.last_cav = ci;
        }
        ++f.nrun;
        if (newmat) f.mats[f.nmat++] = p.mat;
        z += k;
      }
    }
  }
  return used;
}

// Pack the batch for shape (C, nclusters) under a per-CTA dynamic shared-memory budget.
int pack(const std::vector<BCav>& cavs, const std::vector<HostMat>& mats, size_t esz, bool inc, int C, int T,
         int nclusters, int64_t cap, Plan& plan, std::string& why) {
  const int ncav = (int)cavs.size();
  plan = Plan();
  plan.C = C;
  if (nclusters <= 0 || C <= 0) return why = "no cluster of this shape fits the device", FDTDBATH_ERR_UNSUPPORTED;
  nclusters = std::min(nclusters, ncav);
  plan.nclusters = nclusters;
  // longest processing time first, with a shared-memory guard
  std::vector<int> order((size_t)ncav);
  for (int i = 0; i < ncav; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cavs[(size_t)a].work > cavs[(size_t)b].work; });
  std::vector<int64_t> cw((size_t)nclusters, 0), cb((size_t)nclusters, 0);
  std::vector<std::vector<int>> members((size_t)nclusters);
  const int64_t ccap = (int64_t)C * (cap - cta_fixed_bytes()) * 9 / 10;
  plan.cav_cluster.assign((size_t)ncav, -1);
  for (int i : order) {
    int best = -1;
    for (int k = 0; k < nclusters; ++k) {
      if (cb[(size_t)k] + cavs[(size_t)i].bytes > ccap && !members[(size_t)k].empty()) continue;
      if (best < 0 || cw[(size_t)k] < cw[(size_t)best]) best = k;
    }
    if (best < 0) return why = "the cavities do not fit the shared memory of this launch shape", FDTDBATH_ERR_UNSUPPORTED;
    members[(size_t)best].push_back(i);
    cw[(size_t)best] += cavs[(size_t)i].work;
    cb[(size_t)best] += cavs[(size_t)i].bytes;
    plan.cav_cluster[(size_t)i] = best;
  }
  // per cluster: the smallest work bound that fits C CTAs
  plan.ctas.assign((size_t)nclusters * C, PlanCta());
  std::vector<std::vector<int>> cav_slots((size_t)ncav);
  int slot = 0;
  for (int k = 0; k < nclusters; ++k) {
    std::vector<int>& ids = members[(size_t)k];
    std::sort(ids.begin(), ids.end());
    int64_t tot = 0, maxw = 0;
    for (int i : ids) {
      tot += cavs[(size_t)i].work;
      for (const Piece& p : cavs[(size_t)i].pieces) maxw = std::max(maxw, p.work);
    }
    // bound on the work of one thread: at least an even share of the cluster and one cell
    int64_t lo = std::max<int64_t>((tot + (int64_t)C * T - 1) / ((int64_t)C * T), maxw), hi = std::max<int64_t>(tot, lo);
    if (greedy_fill(cavs, mats, ids, hi, cap, esz, T, C, nullptr) > C)
      return why = "a cluster's cavities do not fit its CTAs' shared memory", FDTDBATH_ERR_UNSUPPORTED;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (greedy_fill(cavs, mats, ids, mid, cap, esz, T, C, nullptr) <= C) hi = mid;
      else lo = mid + 1;
    }
    std::vector<std::pair<int, int64_t>> starts;
    greedy_fill(cavs, mats, ids, lo, cap, esz, T, C, &starts);
    // build the CTAs: CTA r holds cells from starts[r] up to starts[r+1]
    for (int r = 0; r < C; ++r) {
      PlanCta& pc = plan.ctas[(size_t)k * C + r];
      if (r >= (int)starts.size()) continue;
      const int ci0 = starts[(size_t)r].first;
      const int64_t z0 = starts[(size_t)r].second;
      const int ci1 = r + 1 < (int)starts.size() ? starts[(size_t)r + 1].first : (int)ids.size();
      const int64_t z1 = r + 1 < (int)starts.size() ? starts[(size_t)r + 1].second : 0;
      int l = 0;
      for (int ci = ci0; ci <= ci1 && ci < (int)ids.size(); ++ci) {
        const BCav& c = cavs[(size_t)ids[(size_t)ci]];
        const int64_t a = ci == ci0 ? z0 : 0;
        const int64_t e = ci == ci1 ? z1 : c.nz;
        if (e <= a) continue;
        BatchSeg g{};
        g.cav = ids[(size_t)ci];
        g.z0 = (int)a;
        g.z1 = (int)e;
        g.l0 = l;
        g.l1 = l + (int)(e - a);
        g.link_left = a > 0;
        g.link_right = e < c.nz;
        g.src_l = (c.src_z >= a && c.src_z < e) ? l + (int)(c.src_z - a) : -1;
        g.slot = slot;
        cav_slots[(size_t)g.cav].push_back(slot);
        ++slot;
        g.g0 = c.off + a;
        g.src_off = c.src_off;
        g.src_len = c.src_len;
        const int segi = (int)pc.segs.size();
        for (const Piece& p : c.pieces) {
          const int64_t pa = std::max(p.z0, a), pe = std::min(p.z1, e);
          if (pe <= pa) continue;
          BatchRun R{};
          R.l0 = l + (int)(pa - a);
          R.l1 = l + (int)(pe - a);
          R.kind = p.kind;
          R.seg = segi;
          R.inbox = p.inbox;
          R.psiE = p.psiE;
          R.psiH = p.psiH;
          R.nb = p.nb;
          R.mslot = -1;
          if (p.kind != kRunVacuum) {
            int s = -1;
            for (int q = 0; q < (int)pc.mslots.size(); ++q)
              if (pc.mslots[(size_t)q] == p.mat) s = q;
            if (s < 0) {
              s = (int)pc.mslots.size();
              pc.mslots.push_back(p.mat);
            }
            R.mslot = s;
          }
          pc.runs.push_back(R);
          pc.work += p.work * (pe - pa);
        }
        pc.segs.push_back(g);
        l += (int)(e - a);
      }
      pc.d.ncell = l;
    }
  }
  // slots of every cavity, in CTA order
  plan.nslots = slot;
  plan.slot_ptr.assign((size_t)ncav + 1, 0);
  for (int i = 0; i < ncav; ++i) {
    plan.slot_ptr[(size_t)i + 1] = plan.slot_ptr[(size_t)i] + (int)cav_slots[(size_t)i].size();
    for (int s : cav_slots[(size_t)i]) plan.slot_idx.push_back(s);
  }
  // shared-memory layout of every CTA
  int maxsmem = 16;
  for (size_t r = 0; r < plan.ctas.size(); ++r) {
    PlanCta& pc = plan.ctas[r];
    BatchCta& d = pc.d;
    d.nseg = (int)pc.segs.size();
    d.nrun = (int)pc.runs.size();
    d.nmat = (int)pc.mslots.size();
    if (d.nseg > kBatchMaxSeg || d.nrun > kBatchMaxRun || d.nmat > kBatchMaxMat)
      return why = "CTA descriptor limits exceeded", FDTDBATH_ERR_UNSUPPORTED;
    int npsi = 0;
    for (auto& R : pc.runs)
      if (R.psiE || R.psiH) {
        R.psi0 = npsi;
        npsi += R.l1 - R.l0;
      }
    d.npsi = npsi;
    int rows = 0;
    for (int m : pc.mslots) rows += mats[(size_t)m].kind == FDTDBATH_LORENTZ_BATH ? mats[(size_t)m].nb : 0;
    d.coef_rows = rows;
    int64_t off = 0;
    d.off_E = 0;   // the next CTA's E_x is read at offset 0 of its shared memory
    off = align16(off + (int64_t)esz * d.ncell);
    d.off_H = (int)off;
    off = align16(off + (int64_t)esz * d.ncell);
    d.off_psi = (int)off;
    off = align16(off + (int64_t)esz * 6 * npsi);
    d.off_coef = (int)off;
    off = align16(off + (int64_t)esz * kCoefStride * rows);
    d.off_P = (int)off;
    int64_t el = 0;   // element offsets inside the P/Y area, 16-byte aligned
    const int64_t al = 16 / (int64_t)esz;
    for (auto& R : pc.runs) {
      const int len = R.l1 - R.l0;
      if (R.kind != kRunVacuum) {
        R.p0 = (int)el;
        el += (inc ? 2 : 3) * (int64_t)len;
        el = (el + al - 1) / al * al;
      }
      if (R.kind == kRunBath) {
        R.y0 = (int)el;
        el += 2 * (int64_t)R.nb * len;
        el = (el + al - 1) / al * al;
      }
    }
    off += el * (int64_t)esz;
    d.smem_bytes = (int)align16(off);
    if (d.smem_bytes > cap) return why = "a CTA exceeds its shared-memory budget", FDTDBATH_ERR_UNSUPPORTED;
    maxsmem = std::max(maxsmem, d.smem_bytes);
    d.prev_ncell = (r % (size_t)C) ? plan.ctas[r - 1].d.ncell : 0;
    d.prev_off_H = (r % (size_t)C) ? plan.ctas[r - 1].d.off_H : 0;
  }
  plan.smem = maxsmem;
  // global descriptor offsets
  int s0 = 0, r0 = 0, m0 = 0;
  for (auto& pc : plan.ctas) {
    pc.d.seg0 = s0;
    pc.d.run0 = r0;
    pc.d.mat0 = m0;
    s0 += pc.d.nseg;
    r0 += pc.d.nrun;
    m0 += pc.d.nmat;
  }
  return 0;
}

// Validate the cavities and fill b->cavs / b->mats (no device work).
int build_cavities(fdtdbath_batch* b, const fdtdbath_cavity* cavities, int ncav, std::string& why) {
  if (ncav < 1 || !cavities) return why = "need at least one cavity", FDTDBATH_ERR_ARG;
  int64_t off = 0, yb = 0, srcoff = 0;
  b->cavs.clear();
  b->mats.clear();
  for (int i = 0; i < ncav; ++i) {
    const fdtdbath_cavity& cv = cavities[i];
    BCav c{};
    c.nz = cv.nz;
    c.npml = cv.pml_cells;
    c.off = off;
    c.src_z = -1;
    char buf[96];
    std::snprintf(buf, sizeof buf, "cavity %d: ", i);
    const std::string pre(buf);
    if (cv.nz < 64 || cv.nz > (1 << 24)) return why = pre + "nz must be in [64, 2^24]", FDTDBATH_ERR_ARG;
    if (cv.pml_cells < 0 || 2 * (int64_t)cv.pml_cells + 2 > cv.nz) return why = pre + "bad pml_cells", FDTDBATH_ERR_ARG;
    if (cv.nmat < 0 || cv.nmat > kMaxMat || (cv.nmat && !cv.materials)) return why = pre + "bad material list", FDTDBATH_ERR_ARG;
    std::vector<int> order((size_t)cv.nmat);
    for (int m = 0; m < cv.nmat; ++m) order[(size_t)m] = m;
    std::sort(order.begin(), order.end(), [&](int a, int c2) { return cv.materials[a].z_lo < cv.materials[c2].z_lo; });
    int64_t prev_hi = 0;
    for (int m : order) {
      const fdtdbath_material& M = cv.materials[m];
      if (M.z_lo < 0 || M.z_hi > cv.nz || M.z_lo >= M.z_hi) return why = pre + "material z-range outside the cavity", FDTDBATH_ERR_ARG;
      if (M.z_lo < prev_hi) return why = pre + "material layers overlap", FDTDBATH_ERR_ARG;
      prev_hi = M.z_hi;
      HostMat h{};
      std::string w;
      const int rc = build_material(M, 1, b->dt, b->courant, 1, h, w);
      if (rc) return why = pre + w, rc;
      if (h.nb > kMaxBathStep) return why = pre + "the batch holds at most 128 bath modes per material", FDTDBATH_ERR_ARG;
      h.base = 0;
      h.ybase = yb;
      yb += (int64_t)h.nb * h.ncell;
      c.mats.push_back((int)b->mats.size());
      b->mats.push_back(h);
    }
    c.elo = cv.energy_lo;
    c.ehi = cv.energy_hi;
    if (c.ehi > c.elo && (c.elo < 0 || c.ehi > c.nz)) return why = pre + "energy box outside the cavity", FDTDBATH_ERR_ARG;
    if (cv.source) {
      const fdtdbath_source& S = *cv.source;
      if (S.component != 0) return why = pre + "the batched form advances E_x: the source must be on component 0", FDTDBATH_ERR_ARG;
      if (S.z < 0 || S.z >= cv.nz) return why = pre + "source outside the cavity", FDTDBATH_ERR_ARG;
      if (!(S.fwidth > 0)) return why = pre + "source fwidth must be positive", FDTDBATH_ERR_ARG;
      c.src_z = S.z;
      c.amp = S.amplitude;
      c.nu = S.center;
      c.fwidth = S.fwidth;
      c.t0 = S.t0;
      c.phase = S.phase ? S.phase[0] : 0.0;
      c.src_off = srcoff;
      // amplitudes until the Gaussian envelope underflows to exactly zero (it then stays zero)
      const double tau = 1.0 / (2.0 * M_PI * c.fwidth);
      int64_t len = 0;
      for (int64_t nn = 0; nn < (int64_t)1 << 26; ++nn) {
        const double t = (double)nn * b->dt;
        const double u = t - c.t0;
        if (u > 0 && std::exp(-u * u / (2.0 * tau * tau)) == 0.0) break;
        len = nn + 1;
      }
      c.src_len = (int)len;
      srcoff += len;
    }
    off += c.nz;
    b->cavs.push_back(c);
  }
  b->ncell = off;
  b->nyall = yb;
  if (off > ((int64_t)1 << 31) - 1 || yb > ((int64_t)1 << 31) - 1)
    return why = "batch state above 2^31 elements", FDTDBATH_ERR_ARG;
  for (auto& c : b->cavs) make_pieces(b->mats, c, b->esz, b->prec == 32);
  return 0;
}

template <typename T>
BatchParams<T> batch_params(fdtdbath_batch* b, int nsteps, int energy) {
  BatchParams<T> p{};
  p.ctr = b->ctr;
  p.nsteps = nsteps;
  p.S = (T)(b->dt / b->dx);
  p.dt = (T)b->dt;
  p.ctas = (const BatchCta*)b->ctas_d;
  p.segs = (const BatchSeg*)b->segs_d;
  p.runs = (const BatchRun*)b->runs_d;
  p.matslot = (const int*)b->mslot_d;
  p.mats = (const MatK<T>*)b->mats_d;
  p.coef = (const T*)b->coef_d;
  T* s = (T*)b->state;
  const int64_t n = b->ncell;
  p.E = s;
  p.H = s + n;
  p.P = s + 2 * n;
  p.PM = s + 3 * n;
  p.D = s + 4 * n;
  p.psiE = s + 5 * n;
  p.psiH = s + 6 * n;
  p.bE = s + 7 * n;
  p.cE = s + 8 * n;
  p.bH = s + 9 * n;
  p.cH = s + 10 * n;
  p.Y0 = s + 11 * n;
  p.Y1 = s + 11 * n + b->nyall;
  p.src_tab = (const double*)b->src_d;
  p.energy_on = energy;
  p.every = b->every;
  p.ring_cap = b->ring_cap;
  p.ring_stride = 4 * (int64_t)std::max(1, b->plan.nslots);
  p.partial = (double*)b->partial;
  return p;
}

int launch_kernel(fdtdbath_batch* b, int nsteps, int energy, cudaStream_t st) {
  const Plan& P = b->plan;
  int rc;
  if (b->prec == 32)
    rc = launch_batch1d_f32(batch_params<float>(b, nsteps, energy), (int)P.ctas.size(), P.C, P.T, P.smem, st);
  else
    rc = launch_batch1d_f64(batch_params<double>(b, nsteps, energy), (int)P.ctas.size(), P.C, P.T, P.smem, st);
  if (rc) return bcuda(b, (cudaError_t)rc, "batch kernel launch");
  return 0;
}

int upload(fdtdbath_batch* b, void** dst, size_t* capb, const void* src, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (*capb < bytes) {
    bfree(b, *dst);
    *dst = balloc(b, bytes);
    if (!*dst) return bfail(b, FDTDBATH_ERR_OOM, "device allocation failed");
    *capb = bytes;
  }
  if (src) {
    cudaError_t e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "plan upload");
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "plan upload");
  }
  return 0;
}

void drop_graphs(fdtdbath_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
}

int install_plan(fdtdbath_batch* b, Plan&& plan) {
  drop_graphs(b);
  b->plan = std::move(plan);
  Plan& P = b->plan;
  std::vector<BatchCta> ctas;
  std::vector<BatchSeg> segs;
  std::vector<BatchRun> runs;
  std::vector<int> ms;
  for (auto& pc : P.ctas) {
    ctas.push_back(pc.d);
    segs.insert(segs.end(), pc.segs.begin(), pc.segs.end());
    runs.insert(runs.end(), pc.runs.begin(), pc.runs.end());
    ms.insert(ms.end(), pc.mslots.begin(), pc.mslots.end());
  }
  int rc;
  if ((rc = upload(b, &b->ctas_d, &b->plan_cap[0], ctas.data(), ctas.size() * sizeof(BatchCta)))) return rc;
  if ((rc = upload(b, &b->segs_d, &b->plan_cap[1], segs.data(), segs.size() * sizeof(BatchSeg)))) return rc;
  if ((rc = upload(b, &b->runs_d, &b->plan_cap[2], runs.data(), runs.size() * sizeof(BatchRun)))) return rc;
  if ((rc = upload(b, &b->mslot_d, &b->plan_cap[3], ms.data(), ms.size() * sizeof(int)))) return rc;
  if ((rc = upload(b, &b->slot_ptr_d, &b->plan_cap[4], P.slot_ptr.data(), P.slot_ptr.size() * sizeof(int)))) return rc;
  if ((rc = upload(b, &b->slot_idx_d, &b->plan_cap[5], P.slot_idx.data(), P.slot_idx.size() * sizeof(int)))) return rc;
  const size_t need = (size_t)b->ring_cap * 4 * (size_t)std::max(1, P.nslots) * sizeof(double);
  if (b->partial_cap < need) {
    bfree(b, b->partial);
    b->partial = balloc(b, need);
    if (!b->partial) return bfail(b, FDTDBATH_ERR_OOM, "device allocation failed");
    b->partial_cap = need;
  }
  b->planned = true;
  return 0;
}

// Plan for one launch shape on this device: occupancy-limited cluster count, then the packer.
int plan_shape(fdtdbath_batch* b, int C, int T, int ctas_per_sm, Plan& out, std::string& why) {
  int maxc = 0, stat = 0;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, b->device);
  if (e != cudaSuccess) return why = cudaGetErrorString(e), FDTDBATH_ERR_CUDA;
  const int64_t per_sm = (int64_t)prop.sharedMemPerMultiprocessor;
  int rc = batch1d_occupancy(b->prec, C, T, 16, &maxc, &stat);
  if (rc) return why = cudaGetErrorString((cudaError_t)rc), FDTDBATH_ERR_CUDA;
  int64_t cap = per_sm / ctas_per_sm - stat - 1024;
  cap = std::min<int64_t>(cap, (int64_t)prop.sharedMemPerBlockOptin - stat);
  cap &= ~int64_t(15);
  if (cap <= 1024) return why = "no shared memory left", FDTDBATH_ERR_UNSUPPORTED;
  rc = batch1d_occupancy(b->prec, C, T, (int)cap, &maxc, &stat);
  if (rc) return why = cudaGetErrorString((cudaError_t)rc), FDTDBATH_ERR_CUDA;
  if (maxc <= 0) return why = "launch shape cannot be resident", FDTDBATH_ERR_UNSUPPORTED;
  rc = pack(b->cavs, b->mats, b->esz, b->prec == 32, C, T, maxc, cap, out, why);
  if (rc) return rc;
  out.T = T;
  return 0;
}

int timed_probe(fdtdbath_batch* b, int steps, float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = launch_kernel(b, 8, b->energy_on, b->stream);   // warm-up
  if (!rc) {
    cudaEventRecord(e0, b->stream);
    rc = launch_kernel(b, steps, b->energy_on, b->stream);
    cudaEventRecord(e1, b->stream);
  }
  cudaError_t e = cudaEventSynchronize(e1);
  if (!rc && e != cudaSuccess) rc = bcuda(b, e, "autotune probe");
  if (!rc) cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int autotune(fdtdbath_batch* b, int probe_steps) {
  // the probes advance the state: keep a snapshot and put it back afterwards
  if (!b->snap) {
    b->snap = balloc(b, b->state_bytes);
    if (!b->snap) return bfail(b, FDTDBATH_ERR_OOM, "device allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(b->snap, b->state, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "autotune snapshot");
  float best = 1e30f;
  Plan bestp;
  bool found = false;
  std::string last;
  const char* ev = std::getenv("FDTDBATH_TUNE_VERBOSE");   // print every candidate's time
  const bool verbose = ev && *ev && *ev != '0';
  const int Cs[] = {1, 2, 4, 8, 16};
  // thread counts between the powers of two too: a Lorentz-Bath run's cells are dealt round-robin,
  // so the count decides how evenly its remainder spreads over the threads
  const int Ts[] = {128, 256, 384, 512, 640, 768, 896, 1024};
  for (int C : Cs)
    for (int T : Ts)
      for (int k = 1; k <= 2; ++k) {
        if (b->fixed_C && C != b->fixed_C) continue;
        if (b->fixed_T && T != b->fixed_T) continue;
        Plan P;
        std::string why;
        if (plan_shape(b, C, T, k, P, why)) {
          last = why;
          continue;
        }
        Plan keep = P;
        int rc = install_plan(b, std::move(P));
        if (rc) return rc;
        float ms = 0.f;
        rc = timed_probe(b, probe_steps, &ms);
        if (rc) return rc;
        if (verbose)
          std::fprintf(stderr, "fdtdbath batch autotune: C=%d T=%d ctas/SM=%d clusters=%d smem=%d: %.4f ms/step\n", C, T,
                       k, b->plan.nclusters, b->plan.smem, ms / (float)probe_steps);
        if (ms < best) {
          best = ms;
          bestp = std::move(keep);
          found = true;
        }
      }
  e = cudaMemcpyAsync(b->state, b->snap, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "autotune restore");
  if (!found) return bfail(b, FDTDBATH_ERR_UNSUPPORTED, "no launch shape fits this batch: " + last);
  b->tuned_ms = best / (float)probe_steps;
  return install_plan(b, std::move(bestp));
}

int run_chunk(fdtdbath_batch* b, int m, cudaStream_t st) {
  int rc = launch_kernel(b, m, b->energy_on, st);
  if (rc) return rc;
  if (b->energy_on) {
    BatchReduceParams r{};
    r.ctr = b->ctr;
    r.nsteps = m;
    r.every = b->every;
    r.ring_cap = b->ring_cap;
    r.ring_stride = 4 * (int64_t)std::max(1, b->plan.nslots);
    r.partial = (const double*)b->partial;
    r.slot_ptr = (const int*)b->slot_ptr_d;
    r.slot_idx = (const int*)b->slot_idx_d;
    r.ncav = (int)b->cavs.size();
    r.trace = (double*)b->trace;
    r.trace_cap = b->cap_rec;
    r.ew = b->dx;
    rc = launch_batch_reduce(r, st);
    if (rc) return bcuda(b, (cudaError_t)rc, "batch reduce launch");
  }
  rc = launch_batch_advance(b->ctr, m, st);
  if (rc) return bcuda(b, (cudaError_t)rc, "batch counter launch");
  return 0;
}

int graph_for(fdtdbath_batch* b, int m, cudaGraphExec_t* out) {
  auto it = b->graphs.find(m);
  if (it != b->graphs.end()) {
    *out = it->second;
    return 0;
  }
  if (!b->cap) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bcuda(b, e, "capture stream");
  }
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamBeginCapture");
  int rc = run_chunk(b, m, b->cap);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
  if (b->graphs.size() >= 4) drop_graphs(b);
  b->graphs[m] = x;
  *out = x;
  return 0;
}

}  // namespace

extern "C" {

int fdtdbath_batch_create(const fdtdbath_cavity* cavities, int32_t ncav, double resolution, double courant,
                          const fdtdbath_batch_options* opt, fdtdbath_batch** out) {
  g_batch_create_error.clear();
  if (!out || !opt) return bfail(nullptr, FDTDBATH_ERR_ARG, "null argument");
  *out = nullptr;
  if (opt->precision != 32 && opt->precision != 64) return bfail(nullptr, FDTDBATH_ERR_ARG, "precision must be 32 or 64");
  if (!(resolution > 0)) return bfail(nullptr, FDTDBATH_ERR_ARG, "resolution must be positive");
  if (!(courant > 0) || courant > 1.0) return bfail(nullptr, FDTDBATH_ERR_CFL, "Courant number must be in (0, 1] in 1D");
  if (opt->energy_every < 0) return bfail(nullptr, FDTDBATH_ERR_ARG, "energy_every must be >= 0");
  if (opt->cluster_ctas < 0 || opt->cluster_ctas > kBatchMaxCluster || opt->block_threads < 0 ||
      opt->block_threads > kBatchMaxThreads || opt->block_threads % 32)
    return bfail(nullptr, FDTDBATH_ERR_ARG, "bad launch shape (cluster 0..16 CTAs, threads a multiple of 32 up to 1024)");
  if ((opt->alloc == nullptr) != (opt->free == nullptr))
    return bfail(nullptr, FDTDBATH_ERR_ARG, "alloc and free must both be set or both NULL");
  fdtdbath_batch* b = new fdtdbath_batch();
  b->prec = opt->precision;
  b->esz = b->prec == 64 ? 8 : 4;
  b->res = resolution;
  b->courant = courant;
  b->dx = 1.0 / resolution;
  b->dt = courant * b->dx;
  b->stream = (cudaStream_t)opt->cuda_stream;
  b->device = opt->device;
  b->ualloc = opt->alloc;
  b->ufree = opt->free;
  b->uctx = opt->alloc_ctx;
  b->fixed_C = opt->cluster_ctas;
  b->fixed_T = opt->block_threads;
  b->use_graph = opt->use_graph != 0;
  auto bail = [&](int code, const std::string& msg) {
    fdtdbath_batch_destroy(b);
    g_batch_create_error = msg;
    return code;
  };
  std::string why;
  int rc = build_cavities(b, cavities, ncav, why);
  if (rc) return bail(rc, why);
  for (auto& c : b->cavs)
    if (c.ehi > c.elo) b->energy_on = true;
  b->every = std::max(1, opt->energy_every);
  b->cap_rec = opt->energy_capacity > 0 ? opt->energy_capacity : 65536;
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bail(FDTDBATH_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  // ---- device state ----
  b->state_bytes = b->esz * (size_t)(11 * b->ncell + 2 * b->nyall);
  b->state = balloc(b, b->state_bytes);
  b->ctr = (long long*)balloc(b, sizeof(long long));
  if (!b->state || !b->ctr) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  // CPML coefficients, material table and coefficient rows, source tables
  {
    std::vector<double> bE((size_t)b->ncell, 1.0), cE((size_t)b->ncell, 0.0), bH((size_t)b->ncell, 1.0),
        cH((size_t)b->ncell, 0.0);
    for (auto& c : b->cavs)
      for (int64_t z = 0; z < c.nz; ++z) {
        const size_t g = (size_t)(c.off + z);
        cpml_coeffs(c.npml, c.nz, b->dx, b->dt, (double)z, &bE[g], &cE[g]);
        cpml_coeffs(c.npml, c.nz, b->dx, b->dt, (double)z + 0.5, &bH[g], &cH[g]);
      }
    std::vector<double> rows;
    std::vector<int> coef_off;
    for (auto& m : b->mats) {
      coef_off.push_back((int)(rows.size() / kCoefStride));
      const auto& src = b->prec == 64 ? m.rowsLit : m.rowsInc;
      rows.insert(rows.end(), src.begin(), src.end());
    }
    if (rows.empty()) rows.assign(kCoefStride, 0.0);
    std::vector<double> tab;
    for (auto& c : b->cavs) {
      if (c.src_z < 0) continue;
      const double tau = 1.0 / (2.0 * M_PI * c.fwidth);
      for (int64_t nn = 0; nn < c.src_len; ++nn) {
        const double t = (double)nn * b->dt;
        const double u = t - c.t0;
        tab.push_back(c.amp * std::exp(-u * u / (2.0 * tau * tau)) * std::sin(2.0 * M_PI * c.nu * u + c.phase));
      }
    }
    if (tab.empty()) tab.push_back(0.0);
    b->src_d = balloc(b, tab.size() * sizeof(double));
    if (!b->src_d) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
    e = cudaMemcpyAsync(b->src_d, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bail(FDTDBATH_ERR_CUDA, "source table upload");
    const int64_t n = b->ncell;
    auto put = [&](int64_t at, const std::vector<double>& v) -> cudaError_t {
      if (b->prec == 64)
        return cudaMemcpyAsync((double*)b->state + at, v.data(), v.size() * 8, cudaMemcpyHostToDevice, b->stream);
      std::vector<float> f(v.size());
      for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
      cudaError_t r = cudaMemcpyAsync((float*)b->state + at, f.data(), f.size() * 4, cudaMemcpyHostToDevice, b->stream);
      if (r == cudaSuccess) r = cudaStreamSynchronize(b->stream);
      return r;
    };
    if ((e = put(7 * n, bE)) != cudaSuccess || (e = put(8 * n, cE)) != cudaSuccess ||
        (e = put(9 * n, bH)) != cudaSuccess || (e = put(10 * n, cH)) != cudaSuccess)
      return bail(FDTDBATH_ERR_CUDA, std::string("CPML upload: ") + cudaGetErrorString(e));
    // coefficient rows in the state precision, material table
    b->coef_d = balloc(b, rows.size() * b->esz);
    b->mats_d = balloc(b, b->mats.size() * (b->prec == 64 ? sizeof(MatK<double>) : sizeof(MatK<float>)) + 16);
    if (!b->coef_d || !b->mats_d) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
    if (b->prec == 64) {
      std::vector<MatK<double>> mk;
      for (size_t m = 0; m < b->mats.size(); ++m) mk.push_back(mat_k<double>(b->mats[m], coef_off[m], b->dt));
      e = cudaMemcpyAsync(b->coef_d, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess && !mk.empty())
        e = cudaMemcpyAsync(b->mats_d, mk.data(), mk.size() * sizeof(MatK<double>), cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    } else {
      std::vector<MatK<float>> mk;
      for (size_t m = 0; m < b->mats.size(); ++m) mk.push_back(mat_k<float>(b->mats[m], coef_off[m], b->dt));
      std::vector<float> rf(rows.size());
      for (size_t i = 0; i < rows.size(); ++i) rf[i] = (float)rows[i];
      e = cudaMemcpyAsync(b->coef_d, rf.data(), rf.size() * 4, cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess && !mk.empty())
        e = cudaMemcpyAsync(b->mats_d, mk.data(), mk.size() * sizeof(MatK<float>), cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) return bail(FDTDBATH_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
  }
  if (b->energy_on) {
    b->trace = balloc(b, (size_t)b->cavs.size() * (size_t)b->cap_rec * 4 * sizeof(double));
    if (!b->trace) return bail(FDTDBATH_ERR_OOM, "device allocation failed");
  }
  e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bail(FDTDBATH_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
  // a fixed launch shape is planned now; otherwise the first step runs the autotuner
  if (b->fixed_C && b->fixed_T) {
    Plan P;
    rc = plan_shape(b, b->fixed_C, b->fixed_T, 1, P, why);
    if (rc) return bail(rc, why);
    rc = install_plan(b, std::move(P));
    if (rc) return bail(rc, b->err);
  }
  *out = b;
  return 0;
}

int fdtdbath_batch_autotune(fdtdbath_batch* b, int32_t probe_steps, int32_t* cluster_ctas, int32_t* block_threads,
                            float* ms_per_step) {
  if (!b) return FDTDBATH_ERR_ARG;
  if (probe_steps < 1) return bfail(b, FDTDBATH_ERR_ARG, "probe_steps must be >= 1");
  cudaSetDevice(b->device);
  int rc = autotune(b, probe_steps);
  if (rc) return rc;
  if (cluster_ctas) *cluster_ctas = b->plan.C;
  if (block_threads) *block_threads = b->plan.T;
  if (ms_per_step) *ms_per_step = b->tuned_ms;
  return 0;
}

int fdtdbath_batch_step(fdtdbath_batch* b, int64_t nsteps) {
  if (!b) return FDTDBATH_ERR_ARG;
  if (nsteps < 0) return bfail(b, FDTDBATH_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return 0;
  cudaSetDevice(b->device);
  int rc;
  if (!b->planned && (rc = autotune(b, 64))) return rc;
  const int64_t chunk = b->energy_on ? (int64_t)b->ring_cap * b->every : 4096;
  while (nsteps > 0) {
    const int m = (int)std::min<int64_t>(nsteps, chunk);
    if (b->use_graph) {
      cudaGraphExec_t x;
      if ((rc = graph_for(b, m, &x))) return rc;
      cudaError_t e = cudaGraphLaunch(x, b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
      ++b->replays;
    } else if ((rc = run_chunk(b, m, b->stream))) {
      return rc;
    }
    b->launches += b->energy_on ? 3 : 2;
    b->n += m;
    nsteps -= m;
  }
  return 0;
}

int fdtdbath_batch_sync(fdtdbath_batch* b) {
  if (!b) return FDTDBATH_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
  return 0;
}

int fdtdbath_batch_read_field(fdtdbath_batch* b, int32_t cavity, int32_t field, void* dst, size_t dst_bytes) {
  if (!b || !dst) return FDTDBATH_ERR_ARG;
  if (cavity < 0 || cavity >= (int)b->cavs.size()) return bfail(b, FDTDBATH_ERR_ARG, "cavity index out of range");
  const BCav& c = b->cavs[(size_t)cavity];
  if (dst_bytes < (size_t)c.nz * b->esz) return bfail(b, FDTDBATH_ERR_ARG, "destination too small");
  cudaSetDevice(b->device);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
  const int64_t n = b->ncell;
  char* base = (char*)b->state;
  int64_t arr = -1;
  if (field == FDTDBATH_FIELD_E(0)) arr = 0;
  else if (field == FDTDBATH_FIELD_H(1)) arr = 1;
  else if (field == FDTDBATH_FIELD_P(0)) arr = 2;
  else if (field == FDTDBATH_FIELD_PM(0)) arr = 3;
  if (arr >= 0) {
    e = cudaMemcpy(dst, base + b->esz * (size_t)(arr * n + c.off), (size_t)c.nz * b->esz, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "read");
    return 0;
  }
  if (field >= FDTDBATH_FIELD_Y(0, 0, 0) && field < FDTDBATH_FIELD_Y(0, 0, 2)) {
    const int lev = (field - FDTDBATH_FIELD_Y(0, 0, 0)) / 256, j = (field - FDTDBATH_FIELD_Y(0, 0, 0)) % 256;
    std::memset(dst, 0, (size_t)c.nz * b->esz);
    for (int m : c.mats) {
      const HostMat& M = b->mats[(size_t)m];
      if (M.kind != FDTDBATH_LORENTZ_BATH || j >= M.nb) continue;
      const size_t at = (size_t)(11 * n + lev * b->nyall + M.ybase + (int64_t)j * M.ncell);
      e = cudaMemcpy((char*)dst + b->esz * (size_t)M.zlo, base + b->esz * at, (size_t)M.ncell * b->esz,
                     cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return bcuda(b, e, "read");
    }
    return 0;
  }
  return bfail(b, FDTDBATH_ERR_ARG, "the batched form holds E_x, H_y, P_x, PM_x and the x bath modes only");
}

int fdtdbath_batch_energy(fdtdbath_batch* b, int32_t cavity, double* trace, int64_t maxlen, int64_t* len) {
  if (!b || !len) return FDTDBATH_ERR_ARG;
  if (cavity < 0 || cavity >= (int)b->cavs.size()) return bfail(b, FDTDBATH_ERR_ARG, "cavity index out of range");
  *len = 0;
  if (!b->energy_on) return 0;
  cudaSetDevice(b->device);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
  int64_t have = (b->n + b->every - 1) / b->every;
  have = std::min(have, b->cap_rec);
  const int64_t k = std::min(have, maxlen);
  if (k > 0 && trace) {
    e = cudaMemcpy(trace, (double*)b->trace + (size_t)cavity * (size_t)b->cap_rec * 4, (size_t)k * 4 * sizeof(double),
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "energy read");
  }
  *len = k;
  return 0;
}

int64_t fdtdbath_batch_query(const fdtdbath_batch* b, int32_t key) {
  if (!b) return -1;
  switch (key) {
    case 0: return b->launches;
    case 1: return b->plan.nclusters;
    case 2: return (int64_t)b->plan.ctas.size();
    case 3: return b->plan.C;
    case 4: return b->plan.T;
    case 5: return (int64_t)b->bytes_held;
    case 6: return b->replays;
    case 7: return b->n;
    case 8: return b->plan.smem;
    case 9: return b->ncell;
    default: return -1;
  }
}

const char* fdtdbath_batch_last_error(const fdtdbath_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

void fdtdbath_batch_destroy(fdtdbath_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (void* p : b->allocs) {
    if (b->ufree) b->ufree(p, b->uctx);
    else cudaFree(p);
  }
  delete b;
}

int fdtdbath_batch_plan(const fdtdbath_cavity* cavities, int32_t ncav, double resolution, double courant,
                        int32_t precision, int32_t cluster_ctas, int32_t block_threads, int32_t nclusters,
                        int32_t smem_per_cta, int64_t* cta_work, int32_t* cta_ncell, int32_t* cta_smem,
                        int32_t* cav_cluster) {
  g_batch_create_error.clear();
  if (precision != 32 && precision != 64) return bfail(nullptr, FDTDBATH_ERR_ARG, "precision must be 32 or 64");
  if (cluster_ctas < 1 || cluster_ctas > kBatchMaxCluster || block_threads < 1 || block_threads > 1024 || nclusters < 1 ||
      smem_per_cta < 1024 || !(resolution > 0))
    return bfail(nullptr, FDTDBATH_ERR_ARG, "bad plan shape");
  fdtdbath_batch tmp;
  tmp.prec = precision;
  tmp.esz = precision == 64 ? 8 : 4;
  tmp.dx = 1.0 / resolution;
  tmp.courant = courant;
  tmp.dt = courant * tmp.dx;
  std::string why;
  int rc = build_cavities(&tmp, cavities, ncav, why);
  if (rc) return bfail(nullptr, rc, why);
  Plan P;
  rc = pack(tmp.cavs, tmp.mats, tmp.esz, precision == 32, cluster_ctas, block_threads, nclusters, smem_per_cta, P, why);
  if (rc) return bfail(nullptr, rc, why);
  for (size_t r = 0; r < P.ctas.size(); ++r) {
    if (cta_work) cta_work[r] = P.ctas[r].work;
    if (cta_ncell) cta_ncell[r] = P.ctas[r].d.ncell;
    if (cta_smem) cta_smem[r] = P.ctas[r].d.smem_bytes;
  }
  if (cav_cluster)
    for (int i = 0; i < ncav; ++i) cav_cluster[i] = P.cav_cluster[(size_t)i];
  return (int)P.ctas.size();
}

}  // extern "C"
