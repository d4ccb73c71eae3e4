// host_common.h -- host-side pieces shared by the single-simulation planner (api.cpp) and the
// batch planner (batch.cpp): the per-material coefficients of the explicit ADE updates
// (Eq. Pz_1D_Lorentz, Pz_update-LB, Yzj_finite_difference), the stability checks and the CPML
// profile.  Both planners must produce bit-identical coefficients for the same material.
#pragma once

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fdtdbath.h"
#include "internal.h"

namespace fdtdbath {

struct HostMat {
  int kind, nb;
  int64_t zlo, zhi, ncell, base, ybase;
  double eps, w0, g0, sigma;
  std::vector<double> wj, gj, kj;
  // derived (double)
  double cE, c1m, W, c2, A, rho, w0r2;
  double dcE, rho_s;   // per unit sigma(r): cE = dcE sigma(r), rho = rho_s / sigma(r)
  std::vector<double> rowsLit, rowsInc;  // [nb][kCoefStride]
  int user_index = -1;                    // position in the caller's material list
};

// CPML profile (Roden-Gedney, kappa = 1) at a z position in cells of an nz-cell axis with npml
// absorbing cells at each end.  The left absorber interface sits at z = npml, the right one at
// z = nz-1-npml; depth d is clamped to npml; sigma = 0.8 (m+1)/dx (d/npml)^m with m = 3;
// alpha = 2 pi 0.05 (1 - d/npml); b = exp(-(sigma + alpha) dt), c = sigma/(sigma + alpha) (b - 1).
inline void cpml_coeffs(int npml, int64_t nz, double dx, double dt, double zpos, double* b, double* c) {
  *b = 1.0;
  *c = 0.0;
  if (npml <= 0) return;
  const double zl = (double)npml, zr = (double)(nz - 1 - npml);
  double d = 0.0;
  if (zpos < zl) d = zl - zpos;
  else if (zpos > zr) d = zpos - zr;
  if (d > (double)npml) d = (double)npml;
  if (d <= 0.0) return;
  const double r = d / (double)npml;
  const double sig = 0.8 * 4.0 / dx * r * r * r;
  const double alpha = 2.0 * M_PI * 0.05 * (1.0 - r);
  *b = std::exp(-(sig + alpha) * dt);
  *c = sig / (sig + alpha) * (*b - 1.0);
}

// Coefficients of the explicit updates of one material (double precision).
inline void expand_material(HostMat& m, double dt) {
  const double dt2 = dt * dt;
  double S = 0.0;
  m.rowsLit.assign((size_t)m.nb * kCoefStride, 0.0);
  m.rowsInc.assign((size_t)m.nb * kCoefStride, 0.0);
  for (int j = 0; j < m.nb; ++j) {
    const double wj = m.wj[j], gj = m.gj[j], kj = m.kj[j];
    const double den = 1.0 + 0.5 * gj * dt;
    const double a = (2.0 - wj * wj * dt * dt) / den;   // a_j
    const double b = -2.0 / den;                        // b_j
    const double c = kj * dt / (2.0 * den);             // c_j
    S += kj * c;
    const double apb = -(wj * wj * dt2) / den;          // a_j + b_j without cancellation
    const double mbp1 = (1.0 - 0.5 * gj * dt) / den;    // -(b_j + 1)
    double* L = &m.rowsLit[(size_t)j * kCoefStride];
    L[0] = kj;
    L[1] = a;
    L[2] = b;
    L[3] = b + 1.0;
    L[4] = c;
    L[5] = wj * wj * dt2;
    double* I = &m.rowsInc[(size_t)j * kCoefStride];
    I[0] = kj * apb;
    I[1] = -kj * b;
    I[2] = apb;
    I[3] = mbp1;
    I[4] = c;
    I[5] = wj * wj * dt2;
  }
  const double w0 = m.w0, g0 = m.g0;
  m.cE = w0 * w0 * dt * dt * m.sigma;
  if (m.kind == FDTDBATH_DRUDE) {
    m.c1m = 0.0 * dt * dt - 2.0;
    m.W = 0.0;
    m.w0r2 = 0.0;
  } else {
    m.c1m = w0 * w0 * dt * dt - 2.0;
    m.W = w0 * w0 * dt * dt;
    m.w0r2 = w0 * w0;
  }
  if (m.kind == FDTDBATH_LORENTZ_BATH) {
    m.c2 = 1.0 - 0.5 * g0 * dt - 0.5 * dt * S;
    m.A = 1.0 + 0.5 * g0 * dt + 0.5 * dt * S;
  } else {
    m.c2 = 1.0 - 0.5 * g0 * dt;
    m.A = 1.0 + 0.5 * g0 * dt;
  }
  m.rho = (m.sigma > 0.0 && w0 > 0.0) ? 1.0 / (m.sigma * w0 * w0) : 0.0;
  m.dcE = w0 * w0 * dt * dt;
  m.rho_s = w0 > 0.0 ? 1.0 / (w0 * w0) : 0.0;
  if (m.kind == FDTDBATH_VACUUM) {
    m.cE = m.c1m = m.W = m.c2 = 0.0;
    m.A = 1.0;
    m.rho = 0.0;
    m.dcE = m.rho_s = 0.0;
  }
}

// Coupled field + oscillator stability of a layer at oscillator strength sigma: a plane wave of
// the scheme obeys Omega^2 (eps_inf + chi_d) = K^2 with Omega = 2 sin(w dt/2)/dt and
// K^2 <= 4 dims/dx^2, and its largest Omega^2 is below w_max^2 + K^2/eps_inf (w_max^2 =
// w0^2 (1 + sigma) + sum k_j^2, or w0^2 sigma for Drude); every root stays on the unit circle
// while that is <= 4/dt^2.  With a per-cell sigma(r) the bound holds cell by cell, so the largest
// sigma(r) of the layer decides.
inline bool oscillator_stable(const HostMat& h, double sigma, double dt, double courant, int dims) {
  double wmax2 = 0.0;
  if (h.kind == FDTDBATH_DRUDE) wmax2 = h.w0 * h.w0 * sigma;
  else if (h.kind != FDTDBATH_VACUUM) wmax2 = h.w0 * h.w0 * (1.0 + sigma);
  for (double k : h.kj) wmax2 += k * k;
  const double lhs = wmax2 * dt * dt + 4.0 * courant * courant * dims / h.eps;
  return !(lhs > 4.0 * (1.0 + 1e-12));
}

// Validate one layer and fill h (nu-units scaled by 2 pi, coefficients expanded).  `plane` is the
// number of cells per z-plane, `dims` the number of axes with more than one cell.  Returns 0 or
// a FDTDBATH_ERR_* code with the reason in why.  The z-range itself is checked by the caller.
inline int build_material(const fdtdbath_material& M, int64_t plane, double dt, double courant, int dims,
                          HostMat& h, std::string& why) {
  if (M.kind < 0 || M.kind > 3) return why = "unknown material kind", FDTDBATH_ERR_ARG;
  if (!(M.eps_inf > 0)) return why = "eps_inf must be positive", FDTDBATH_ERR_ARG;
  if (M.sigma < 0 || M.gamma < 0 || M.frequency < 0) return why = "negative material parameter", FDTDBATH_ERR_ARG;
  h = HostMat{};
  h.kind = M.kind;
  h.zlo = M.z_lo;
  h.zhi = M.z_hi;
  h.ncell = (M.z_hi - M.z_lo) * plane;
  h.eps = M.eps_inf;
  h.w0 = 2.0 * M_PI * M.frequency;
  h.g0 = 2.0 * M_PI * M.gamma;
  h.sigma = M.sigma;
  h.nb = 0;
  if (M.kind == FDTDBATH_LORENTZ_BATH) {
    if (M.num_bath < 0 || M.num_bath > kMaxBathStep) return why = "num_bath must be in [0, 128]", FDTDBATH_ERR_ARG;
    if (M.num_bath && (!M.bath_frequencies || !M.bath_gammas || !M.bath_couplings))
      return why = "bath arrays missing", FDTDBATH_ERR_ARG;
    h.nb = M.num_bath;
    for (int j = 0; j < h.nb; ++j) {
      if (M.bath_frequencies[j] < 0 || M.bath_gammas[j] < 0) return why = "negative bath parameter", FDTDBATH_ERR_ARG;
      h.wj.push_back(2.0 * M_PI * M.bath_frequencies[j]);
      h.gj.push_back(2.0 * M_PI * M.bath_gammas[j]);
      h.kj.push_back(2.0 * M_PI * M.bath_couplings[j]);
    }
  }
  // explicit oscillator updates are stable only for w dt < 2
  if (M.kind != FDTDBATH_DRUDE && M.kind != FDTDBATH_VACUUM && h.w0 * dt >= 2.0)
    return why = "w0 dt >= 2: oscillator update unstable", FDTDBATH_ERR_CFL;
  for (double w : h.wj)
    if (w * dt >= 2.0) return why = "w_j dt >= 2: bath update unstable", FDTDBATH_ERR_CFL;
  // coupled field + oscillator stability (oscillator_stable)
  if (!oscillator_stable(h, h.sigma, dt, courant, dims))
    return why = "field-oscillator update unstable: w_max^2 dt^2 + 4 S^2 dims/eps_inf > 4", FDTDBATH_ERR_CFL;
  expand_material(h, dt);
  return 0;
}

template <typename T>
MatK<T> mat_k(const HostMat& m, int coef_off, double dt) {
  MatK<T> k{};
  k.zlo = (int)m.zlo;
  k.zhi = (int)m.zhi;
  k.kind = m.kind;
  k.nb = m.nb;
  k.base = m.base;
  k.ybase = m.ybase;
  k.ncell = m.ncell;
  k.coef_off = coef_off;
  k.eps = (T)m.eps;
  k.cE = (T)m.cE;
  k.c1m = (T)m.c1m;
  k.W = (T)m.W;
  k.c2 = (T)m.c2;
  k.A = (T)m.A;
  k.inv_A = (T)(1.0 / m.A);
  k.inv_eps = (T)(1.0 / m.eps);
  k.rho_idt2 = (T)(m.rho / (dt * dt));
  k.w0r2dt2 = (T)(m.w0r2 * dt * dt);
  k.dcE = (T)m.dcE;
  k.rho_s = (T)(m.rho_s / (dt * dt));
  return k;
}

}  // namespace fdtdbath
