/*
 * fdtd_oracle.c -- plain FP64 CPU oracle of the FDTD-Bath time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg and reference arm load this file.  It shares no code, header,
 * table or constant generator with the CUDA library; it reads the same seeded
 * inputs and nothing else.
 *
 * What it computes (T. E. Li, "FDTD with Auxiliary Bath Fields for
 * Condensed-Phase Polaritonics", arXiv 2505.23963):
 *   - Maxwell curl equations, Eq. (1a,b), on a Yee grid; D = eps0 E + P (Sec. II);
 *     the loop order of Eq. (FDTD-1D): D^{n+1/2} from H^n, E^{n+1/2} = (D-P^{n+1/2})/eps,
 *     "evaluate P^{n+3/2}", H^{n+1} from E^{n+1/2}, generalised to 3D with the
 *     standard curl (Sec. II.C, last paragraph).  The 1D H update is taken with the
 *     sign that Maxwell's Eq. (1b) fixes (the printed 1D H update has the opposite
 *     sign, which does not give a wave equation).
 *   - Lorentz polarization update, Eq. (Pz_1D_Lorentz); Drude = the same with the
 *     restoring term w0^2 set to zero and the numerator w0^2*sigma kept (Eq. chi_L text).
 *   - Lorentz-Bath polarization update, Eq. (Pz_update-LB) with A, and the bath
 *     mode update Eq. (Yzj_finite_difference) with a_j, b_j, c_j.  P first, then
 *     every Y_j with the new P.  One independent bath set per P component.
 *   - A convolutional PML (Roden-Gedney CPML, kappa = 1) on the two z ends; the
 *     paper's absorber is MEEP's PML and is not specified further.  Its memory is kept
 *     in units of a field difference (dx times the usual psi), so that every curl term
 *     enters as (dt/dx) times a difference, the form Eq. (FDTD-1D) prints.
 *   - A soft Gaussian-pulse source, running-DFT monitors of the plane-mean fields,
 *     EM/oscillator/bath energy traces and the exact discrete energy invariant
 *     (derived from the Hamiltonian density, Eq. H_full).
 *
 * Units: c = eps0 = mu0 = 1.  Frequencies arrive in nu-units (nu = omega/2pi, as MEEP
 * and the paper report them) and are turned into angular values here.
 *
 * Layout: every field is a full [nz][ny][nx] array (x fastest); x and y are periodic;
 * outside 0 <= k < nz every field is zero.  Yee positions (cell units):
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
 *   Hx (i, j+1/2, k+1/2)  Hy (i+1/2, j, k+1/2)  Hz (i+1/2, j+1/2, k)
 * A material fills whole z-planes lo <= k < hi for every component.  Its oscillator strength may
 * vary per cell, sigma(r) in Eq. EOM_Lorentz / EOM_LorentzBath-1: one value per cell (i, j, k) of
 * the layer, shared by the three components of that cell, entering the drive term of the P update
 * and the mass density rho(r) = 1/(sigma(r) w0^2) of the energy (Eq. H_full).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXMAT 16
#define ORC_MAXSRC 8
#define ORC_MAXMON 8

enum { ORC_VACUUM = 0, ORC_LORENTZ = 1, ORC_DRUDE = 2, ORC_LORENTZ_BATH = 3 };

typedef struct {
  int kind;
  int64_t zlo, zhi;
  double eps_inf;
  double w0, g0, sigma; /* angular frequency, angular damping, oscillator strength */
  int nb;
  double *wj, *gj, *kj; /* bath frequencies, dampings, couplings (angular) */
  int64_t ncell;        /* cells in the material's planes */
  double *P[3], *Pm[3]; /* P^{n+1/2}, P^{n-1/2} per component */
  double *Y[3], *Ym[3]; /* Y_j^{n+1/2}, Y_j^{n-1/2}: [nb][ncell] per component */
  double *sig;          /* sigma(r) per cell [ncell] (Eq. EOM_Lorentz), or NULL: sigma everywhere */
} omat;

typedef struct {
  int comp;
  int64_t z;
  double nu_c, fwidth, amp, t0;
  double *phase; /* nx*ny values or NULL */
} osrc;

typedef struct {
  int64_t z;
  int nfreq;
  double *nu;
  double *acc; /* [nfreq][4 fields Ex,Ey,Hx,Hy][re,im] */
} omon;

typedef struct {
  int64_t nx, ny, nz, ncell;
  double dx, dt;
  int npml;
  int64_t n; /* completed steps */
  double *E[3], *H[3], *D[3];
  double *psiE[2], *psiH[2]; /* CPML memory of d/dz terms: Ex<-dHy/dz, Ey<-dHx/dz; Hx<-dEy/dz, Hy<-dEx/dz */
  double *bE, *cE, *bH, *cH; /* CPML coefficients per z at E (integer) and H (half) positions */
  int *mat_of_k;
  int nmat, nsrc, nmon;
  omat mat[ORC_MAXMAT];
  osrc src[ORC_MAXSRC];
  omon mon[ORC_MAXMON];
  /* energy box and traces */
  int64_t ebox_lo, ebox_hi;
  int64_t ntrace, trace_cap;
  double *trace; /* [cap][4]: U_EM, U_P, U_bath, invariant */
  int record_invariant;
} osim;

static void *xcalloc(size_t n, size_t sz) {
  void *p = calloc(n ? n : 1, sz);
  return p;
}

/* ---- CPML profile: Roden-Gedney convolutional PML with kappa = 1. -----------------
 * Depth d (cells) of a z position (cells) into the absorber: the left interface
 * sits at z = npml and the right one at z = nz-1-npml; d is clamped to npml.
 * sigma(d) = sigma_max (d/npml)^3, sigma_max = 0.8*(3+1)/dx, alpha(d) =
 * alpha_max (1 - d/npml), alpha_max = 2*pi*0.05.  b = exp(-(sigma+alpha) dt),
 * c = sigma/(sigma+alpha) (b-1).  Outside the absorber b = 1 and c = 0.        */
static void orc_pml_coef(const osim *s, double zpos, double *b, double *c) {
  double d = 0.0;
  double zl = (double)s->npml, zr = (double)(s->nz - 1 - s->npml);
  if (s->npml <= 0) {
    *b = 1.0;
    *c = 0.0;
    return;
  }
  if (zpos < zl) d = zl - zpos;
  else if (zpos > zr) d = zpos - zr;
  if (d > (double)s->npml) d = (double)s->npml;
  if (d <= 0.0) {
    *b = 1.0;
    *c = 0.0;
    return;
  }
  double r = d / (double)s->npml;
  double sigma = 0.8 * 4.0 / s->dx * r * r * r;
  double alpha = 2.0 * M_PI * 0.05 * (1.0 - r);
  *b = exp(-(sigma + alpha) * s->dt);
  *c = sigma / (sigma + alpha) * (*b - 1.0);
}

osim *orc_new(int64_t nx, int64_t ny, int64_t nz, double resolution, double courant, int npml) {
  osim *s = (osim *)xcalloc(1, sizeof(osim));
  if (!s) return NULL;
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->ncell = nx * ny * nz;
  s->dx = 1.0 / resolution;
  s->dt = courant * s->dx;
  s->npml = npml;
  for (int c = 0; c < 3; ++c) {
    s->E[c] = (double *)xcalloc(s->ncell, sizeof(double));
    s->H[c] = (double *)xcalloc(s->ncell, sizeof(double));
    s->D[c] = (double *)xcalloc(s->ncell, sizeof(double));
  }
  for (int c = 0; c < 2; ++c) {
    s->psiE[c] = (double *)xcalloc(s->ncell, sizeof(double));
    s->psiH[c] = (double *)xcalloc(s->ncell, sizeof(double));
  }
  s->bE = (double *)xcalloc(nz, sizeof(double));
  s->cE = (double *)xcalloc(nz, sizeof(double));
  s->bH = (double *)xcalloc(nz, sizeof(double));
  s->cH = (double *)xcalloc(nz, sizeof(double));
  for (int64_t k = 0; k < nz; ++k) {
    orc_pml_coef(s, (double)k, &s->bE[k], &s->cE[k]);
    orc_pml_coef(s, (double)k + 0.5, &s->bH[k], &s->cH[k]);
  }
  s->mat_of_k = (int *)xcalloc(nz, sizeof(int));
  for (int64_t k = 0; k < nz; ++k) s->mat_of_k[k] = -1;
  s->ebox_lo = 0;
  s->ebox_hi = 0;
  return s;
}

/* Material in nu-units (frequency, gamma, sigma, bath arrays); stored angular. */
int orc_add_material(osim *s, int kind, int64_t zlo, int64_t zhi, double eps_inf, double freq,
                     double gamma, double sigma, int nb, const double *bath_freq,
                     const double *bath_gamma, const double *bath_coupling) {
  if (s->nmat >= ORC_MAXMAT || zlo < 0 || zhi > s->nz || zlo >= zhi) return -1;
  for (int64_t k = zlo; k < zhi; ++k)
    if (s->mat_of_k[k] >= 0) return -2;
  omat *m = &s->mat[s->nmat];
  memset(m, 0, sizeof(*m));
  m->kind = kind;
  m->zlo = zlo;
  m->zhi = zhi;
  m->eps_inf = eps_inf;
  m->w0 = 2.0 * M_PI * freq;
  m->g0 = 2.0 * M_PI * gamma;
  m->sigma = sigma;
  m->nb = (kind == ORC_LORENTZ_BATH) ? nb : 0;
  m->ncell = (zhi - zlo) * s->nx * s->ny;
  m->wj = (double *)xcalloc(m->nb, sizeof(double));
  m->gj = (double *)xcalloc(m->nb, sizeof(double));
  m->kj = (double *)xcalloc(m->nb, sizeof(double));
  for (int j = 0; j < m->nb; ++j) {
    m->wj[j] = 2.0 * M_PI * bath_freq[j];
    m->gj[j] = 2.0 * M_PI * bath_gamma[j];
    m->kj[j] = 2.0 * M_PI * bath_coupling[j];
  }
  for (int c = 0; c < 3; ++c) {
    m->P[c] = (double *)xcalloc(m->ncell, sizeof(double));
    m->Pm[c] = (double *)xcalloc(m->ncell, sizeof(double));
    m->Y[c] = (double *)xcalloc((size_t)m->nb * m->ncell, sizeof(double));
    m->Ym[c] = (double *)xcalloc((size_t)m->nb * m->ncell, sizeof(double));
  }
  for (int64_t k = zlo; k < zhi; ++k) s->mat_of_k[k] = s->nmat;
  s->nmat++;
  return 0;
}

int orc_add_source(osim *s, int comp, int64_t z, double nu_c, double fwidth, double amp, double t0,
                   const double *phase) {
  if (s->nsrc >= ORC_MAXSRC || comp < 0 || comp > 2 || z < 0 || z >= s->nz) return -1;
  osrc *q = &s->src[s->nsrc++];
  q->comp = comp;
  q->z = z;
  q->nu_c = nu_c;
  q->fwidth = fwidth;
  q->amp = amp;
  q->t0 = t0;
  q->phase = NULL;
  if (phase) {
    q->phase = (double *)xcalloc(s->nx * s->ny, sizeof(double));
    memcpy(q->phase, phase, sizeof(double) * s->nx * s->ny);
  }
  return 0;
}

int orc_add_monitor(osim *s, int64_t z, int nfreq, const double *nu) {
  if (s->nmon >= ORC_MAXMON || z < 1 || z >= s->nz) return -1;
  omon *m = &s->mon[s->nmon++];
  m->z = z;
  m->nfreq = nfreq;
  m->nu = (double *)xcalloc(nfreq, sizeof(double));
  memcpy(m->nu, nu, sizeof(double) * nfreq);
  m->acc = (double *)xcalloc((size_t)nfreq * 8, sizeof(double));
  return 0;
}

void orc_set_energy_box(osim *s, int64_t zlo, int64_t zhi, int64_t cap, int record_invariant) {
  s->ebox_lo = zlo;
  s->ebox_hi = zhi;
  free(s->trace);
  s->trace_cap = cap;
  s->ntrace = 0;
  s->trace = (double *)xcalloc((size_t)cap * 4, sizeof(double));
  s->record_invariant = record_invariant;
}

/* ---- index helpers -------------------------------------------------------------- */
static inline int64_t IDX(const osim *s, int64_t i, int64_t j, int64_t k) {
  return (k * s->ny + j) * s->nx + i;
}
static inline int64_t WX(const osim *s, int64_t i) { return (i % s->nx + s->nx) % s->nx; }
static inline int64_t WY(const osim *s, int64_t j) { return (j % s->ny + s->ny) % s->ny; }
/* field value with periodic x,y and zero outside 0 <= k < nz */
static inline double F(const osim *s, const double *a, int64_t i, int64_t j, int64_t k) {
  if (k < 0 || k >= s->nz) return 0.0;
  return a[IDX(s, WX(s, i), WY(s, j), k)];
}

/* Soft source waveform: A exp(-(t-t0)^2 / (2 tau^2)) sin(2 pi nu_c (t-t0) + phase), tau = 1/(2 pi fwidth). */
static double orc_wave(const osrc *q, double t, double phase) {
  double tau = 1.0 / (2.0 * M_PI * q->fwidth);
  double u = t - q->t0;
  return q->amp * exp(-u * u / (2.0 * tau * tau)) * sin(2.0 * M_PI * q->nu_c * u + phase);
}

/* ---- the ADE updates, one cell at a time ------------------------------------------ */

/* Eq. (Pz_1D_Lorentz): P^{n+1} = [eps0 w0^2 dt^2 sigma E^n - (w0^2 dt^2 - 2) P^n
 *                                  - (1 - gamma dt/2) P^{n-1}] / (1 + gamma dt/2).        */
double orc_lorentz_update(double E, double P, double Pm, double w0, double g, double sigma, double dt) {
  double num = w0 * w0 * dt * dt * sigma * E - (w0 * w0 * dt * dt - 2.0) * P - (1.0 - 0.5 * g * dt) * Pm;
  return (1.0 / (1.0 + 0.5 * g * dt)) * num;
}

/* Drude limit (text after Eq. chi_L): w0^2 := 0 in the restoring term only;
 * the driving term keeps w0^2 sigma (the squared plasma frequency).             */
double orc_drude_update(double E, double P, double Pm, double w0, double g, double sigma, double dt) {
  double num = w0 * w0 * dt * dt * sigma * E - (0.0 * dt * dt - 2.0) * P - (1.0 - 0.5 * g * dt) * Pm;
  return (1.0 / (1.0 + 0.5 * g * dt)) * num;
}

/* Eq. (Yzj_finite_difference) coefficients. */
static void orc_bath_abc(double wj, double gj, double kj, double dt, double *a, double *b, double *c) {
  double den = 1.0 + 0.5 * gj * dt;
  *a = (2.0 - wj * wj * dt * dt) / den;
  *b = -2.0 / den;
  *c = kj * dt / (2.0 * den);
}

/* Eq. (Pz_update-LB) for P^{n+1}, then Eq. (Yzj_finite_difference) for every Y_j^{n+1}.
 * Y[j], Ym[j] hold Y_j^n, Y_j^{n-1} on entry and Y_j^{n+1}, Y_j^n on exit; returns P^{n+1}. */
double orc_lorentz_bath_update(double E, double P, double Pm, double w0, double g0, double sigma,
                               int nb, const double *wj, const double *gj, const double *kj,
                               double *Y, double *Ym, double dt) {
  double S = 0.0, bath = 0.0;
  for (int j = 0; j < nb; ++j) {
    double a, b, c;
    orc_bath_abc(wj[j], gj[j], kj[j], dt, &a, &b, &c);
    S += kj[j] * c;
    bath += kj[j] * (a * Y[j] + b * Ym[j]);
  }
  double A = 1.0 + 0.5 * g0 * dt + 0.5 * dt * S;
  double num = w0 * w0 * dt * dt * sigma * E - (w0 * w0 * dt * dt - 2.0) * P -
               (1.0 - 0.5 * g0 * dt - 0.5 * dt * S) * Pm - 0.5 * dt * bath;
  double Pn = (1.0 / A) * num;
  for (int j = 0; j < nb; ++j) {
    double a, b, c;
    orc_bath_abc(wj[j], gj[j], kj[j], dt, &a, &b, &c);
    double Yn = a * Y[j] + (b + 1.0) * Ym[j] + c * (Pn - Pm);
    Ym[j] = Y[j];
    Y[j] = Yn;
  }
  return Pn;
}

/* ---- one full time step ------------------------------------------------------------ */

static void orc_update_D(osim *s) {
  const double dt = s->dt, S = s->dt / s->dx;
  const double tn = (double)s->n * dt; /* D^{n-1/2} -> D^{n+1/2} is centred on t_n */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < s->nz; ++k) {
    for (int64_t j = 0; j < s->ny; ++j) {
      for (int64_t i = 0; i < s->nx; ++i) {
        int64_t q = IDX(s, i, j, k);
        /* dt (curl H)_x = dt/dx [dHz along y - dHy along z], the latter with the CPML memory */
        double dyHz = F(s, s->H[2], i, j, k) - F(s, s->H[2], i, j - 1, k);
        double dzHy = F(s, s->H[1], i, j, k) - F(s, s->H[1], i, j, k - 1);
        s->psiE[0][q] = s->bE[k] * s->psiE[0][q] + s->cE[k] * dzHy;
        s->D[0][q] += S * (dyHz - (dzHy + s->psiE[0][q]));
        /* dt (curl H)_y = dt/dx [dHx along z - dHz along x] */
        double dzHx = F(s, s->H[0], i, j, k) - F(s, s->H[0], i, j, k - 1);
        double dxHz = F(s, s->H[2], i, j, k) - F(s, s->H[2], i - 1, j, k);
        s->psiE[1][q] = s->bE[k] * s->psiE[1][q] + s->cE[k] * dzHx;
        s->D[1][q] += S * ((dzHx + s->psiE[1][q]) - dxHz);
        /* dt (curl H)_z = dt/dx [dHy along x - dHx along y] */
        double dxHy = F(s, s->H[1], i, j, k) - F(s, s->H[1], i - 1, j, k);
        double dyHx = F(s, s->H[0], i, j, k) - F(s, s->H[0], i, j - 1, k);
        s->D[2][q] += S * (dxHy - dyHx);
      }
    }
  }
  /* soft source: D += dt * s(t_n) on the source plane */
  for (int m = 0; m < s->nsrc; ++m) {
    const osrc *q = &s->src[m];
    for (int64_t j = 0; j < s->ny; ++j)
      for (int64_t i = 0; i < s->nx; ++i) {
        double ph = q->phase ? q->phase[j * s->nx + i] : 0.0;
        s->D[q->comp][IDX(s, i, j, q->z)] += dt * orc_wave(q, tn, ph);
      }
  }
}

/* E^{n+1/2} = (1/eps_inf) (D^{n+1/2} - P^{n+1/2})  (eps0 = 1). */
static void orc_update_E(osim *s) {
  const int64_t plane = s->nx * s->ny;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < s->nz; ++k) {
    int mi = s->mat_of_k[k];
    for (int64_t p = 0; p < plane; ++p) {
      int64_t q = k * plane + p;
      for (int c = 0; c < 3; ++c) {
        if (mi < 0) {
          s->E[c][q] = 1.0 * (s->D[c][q] - 0.0);
        } else {
          const omat *m = &s->mat[mi];
          int64_t r = (k - m->zlo) * plane + p;
          s->E[c][q] = (1.0 / m->eps_inf) * (s->D[c][q] - m->P[c][r]);
        }
      }
    }
  }
}

/* Evaluate P^{n+3/2} (and the bath modes) from E^{n+1/2}. */
static void orc_update_P(osim *s) {
  const int64_t plane = s->nx * s->ny;
  for (int mi = 0; mi < s->nmat; ++mi) {
    omat *m = &s->mat[mi];
    if (m->kind == ORC_VACUUM) continue;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m->ncell; ++r) {
      double Yl[128], Yml[128];
      int64_t q = m->zlo * plane + r;
      for (int c = 0; c < 3; ++c) {
        double E = s->E[c][q], P = m->P[c][r], Pm = m->Pm[c][r], Pn;
        const double sg = m->sig ? m->sig[r] : m->sigma;   /* sigma(r) */
        if (m->kind == ORC_LORENTZ) {
          Pn = orc_lorentz_update(E, P, Pm, m->w0, m->g0, sg, s->dt);
        } else if (m->kind == ORC_DRUDE) {
          Pn = orc_drude_update(E, P, Pm, m->w0, m->g0, sg, s->dt);
        } else {
          for (int j = 0; j < m->nb; ++j) {
            Yl[j] = m->Y[c][(int64_t)j * m->ncell + r];
            Yml[j] = m->Ym[c][(int64_t)j * m->ncell + r];
          }
          Pn = orc_lorentz_bath_update(E, P, Pm, m->w0, m->g0, sg, m->nb, m->wj, m->gj, m->kj,
                                       Yl, Yml, s->dt);
          for (int j = 0; j < m->nb; ++j) {
            m->Y[c][(int64_t)j * m->ncell + r] = Yl[j];
            m->Ym[c][(int64_t)j * m->ncell + r] = Yml[j];
          }
        }
        m->Pm[c][r] = P;
        m->P[c][r] = Pn;
      }
    }
  }
}

/* H^{n+1} = H^n - dt (curl E^{n+1/2})  (mu0 = 1), with CPML on the d/dz terms.
 * If hdot != NULL it receives sum over cells of H^n . H^{n+1}. */
static void orc_update_H(osim *s, double *hdot) {
  const double S = s->dt / s->dx;
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
  for (int64_t k = 0; k < s->nz; ++k) {
    for (int64_t j = 0; j < s->ny; ++j) {
      for (int64_t i = 0; i < s->nx; ++i) {
        int64_t q = IDX(s, i, j, k);
        double h0[3] = {s->H[0][q], s->H[1][q], s->H[2][q]};
        /* dt (curl E)_x = dt/dx [dEz along y - dEy along z], the latter with the CPML memory */
        double dyEz = F(s, s->E[2], i, j + 1, k) - F(s, s->E[2], i, j, k);
        double dzEy = F(s, s->E[1], i, j, k + 1) - F(s, s->E[1], i, j, k);
        s->psiH[0][q] = s->bH[k] * s->psiH[0][q] + s->cH[k] * dzEy;
        s->H[0][q] -= S * (dyEz - (dzEy + s->psiH[0][q]));
        /* dt (curl E)_y = dt/dx [dEx along z - dEz along x] */
        double dzEx = F(s, s->E[0], i, j, k + 1) - F(s, s->E[0], i, j, k);
        double dxEz = F(s, s->E[2], i + 1, j, k) - F(s, s->E[2], i, j, k);
        s->psiH[1][q] = s->bH[k] * s->psiH[1][q] + s->cH[k] * dzEx;
        s->H[1][q] -= S * ((dzEx + s->psiH[1][q]) - dxEz);
        /* dt (curl E)_z = dt/dx [dEy along x - dEx along y] */
        double dxEy = F(s, s->E[1], i + 1, j, k) - F(s, s->E[1], i, j, k);
        double dyEx = F(s, s->E[0], i, j + 1, k) - F(s, s->E[0], i, j, k);
        s->H[2][q] -= S * (dxEy - dyEx);
        acc += h0[0] * s->H[0][q] + h0[1] * s->H[1][q] + h0[2] * s->H[2][q];
      }
    }
  }
  if (hdot) *hdot = acc;
}

/* Running DFT of the plane means: F(nu) += f(t) exp(+i 2 pi nu t) dt, with E^{n+1/2} at
 * t = (n+1/2) dt and H^{n+1} (mean of the two H planes around the monitor) at t = (n+1) dt. */
static void orc_monitors(osim *s) {
  const int64_t plane = s->nx * s->ny;
  for (int mm = 0; mm < s->nmon; ++mm) {
    omon *m = &s->mon[mm];
    double f[4] = {0, 0, 0, 0};
    for (int64_t p = 0; p < plane; ++p) {
      f[0] += s->E[0][m->z * plane + p];
      f[1] += s->E[1][m->z * plane + p];
      f[2] += 0.5 * (s->H[0][(m->z - 1) * plane + p] + s->H[0][m->z * plane + p]);
      f[3] += 0.5 * (s->H[1][(m->z - 1) * plane + p] + s->H[1][m->z * plane + p]);
    }
    for (int c = 0; c < 4; ++c) f[c] /= (double)plane;
    double tE = ((double)s->n + 0.5) * s->dt, tH = ((double)s->n + 1.0) * s->dt;
    for (int q = 0; q < m->nfreq; ++q) {
      double aE = 2.0 * M_PI * m->nu[q] * tE, aH = 2.0 * M_PI * m->nu[q] * tH;
      double cE = cos(aE), sE = sin(aE), cH = cos(aH), sH = sin(aH);
      double *acc = m->acc + (size_t)q * 8;
      acc[0] += f[0] * cE * s->dt;
      acc[1] += f[0] * sE * s->dt;
      acc[2] += f[1] * cE * s->dt;
      acc[3] += f[1] * sE * s->dt;
      acc[4] += f[2] * cH * s->dt;
      acc[5] += f[2] * sH * s->dt;
      acc[6] += f[3] * cH * s->dt;
      acc[7] += f[3] * sH * s->dt;
    }
  }
}

/* Energy per unit transverse area inside the box, from the stored state after a step:
 *   U_EM   = sum dx/(nx ny) * 1/2 (eps_inf E.E + H.H)            (E^{n+1/2}, H^{n+1})
 *   U_P    = sum dx/(nx ny) * rho/2 (((P - Pm)/dt)^2 + w0r^2 P^2)   rho = 1/(sigma(r) w0^2)
 *   U_bath = sum dx/(nx ny) * sum_j rho/2 (((Y_j - Ym_j)/dt)^2 + w_j^2 Y_j^2)
 * (w0r = w0, or 0 for Drude).  This follows the energy density of Eq. (H_full)
 * written with P and the Y_j as coordinates (Pi_P = rho (dP/dt + sum k_j Y_j)).  */
static void orc_energy_box(const osim *s, double out[3]) {
  const int64_t plane = s->nx * s->ny;
  double uem = 0.0, up = 0.0, ub = 0.0;
  const double w = s->dx / (double)plane;
  for (int64_t k = s->ebox_lo; k < s->ebox_hi; ++k) {
    int mi = s->mat_of_k[k];
    double eps = (mi >= 0) ? s->mat[mi].eps_inf : 1.0;
    for (int64_t p = 0; p < plane; ++p) {
      int64_t q = k * plane + p;
      for (int c = 0; c < 3; ++c) uem += w * 0.5 * (eps * s->E[c][q] * s->E[c][q] + s->H[c][q] * s->H[c][q]);
      if (mi < 0) continue;
      const omat *m = &s->mat[mi];
      if (m->kind == ORC_VACUUM) continue;
      int64_t r = (k - m->zlo) * plane + p;
      const double sg = m->sig ? m->sig[r] : m->sigma;
      if (sg == 0.0) continue;
      double rho = 1.0 / (sg * m->w0 * m->w0);
      double w0r = (m->kind == ORC_DRUDE) ? 0.0 : m->w0;
      for (int c = 0; c < 3; ++c) {
        double v = (m->P[c][r] - m->Pm[c][r]) / s->dt;
        up += w * 0.5 * rho * (v * v + w0r * w0r * m->P[c][r] * m->P[c][r]);
        for (int j = 0; j < m->nb; ++j) {
          double y = m->Y[c][(int64_t)j * m->ncell + r], ym = m->Ym[c][(int64_t)j * m->ncell + r];
          double vy = (y - ym) / s->dt;
          ub += w * 0.5 * rho * (vy * vy + m->wj[j] * m->wj[j] * y * y);
        }
      }
    }
  }
  out[0] = uem;
  out[1] = up;
  out[2] = ub;
}

/* Exact discrete invariant of the undamped, source-free scheme (closed box, no CPML).
 * With m = n, E_m = E^{n+1/2}, H_m = H^n, p_m = P^{n+1/2}, summed over all cells:
 *   I = eps/2 E_m^2 + 1/2 H_m.H_{m+1} - 1/2 E_m (p_{m+1} - p_m)
 *       + rho/(2 dt^2) [ (p_{m+1}-p_m)^2 + w0r^2 dt^2 p_{m+1} p_m ]
 *       + sum_j rho/(2 dt^2) [ (Y_{m+1}-Y_m)^2 + w_j^2 dt^2 Y_{m+1} Y_m ].
 * Called after the P/Y update (p_{m+1} = P, p_m = Pm) with hdot = H_m.H_{m+1}.
 * Derivation: the Yee pair conserves eps|E_m|^2 + H_m.H_{m+1} up to the exchange
 * term with dP/dt; each central-difference oscillator conserves its leapfrog energy
 * up to the forcing by E (Eq. EOM_LorentzBath-1) and the +/- k_j couplings, which
 * cancel between P and the Y_j (Eq. EOM_LorentzBath-2); summing by parts leaves
 * the boundary term -1/2 E_m (p_{m+1} - p_m).                                     */
static double orc_invariant(const osim *s, double hdot) {
  const int64_t plane = s->nx * s->ny;
  double I = 0.5 * hdot;
  const double dt = s->dt;
  for (int64_t k = 0; k < s->nz; ++k) {
    int mi = s->mat_of_k[k];
    double eps = (mi >= 0) ? s->mat[mi].eps_inf : 1.0;
    for (int64_t p = 0; p < plane; ++p) {
      int64_t q = k * plane + p;
      for (int c = 0; c < 3; ++c) I += 0.5 * eps * s->E[c][q] * s->E[c][q];
      if (mi < 0) continue;
      const omat *m = &s->mat[mi];
      if (m->kind == ORC_VACUUM) continue;
      int64_t r = (k - m->zlo) * plane + p;
      const double sg = m->sig ? m->sig[r] : m->sigma;
      if (sg == 0.0) continue;
      double rho = 1.0 / (sg * m->w0 * m->w0);
      double w0r = (m->kind == ORC_DRUDE) ? 0.0 : m->w0;
      for (int c = 0; c < 3; ++c) {
        double p1 = m->P[c][r], p0 = m->Pm[c][r];
        I += -0.5 * s->E[c][q] * (p1 - p0);
        I += rho / (2.0 * dt * dt) * ((p1 - p0) * (p1 - p0) + w0r * w0r * dt * dt * p1 * p0);
        for (int j = 0; j < m->nb; ++j) {
          double y1 = m->Y[c][(int64_t)j * m->ncell + r], y0 = m->Ym[c][(int64_t)j * m->ncell + r];
          I += rho / (2.0 * dt * dt) * ((y1 - y0) * (y1 - y0) + m->wj[j] * m->wj[j] * dt * dt * y1 * y0);
        }
      }
    }
  }
  return I;
}

void orc_step(osim *s, int64_t nsteps) {
  for (int64_t it = 0; it < nsteps; ++it) {
    orc_update_D(s);
    orc_update_E(s);
    orc_update_P(s);
    double hdot = 0.0;
    orc_update_H(s, s->record_invariant ? &hdot : NULL);
    orc_monitors(s);
    if (s->trace && s->ntrace < s->trace_cap) {
      double u[3];
      orc_energy_box(s, u);
      double *t = s->trace + 4 * s->ntrace;
      t[0] = u[0];
      t[1] = u[1];
      t[2] = u[2];
      t[3] = s->record_invariant ? orc_invariant(s, hdot) : 0.0;
      s->ntrace++;
    }
    s->n++;
  }
}

/* ---- state access ------------------------------------------------------------------
 * field ids: 0..2 E, 3..5 H, 6..8 D, 9..11 P^{n+1/2}, 12..14 P^{n-1/2} (full grid, zero
 * outside materials); bath mode j of component c, level l (0: Y^{n+1/2}, 1: Y^{n-1/2}):
 * 64 + (c*2 + l)*128 + j.  CPML memories: 32..33 psiE (x,y), 34..35 psiH (x,y).
 * 16: sigma(r) (full grid; the material's sigma where no map was written, zero outside the
 * dispersive layers; a write sets the map of every dispersive layer).                  */
static double *orc_field_ptr(osim *s, int id, int64_t *is_mat) {
  *is_mat = 0;
  if (id >= 0 && id < 3) return s->E[id];
  if (id >= 3 && id < 6) return s->H[id - 3];
  if (id >= 6 && id < 9) return s->D[id - 6];
  if (id >= 32 && id < 34) return s->psiE[id - 32];
  if (id >= 34 && id < 36) return s->psiH[id - 34];
  *is_mat = 1;
  return NULL;
}

static int orc_access(osim *s, int id, double *buf, int write) {
  int64_t is_mat;
  double *f = orc_field_ptr(s, id, &is_mat);
  if (!is_mat) {
    if (write) memcpy(f, buf, sizeof(double) * s->ncell);
    else memcpy(buf, f, sizeof(double) * s->ncell);
    return 0;
  }
  const int64_t plane = s->nx * s->ny;
  int c, lvl = 0, j = -1;
  if (id >= 9 && id < 12) {
    c = id - 9;
    lvl = 0;
  } else if (id >= 12 && id < 15) {
    c = id - 12;
    lvl = 1;
  } else if (id == 16) {
    c = 0;
    lvl = 0;
  } else if (id >= 64) {
    int r = id - 64;
    j = r % 128;
    c = (r / 128) / 2;
    lvl = (r / 128) % 2;
    if (c > 2) return -1;
  } else {
    return -1;
  }
  if (!write) memset(buf, 0, sizeof(double) * s->ncell);
  for (int mi = 0; mi < s->nmat; ++mi) {
    omat *m = &s->mat[mi];
    double *src;
    if (id == 16) {
      if (m->kind == ORC_VACUUM) continue;
      if (!m->sig) {
        if (!write) {
          for (int64_t r = 0; r < m->ncell; ++r) buf[m->zlo * plane + r] = m->sigma;
          continue;
        }
        m->sig = (double *)xcalloc((size_t)m->ncell, sizeof(double));
      }
      src = m->sig;
    } else if (j < 0) src = lvl ? m->Pm[c] : m->P[c];
    else {
      if (j >= m->nb) continue;
      src = (lvl ? m->Ym[c] : m->Y[c]) + (int64_t)j * m->ncell;
    }
    for (int64_t r = 0; r < m->ncell; ++r) {
      if (write) src[r] = buf[m->zlo * plane + r];
      else buf[m->zlo * plane + r] = src[r];
    }
  }
  return 0;
}

int orc_get_field(osim *s, int id, double *out) { return orc_access(s, id, out, 0); }
int orc_set_field(osim *s, int id, const double *in) { return orc_access(s, id, (double *)in, 1); }

int orc_get_dft(const osim *s, int mon, double *out) {
  if (mon < 0 || mon >= s->nmon) return -1;
  memcpy(out, s->mon[mon].acc, sizeof(double) * 8 * s->mon[mon].nfreq);
  return 0;
}

int64_t orc_get_trace(const osim *s, double *out, int64_t maxlen) {
  int64_t n = s->ntrace < maxlen ? s->ntrace : maxlen;
  memcpy(out, s->trace, sizeof(double) * 4 * n);
  return n;
}

int64_t orc_steps_done(const osim *s) { return s->n; }
double orc_dt(const osim *s) { return s->dt; }

void orc_free(osim *s) {
  if (!s) return;
  for (int c = 0; c < 3; ++c) {
    free(s->E[c]);
    free(s->H[c]);
    free(s->D[c]);
  }
  for (int c = 0; c < 2; ++c) {
    free(s->psiE[c]);
    free(s->psiH[c]);
  }
  free(s->bE);
  free(s->cE);
  free(s->bH);
  free(s->cH);
  free(s->mat_of_k);
  for (int mi = 0; mi < s->nmat; ++mi) {
    omat *m = &s->mat[mi];
    free(m->wj);
    free(m->gj);
    free(m->kj);
    for (int c = 0; c < 3; ++c) {
      free(m->P[c]);
      free(m->Pm[c]);
      free(m->Y[c]);
      free(m->Ym[c]);
    }
    free(m->sig);
  }
  for (int m = 0; m < s->nsrc; ++m) free(s->src[m].phase);
  for (int m = 0; m < s->nmon; ++m) {
    free(s->mon[m].nu);
    free(s->mon[m].acc);
  }
  free(s->trace);
  free(s);
}
