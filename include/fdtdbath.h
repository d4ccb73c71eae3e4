/*
 * fdtdbath.h -- C ABI of the GB300 FDTD-Bath library.
 *
 * The library advances Maxwell's curl equations on a Yee grid (Eq. 1a,b of
 * T. E. Li, "FDTD with Auxiliary Bath Fields for Condensed-Phase Polaritonics",
 * arXiv 2505.23963) with Lorentz, Drude and Lorentz-Bath polarizations
 * (Eq. EOM_Lorentz, EOM_LorentzBath; explicit updates Eq. Pz_1D_Lorentz,
 * Pz_update-LB and Yzj_finite_difference), a convolutional PML on the two z
 * ends, soft Gaussian-pulse sources, running-DFT monitors of the plane-mean
 * fields and FP64 energy traces.  Every step runs in hand-written sm_103a CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions used by every entry point
 *   - Units: c = eps0 = mu0 = 1; dx = 1/resolution, dt = courant*dx.  Every
 *     frequency-like parameter (frequency, gamma, bath frequencies, dampings and
 *     couplings, pulse centre and width, DFT frequencies) is in nu-units,
 *     nu = omega/2pi, as in MEEP and the paper; the library multiplies by 2pi.
 *   - Grid: nx * ny * nz cells, stored [nz][ny][nx] with x fastest; periodic in x
 *     and y (Bloch k = 0); along z every field vanishes outside 0 <= k < nz and a
 *     CPML of pml_cells planes absorbs at each end.  Yee positions in cell units:
 *     Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) Hx(i,j+1/2,k+1/2) Hy(i+1/2,j,k+1/2)
 *     Hz(i+1/2,j+1/2,k).  A material fills whole planes z_lo <= k < z_hi.
 *   - Time levels after n completed steps: E^{n-1/2}, H^n, P^{n+1/2} (field
 *     P) and P^{n-1/2} (field PM), bath modes Y_j^{n+1/2} / Y_j^{n-1/2}.
 *   - Return value: FDTDBATH_OK (0) or a negative FDTDBATH_ERR_* code; the text
 *     of the last error of a simulation is in fdtdbath_last_error().
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership.  Device state belongs to the simulation and lives until
 *     fdtdbath_destroy().
 *   - All device work is queued on options.cuda_stream; calls that return data
 *     to the host synchronize that stream.
 */
#ifndef FDTDBATH_H
#define FDTDBATH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTDBATH_ABI_VERSION 1

enum fdtdbath_status {
  FDTDBATH_OK = 0,
  FDTDBATH_ERR_ARG = -1,         /* malformed argument */
  FDTDBATH_ERR_CFL = -2,         /* unstable time step (Courant or oscillator update) */
  FDTDBATH_ERR_OOM = -3,         /* device allocation failed */
  FDTDBATH_ERR_CUDA = -4,        /* a CUDA call failed; see fdtdbath_last_error */
  FDTDBATH_ERR_NONFINITE = -5,   /* a NaN/Inf appeared in the state */
  FDTDBATH_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
  FDTDBATH_ERR_UNSUPPORTED = -7  /* valid request this build does not implement */
};

enum fdtdbath_kind {
  FDTDBATH_VACUUM = 0,
  FDTDBATH_LORENTZ = 1,       /* Eq. EOM_Lorentz */
  FDTDBATH_DRUDE = 2,         /* Eq. EOM_Lorentz with the w0^2 restoring term removed */
  FDTDBATH_LORENTZ_BATH = 3   /* Eq. EOM_LorentzBath */
};

enum fdtdbath_bath_shape { FDTDBATH_BATH_UNIFORM = 0, FDTDBATH_BATH_LORENTZIAN = 1, FDTDBATH_BATH_GAUSSIAN = 2 };

/* Field ids for read/write.  E, H, P (P^{n+1/2}) and PM (P^{n-1/2}) per component
 * c = 0,1,2; bath mode j (0 <= j < num_bath) of component c at level l (0: Y^{n+1/2},
 * 1: Y^{n-1/2}) is FDTDBATH_FIELD_Y(c, j, l). */
#define FDTDBATH_FIELD_E(c) (0 + (c))
#define FDTDBATH_FIELD_H(c) (3 + (c))
#define FDTDBATH_FIELD_P(c) (6 + (c))
#define FDTDBATH_FIELD_PM(c) (9 + (c))
#define FDTDBATH_FIELD_Y(c, j, l) (1024 + ((c) * 2 + (l)) * 256 + (j))

typedef struct fdtdbath_sim fdtdbath_sim; /* opaque, owned by the library */

typedef struct {
  int64_t n[3];      /* nx, ny, nz (each >= 1) */
  int32_t pml_cells; /* CPML planes at each z end, 0 <= pml_cells, 2*pml_cells + 2 <= nz */
} fdtdbath_grid;

/* One planar layer (Sec. III: MEEP's LorentzianSusceptibility / BathLorentzianSusceptibility
 * keywords).  For FDTDBATH_LORENTZ_BATH, gamma is gamma0 and the three bath arrays give
 * {w_j}, {gamma_j}, {k_j} (host pointers, num_bath entries each, 1 <= num_bath <= 32). */
typedef struct {
  int32_t kind;
  int64_t z_lo, z_hi;
  double eps_inf;                 /* background permittivity (> 0) */
  double frequency, gamma, sigma; /* w0/2pi, gamma/2pi, dimensionless oscillator strength */
  int32_t num_bath;
  const double *bath_frequencies;
  const double *bath_gammas;
  const double *bath_couplings;
} fdtdbath_material;

/* Soft plane source on one E component at plane z:
 *   D_c += dt * amplitude * exp(-(t-t0)^2 / (2 tau^2)) * sin(2 pi center (t - t0) + phase(x,y)),
 * tau = 1/(2 pi fwidth), evaluated at t = n dt for the update D^{n-1/2} -> D^{n+1/2}.
 * phase: host array of ny*nx radians, or NULL for zero phase. */
typedef struct {
  int32_t component;
  int64_t z;
  double center, fwidth, amplitude, t0;
  const double *phase;
} fdtdbath_source;

/* Running DFT of the plane means of Ex, Ey (plane z) and Hx, Hy (mean of planes z-1 and z):
 *   F(nu) = sum_n f(t_n) exp(+i 2 pi nu t_n) dt, with E^{n+1/2} at t = (n+1/2) dt and
 *   H^{n+1} at t = (n+1) dt.  1 <= z < nz; freqs: host array of nfreq nu-values. */
typedef struct {
  int64_t z;
  int32_t nfreq;
  const double *freqs;
} fdtdbath_monitor;

typedef struct {
  int32_t precision;    /* 64: FP64 state and arithmetic; 32: FP32 state and arithmetic */
  int32_t bath_storage; /* 0: bath modes in the state precision; 1: bf16-stored bath modes (precision 32) */
  void *cuda_stream;    /* cudaStream_t to queue work on; NULL = legacy default stream */
  /* Optional device allocator (e.g. a framework's caching allocator); NULL = cudaMalloc/cudaFree. */
  void *(*alloc)(size_t bytes, void *ctx);
  void (*free)(void *ptr, void *ctx);
  void *alloc_ctx;
  int64_t energy_lo, energy_hi; /* energy box planes [lo, hi); energy_hi <= energy_lo disables it */
  int64_t energy_capacity;      /* steps of energy trace kept on the device */
  int32_t device;               /* CUDA device ordinal */
} fdtdbath_options;

/* Build a simulation: validate (Courant <= 1/sqrt(number of axes with more than one cell),
 * 1 + gamma dt/2 > 0, layers inside the grid and disjoint, monitors and sources inside),
 * expand the per-material ADE coefficients of Eq. Pz_update-LB / Yzj_finite_difference,
 * build the CPML profiles, allocate and zero the device state.  *out receives the handle. */
int fdtdbath_create(const fdtdbath_grid *grid, double resolution, double courant,
                    const fdtdbath_material *materials, int32_t nmat,
                    const fdtdbath_source *sources, int32_t nsrc,
                    const fdtdbath_monitor *monitors, int32_t nmon,
                    const fdtdbath_options *options, fdtdbath_sim **out);

/* Advance nsteps full steps (Eq. FDTD-1D generalised to 3D: D, E, "evaluate P" with the
 * bath modes, H), asynchronously on the simulation's stream.  nsteps >= 0. */
int fdtdbath_step(fdtdbath_sim *sim, int64_t nsteps);

/* Wait for queued work; returns a deferred device error, if any. */
int fdtdbath_sync(fdtdbath_sim *sim);

/* Copy one field (see FDTDBATH_FIELD_*) as nz*ny*nx elements of the state precision
 * (float for precision 32 -- bf16 bath modes are widened -- double for 64) into dst.
 * Material-only fields read zero outside their layers.  dst_bytes must be at least
 * nz*ny*nx*element size; dst_on_device selects a device or host destination. */
int fdtdbath_read_fields(fdtdbath_sim *sim, int32_t field, void *dst, size_t dst_bytes,
                         int32_t dst_on_device);

/* Overwrite one field (same ids, layout and element type as read).  Values outside a
 * material-only field's layers are ignored.  The other canonical quantities keep their
 * values (e.g. writing P keeps P^{n-1/2}). */
int fdtdbath_write_fields(fdtdbath_sim *sim, int32_t field, const void *src, size_t src_bytes,
                          int32_t src_on_device);

/* Spectra of monitor `monitor`: host out[nfreq][4][2] = (re, im) of (Ex, Ey, Hx, Hy). */
int fdtdbath_dft(fdtdbath_sim *sim, int32_t monitor, double *out);

/* Energy trace per step (per unit transverse area, inside the energy box), host
 * trace[len][4] = (U_EM, U_P, U_bath, 0):
 *   U_EM = sum dx/(nx ny) 1/2 (eps_inf E.E + H.H) with E^{n+1/2}, H^{n+1};
 *   U_P = sum dx/(nx ny) rho/2 (((P - PM)/dt)^2 + w0^2 P^2), rho = 1/(sigma w0^2), w0 -> 0 in
 *   the potential for Drude;  U_bath = sum dx/(nx ny) sum_j rho/2 (((Y_j - Y_j')/dt)^2 + w_j^2 Y_j^2)
 * (the energy density of Eq. H_full with P and Y_j as coordinates).  *len = steps written. */
int fdtdbath_energy(fdtdbath_sim *sim, double *trace, int64_t maxlen, int64_t *len);

/* Completed steps. */
int64_t fdtdbath_steps_done(const fdtdbath_sim *sim);

/* Text of the last error of sim (or of the last failed create when sim is NULL). */
const char *fdtdbath_last_error(const fdtdbath_sim *sim);

void fdtdbath_destroy(fdtdbath_sim *sim);

/* Table I: expand a bath_form into explicit arrays (host, num_bath >= 2 entries each).
 * frequencies evenly spaced over frequency +/- width/2; gammas = bath_gamma; couplings
 * k_b = sqrt(2 dw/pi * dephasing), dw = width/(num_bath-1), times sqrt(G^2/(G^2+(w_j-w0)^2))
 * (lorentzian) or exp(-(w_j-w0)^2/(4 G^2)) (gaussian), G = gamma + dephasing. */
int fdtdbath_bath_form(int32_t shape, double frequency, double gamma, int32_t num_bath,
                       double width, double bath_gamma, double dephasing, double *frequencies,
                       double *gammas, double *couplings);

/* Runtime facts of a simulation: key 0 element size of the state, 1 kernel launches issued
 * so far, 2 bytes of device memory held, 3 blocks of the 3D step kernel, 4 z-chunks. */
int64_t fdtdbath_query(const fdtdbath_sim *sim, int32_t key);

/* Energy (U_EM, U_P, U_bath) of planes z_lo <= k < z_hi of the current state -- the same
 * quantities and weights as one fdtdbath_energy() entry -- computed WITHOUT allocating memory.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate device
 * memory when they need the result (code running inside a stream capture, a real-time loop that
 * forbids allocation, a host framework that owns the whole memory pool).  Its scratch space is a
 * static device array of this library holding one partial sum per plane: boxes deeper than 4096
 * planes are rejected with FDTDBATH_ERR_ARG.  out receives 3 doubles, in device memory when
 * out_on_device is nonzero, else in host memory; the call waits for the simulation's stream.
 * The first call on a device looks the array's address up (a host-side runtime call), so make
 * it before any stream capture on that device.  All calls on a device share the array: calls
 * that overlap on the GPU (e.g. from two streams) race and must be serialized by the caller. */
int fdtdbath_box_energy_noalloc(fdtdbath_sim *sim, int64_t z_lo, int64_t z_hi, double *out,
                                int32_t out_on_device);

#ifdef __cplusplus
}
#endif

#endif /* FDTDBATH_H */
