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

#define FDTDBATH_ABI_VERSION 3   /* 3: snapshot / restore, FMA-rate measurement; 2: batch_plan takes block_threads */

enum fdtdbath_status {
  FDTDBATH_OK = 0,
  FDTDBATH_ERR_ARG = -1,         /* malformed argument */
  FDTDBATH_ERR_CFL = -2,         /* unstable time step (Courant or oscillator update) */
  FDTDBATH_ERR_OOM = -3,         /* device allocation failed */
  FDTDBATH_ERR_CUDA = -4,        /* a CUDA call failed; see fdtdbath_last_error */
  FDTDBATH_ERR_NONFINITE = -5,   /* a NaN/Inf in the spectra or energy trace read out */
  FDTDBATH_ERR_TIMEOUT = -6,     /* a kernel's bounded (1 s) wait for its staged planes ran out;
                                  * returned by fdtdbath_sync / dft / energy, results invalid */
  FDTDBATH_ERR_UNSUPPORTED = -7  /* valid request the library does not implement */
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
/* The per-cell oscillator strength sigma(r) of Eq. EOM_Lorentz and EOM_LorentzBath-1 (the paper
 * lets sigma depend on position; rho(r) = 1/(sigma(r) w0^2) weighs the energy of Eq. H_full).  One
 * value per cell (i, j, k), shared by the three components of that cell.  Reading it returns the
 * map where one is set, each dispersive layer's own sigma otherwise, and zero outside the Lorentz,
 * Drude and Lorentz-Bath layers.  Writing it sets the map of every such layer (values elsewhere
 * are ignored): FDTDBATH_ERR_ARG for a negative or non-finite value, FDTDBATH_ERR_CFL (nothing
 * changed) when a layer would be unstable at its largest sigma(r) (the bound of fdtdbath_create
 * with that sigma).  The map takes 4 (FP32) or 8 (FP64) bytes per layer cell, read once per step
 * by the step kernels (the TE form's register-streaming kernel leaves its chunks to the general
 * kernel while a map is set); the adjoint and fdtdbath_box_energy_noalloc answer
 * FDTDBATH_ERR_UNSUPPORTED, and a snapshot carries the map. */
#define FDTDBATH_FIELD_SIGMA 12

typedef struct fdtdbath_sim fdtdbath_sim; /* opaque, owned by the library */

typedef struct {
  int64_t n[3];      /* nx, ny, nz (each >= 1) */
  int32_t pml_cells; /* CPML planes at each z end, 0 <= pml_cells, 2*pml_cells + 2 <= nz */
} fdtdbath_grid;

/* One planar layer (Sec. III: MEEP's LorentzianSusceptibility / BathLorentzianSusceptibility
 * keywords).  For FDTDBATH_LORENTZ_BATH, gamma is gamma0 and the three bath arrays give
 * {w_j}, {gamma_j}, {k_j} (host pointers, num_bath entries each, 1 <= num_bath <= 128; the
 * paper's Fig. 2 baths have 100).  Up to 32 modes the step kernel keeps a cell's modes in
 * registers, above it streams them from memory; the batch form keeps every mode in shared
 * memory (up to 128 as well); the adjoint takes at most 32 (FDTDBATH_ERR_UNSUPPORTED). */
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
  int32_t bath_storage; /* 0: bath modes in the state precision.  1 (precision 32 only): every bath
                         * mode stored as a bf16 pair in one 32-bit word -- its value Y^{n+1/2} and
                         * its increment Y^{n+1/2} - Y^{n-1/2} -- updated in place with FP32 arithmetic (8 bytes per
                         * mode and component per step instead of 12); reading level 1 returns
                         * value - increment.  fdtdbath_box_energy_noalloc refuses such simulations
                         * with FDTDBATH_ERR_UNSUPPORTED. */
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
 * build the CPML profiles, allocate and zero the device state.  *out receives the handle.
 * The kernels index the state with 32-bit offsets: a grid whose E / H arrays (3 nx ny nz), pooled
 * polarization (3 x the layer cells), bath-mode array or CPML memories would exceed 2^31 - 1
 * elements (e.g. 1024^3) is refused with FDTDBATH_ERR_ARG. */
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

/* Paint an axis-aligned box of oscillator strength sigma into the sigma(r) map (see
 * FDTDBATH_FIELD_SIGMA) with sub-pixel averaging.  lo, hi: host arrays (x, y, z) in cell units,
 * 0 <= lo < hi <= n on every axis (FDTDBATH_ERR_ARG otherwise); cell (i, j, k) is the unit cube
 * [i, i+1) x [j, j+1) x [k, k+1).  A dispersive-layer cell that the box covers by the fraction f
 * (the product of its overlap lengths along the three axes) takes
 *     sigma(r) <- f sigma + (1 - f) sigma(r),
 * the cell average of the coupling strength (the susceptibility of Eq. chi_L is linear in sigma,
 * so this is the average susceptibility of the cell's two parts).  Cells outside the dispersive
 * layers are left alone; eps_inf is not averaged.  Validation and errors as for writing
 * FDTDBATH_FIELD_SIGMA; synchronizes the simulation's stream. */
int fdtdbath_sigma_box(fdtdbath_sim *sim, const double lo[3], const double hi[3], double sigma);

/* Spectra of monitor `monitor`: host out[nfreq][4][2] = (re, im) of (Ex, Ey, Hx, Hy).
 * FDTDBATH_ERR_NONFINITE (out filled all the same) when a value is NaN or Inf. */
int fdtdbath_dft(fdtdbath_sim *sim, int32_t monitor, double *out);

/* Energy trace per step (per unit transverse area, inside the energy box), host
 * trace[len][4] = (U_EM, U_P, U_bath, 0):
 *   U_EM = sum dx/(nx ny) 1/2 (eps_inf E.E + H.H) with E^{n+1/2}, H^{n+1};
 *   U_P = sum dx/(nx ny) rho/2 (((P - PM)/dt)^2 + w0^2 P^2), rho = 1/(sigma(r) w0^2), w0 -> 0 in
 *   the potential for Drude;  U_bath = sum dx/(nx ny) sum_j rho/2 (((Y_j - Y_j')/dt)^2 + w_j^2 Y_j^2)
 * (the energy density of Eq. H_full with P and Y_j as coordinates).  *len = steps written.
 * FDTDBATH_ERR_NONFINITE (trace and *len filled all the same) when a record is NaN or Inf. */
int fdtdbath_energy(fdtdbath_sim *sim, double *trace, int64_t maxlen, int64_t *len);

/* Completed steps. */
int64_t fdtdbath_steps_done(const fdtdbath_sim *sim);

/* Checkpoint / resume of the whole state: every quantity the following steps read (E^{n-1/2},
 * H, the CPML memories of both half-steps, D in FP64, both time levels of P and of every bath
 * mode of Eq. Pz_update-LB / Yzj_finite_difference), the running DFT accumulators of every
 * monitor, the energy trace and the step count.  The H half-step of the last step, which the
 * library computes in the launch of the next step, stays pending: the snapshot holds H^{n-1} and
 * the partial sums of step n-1, so a simulation restored from it -- the same one later, or a fresh
 * one created with the same arguments -- runs the very launches the original would have and
 * continues bit for bit (on the same device and library).
 * The snapshot is an opaque byte string of fdtdbath_snapshot_size bytes (a header, then the
 * device state), written to dst in host or device memory.  fdtdbath_restore checks that the
 * snapshot comes from a simulation of the same layout (grid, CPML, precision, bath storage,
 * material cells and modes, monitors, energy capacity; FDTDBATH_ERR_ARG otherwise) and replaces
 * this simulation's state, its sigma(r) map included (a snapshot taken without a map returns the
 * layers to their own sigma); a recorded adjoint forward run is discarded.  Both synchronize the
 * simulation's stream. */
int fdtdbath_snapshot_size(fdtdbath_sim *sim, size_t *bytes);
int fdtdbath_snapshot(fdtdbath_sim *sim, void *dst, size_t dst_bytes, int32_t dst_on_device);
int fdtdbath_restore(fdtdbath_sim *sim, const void *src, size_t src_bytes, int32_t src_on_device);

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
 * so far, 2 bytes of device memory held, 3 blocks of the 3D step kernel, 4 z-chunks, 5 whether
 * the step kernel runs the TE form (1) or the general form (0).  The TE form is taken by a
 * y-invariant grid (ny = 1) whose sources all drive E_y (Sec. II.C, the 2D case): E_x, E_z, H_y,
 * P_x, P_z and the x / z bath modes then stay exactly zero and are neither read nor written; the
 * live components are bit-identical to the general form's.  A write_fields call on any of those
 * components returns the simulation to the general form for good.  Key 6: whether the last
 * fdtdbath_adjoint_backward ran the TE form of the reverse sweep (a TE forward run and dL_dF zero
 * for the E_x and H_y spectra).  Key 7: whether the z-chunks without bath modes run the
 * plain-plane kernel (grids of at least 8 rows tiled exactly by its 128 x 8 FP32 or 64 x 8 FP64
 * tiles, ny a multiple of 8, no source plane inside a layer) instead of the general kernel.
 * Key 8: whether the steps run on the persistent 1D cavity kernel (nx = ny = 1, at most one
 * source and one monitor, at most 32 bath modes per material, x polarization only).  Key 9:
 * whether the z-chunks with bath modes run the plain-plane kernel's Lorentz-Bath form (FP32; at
 * most 16 bath modes per material with FP32 or bf16 bath storage, or up to 128 with FP32
 * storage; at most two Lorentz-Bath layers; nx a multiple of 32, ny of 8, no source plane inside a
 * layer).  Key 10: whether the z-chunks of a simulation in the TE form run the TE form's
 * register-streaming kernel (FP32, nx a multiple of 256, no source plane inside a layer; the
 * chunks with bath modes only with FP32 bath storage and at most 8 modes per material).  Key 11:
 * whether a per-cell sigma(r) map is set (FDTDBATH_FIELD_SIGMA).  Key 12: whether pairs of steps
 * run as one launch of the two-steps-per-pass kernel (temporal blocking; taken when the
 * environment variable FDTDBATH_TB=1 is set at creation, on grids without materials, of at least
 * 8 rows, nx a multiple of 32 and ny of 8): fdtdbath_step then advances the state two steps per
 * launch (a single step where one is left over or no H half-step is pending), with the same
 * results -- FP64 state bit for bit -- as single steps. */
int64_t fdtdbath_query(const fdtdbath_sim *sim, int32_t key);

/* Energy (U_EM, U_P, U_bath) of planes z_lo <= k < z_hi of the current state -- the same
 * quantities and weights as one fdtdbath_energy() entry -- computed WITHOUT allocating memory.
 * The paper has no counterpart.  It serves callers that may not allocate device memory at the
 * moment they need the result: a real-time or latency-bound loop (a cudaMalloc can synchronize
 * the device and take unbounded time), a host framework that owns the whole device memory pool
 * and gives this library only the simulation's own buffers, or a process held to a fixed
 * device-memory budget.  Its scratch space is a static device array of this library holding one
 * partial sum per plane: boxes deeper than 4096 planes are rejected with FDTDBATH_ERR_ARG.  out
 * receives 3 doubles, in device memory when out_on_device is nonzero, else in host memory.  The
 * call may first launch the simulation's pending H half-step, and it waits for the simulation's
 * stream before returning.  The first call on a device looks the array's address up (a
 * host-side runtime call, then cached for that device for the life of the process, so the entry
 * point must not be used on a device after cudaDeviceReset); make that first call before any
 * stream capture on the device.  All calls on a device share the array, which keeps the last
 * call's contents: calls that overlap on the GPU (e.g. from two streams) race and must be
 * serialized by the caller. */
int fdtdbath_box_energy_noalloc(fdtdbath_sim *sim, int64_t z_lo, int64_t z_hi, double *out,
                                int32_t out_on_device);

/* Measured fused-multiply-add throughput of the device (flops per second, 2 per FMA) in FP32 or
 * FP64: the best of reps timed launches of independent FMA chains on every SM (CUDA events; no
 * clock or power setting is touched).  The paper has no counterpart: it is the arithmetic ceiling
 * of the step kernels' roofline (the FP64 step is bound by FP64 arithmetic on this part).
 * Allocates a few KB of device memory for the duration of the call. */
int fdtdbath_measure_fma_rate(int32_t precision, int32_t device, int32_t reps, double *flops_per_s);

/* ---------------------------------------------------------------------------------------------
 * Discrete adjoint (differentiation form).  The gradient of a scalar loss L of one monitor's
 * spectra with respect to the oscillator parameters of one layer -- sigma, gamma (gamma0 of a
 * Lorentz-Bath layer) and every bath coupling k_j, in the nu-units of fdtdbath_material -- by the
 * exact transpose of the discrete step (the reverse-time adjoint of Eq. FDTD-1D generalised to the
 * Yee grid with Eq. Pz_update-LB and Yzj_finite_difference), with checkpointing: the forward run
 * keeps a full state every checkpoint_every steps; the reverse sweep recomputes one segment at a
 * time from its checkpoint, recording the layer's E, P and bath modes, and walks it backwards.
 * Device memory: one state per checkpoint, plus the adjoint state and the records of one segment
 * (checkpoint_every + 2 steps of the layer's E, P and bath modes).
 * --------------------------------------------------------------------------------------------- */

/* Advance nsteps steps (as fdtdbath_step), saving the checkpoints of the run; the spectra and
 * energy traces accumulate as usual.  Not available with bf16 bath storage, with more than 32
 * bath modes in a material or with a sigma(r) map (FDTDBATH_ERR_UNSUPPORTED).  A later fdtdbath_step invalidates the recording. */
int fdtdbath_adjoint_forward(fdtdbath_sim *sim, int64_t nsteps, int32_t checkpoint_every);

/* Reverse sweep of the recorded run.  dL_dF: host array nfreq x 4 x 2 with dL/dRe and dL/dIm of
 * the monitor's spectra in the layout of fdtdbath_dft (Ex, Ey, Hx, Hy).  material: index of the
 * layer in the list given to fdtdbath_create (not vacuum).  grad receives 2 + num_bath doubles:
 * dL/dsigma, dL/dgamma, dL/dcoupling_j.  The simulation is left in the state at the end of the
 * recorded run (spectra unchanged). */
int fdtdbath_adjoint_backward(fdtdbath_sim *sim, int32_t monitor, const double *dL_dF, int32_t material,
                              double *grad);

/* ---------------------------------------------------------------------------------------------
 * Batched 1D cavities.  Many independent 1D cavities (nx = ny = 1, x polarization: E_x, H_y, P_x
 * and its bath modes) of uneven length, each advanced by the same scheme as fdtdbath_create /
 * fdtdbath_step (Eq. FDTD-1D with Eq. Pz_update-LB, Pz_1D_Lorentz, Yzj_finite_difference; the
 * Rabi-splitting and bath-parameter sweeps of Sec. IV run one cavity per parameter set), all
 * cavities in ONE persistent launch per chunk of steps.  The library packs the cavities over the
 * thread-block clusters of that launch (whole cavities per cluster, contiguous cell ranges per
 * CTA, the state held in shared memory for the whole chunk), picks the launch shape with its own
 * autotuner unless the options fix it, and replays the chunks from captured CUDA graphs.
 * --------------------------------------------------------------------------------------------- */
typedef struct fdtdbath_batch fdtdbath_batch; /* opaque, owned by the library */

/* One cavity: nz cells (64 <= nz <= 2^24) with a CPML of pml_cells cells at each end, its layers
 * (z in the cavity's own cells, the same rules as fdtdbath_create, at most 128 bath modes per
 * layer), an optional soft source on
 * component 0 (E_x; phase NULL or one value) and an optional energy box [energy_lo, energy_hi)
 * (energy_hi <= energy_lo: none).  Host pointers, copied by fdtdbath_batch_create. */
typedef struct {
  int64_t nz;
  int32_t pml_cells;
  const fdtdbath_material *materials;
  int32_t nmat;
  const fdtdbath_source *source;
  int64_t energy_lo, energy_hi;
} fdtdbath_cavity;

typedef struct {
  int32_t precision;       /* 32: FP32 state, increment arithmetic; 64: FP64, the literal updates */
  void *cuda_stream;       /* cudaStream_t to queue work on; NULL = legacy default stream */
  void *(*alloc)(size_t bytes, void *ctx);   /* optional device allocator, as fdtdbath_options */
  void (*free)(void *ptr, void *ctx);
  void *alloc_ctx;
  int32_t energy_every;    /* record the cavities' energies every this many steps (0 or 1: each) */
  int64_t energy_capacity; /* records kept per cavity (0: 65536); later records are dropped */
  int32_t cluster_ctas;    /* launch shape: CTAs per cluster (1..16) and threads per CTA (a */
  int32_t block_threads;   /* multiple of 32, <= 1024); 0 = chosen by the autotuner at the first step */
  int32_t use_graph;       /* nonzero: replay each chunk of steps from a captured CUDA graph */
  int32_t device;          /* CUDA device ordinal */
} fdtdbath_batch_options;

/* Validate every cavity (errors name the cavity), expand its coefficients exactly as
 * fdtdbath_create does, tabulate each source's amplitude per step (until the Gaussian envelope
 * underflows to exactly zero), allocate and zero the state.  resolution and courant are shared
 * by the batch (dt = courant/resolution).  *out receives the handle. */
int fdtdbath_batch_create(const fdtdbath_cavity *cavities, int32_t ncav, double resolution, double courant,
                          const fdtdbath_batch_options *options, fdtdbath_batch **out);

/* Autotuner: time probe_steps steps of every feasible launch shape (CTAs per cluster in
 * {1,2,4,8,16} x threads in {128,256,512,1024} x 1 or 2 CTAs per SM, each packed for this batch) and
 * keep the fastest; the state is restored afterwards.  Outputs (optional) receive the shape and
 * its time per step in milliseconds.  fdtdbath_batch_step runs it with 64 probe steps when no
 * shape has been chosen yet. */
int fdtdbath_batch_autotune(fdtdbath_batch *batch, int32_t probe_steps, int32_t *cluster_ctas,
                            int32_t *block_threads, float *ms_per_step);

/* Advance every cavity nsteps steps, asynchronously on the batch's stream: chunks of
 * 1024 * energy_every steps (4096 without energy boxes), each one launch of the batch kernel
 * plus the energy reduction, replayed from a CUDA graph when use_graph is set. */
int fdtdbath_batch_step(fdtdbath_batch *batch, int64_t nsteps);

/* Wait for queued work; returns a deferred device error, if any. */
int fdtdbath_batch_sync(fdtdbath_batch *batch);

/* Copy one field of one cavity, nz elements of the state type (float / double), into host dst:
 * FDTDBATH_FIELD_E(0), FDTDBATH_FIELD_H(1), FDTDBATH_FIELD_P(0), FDTDBATH_FIELD_PM(0) or
 * FDTDBATH_FIELD_Y(0, j, l) (zero outside the cavity's Lorentz-Bath layers).  Other ids:
 * FDTDBATH_ERR_ARG.  Synchronizes the batch's stream. */
int fdtdbath_batch_read_field(fdtdbath_batch *batch, int32_t cavity, int32_t field, void *dst,
                              size_t dst_bytes);

/* Energy records of one cavity, host trace[len][4] = (U_EM, U_P, U_bath, 0) with the
 * definitions of fdtdbath_energy (dx weight), record r describing step r * energy_every.
 * *len = records available (at most maxlen and energy_capacity). */
int fdtdbath_batch_energy(fdtdbath_batch *batch, int32_t cavity, double *trace, int64_t maxlen, int64_t *len);

/* Runtime facts: key 0 kernel launches, 1 clusters, 2 CTAs, 3 CTAs per cluster, 4 threads per
 * CTA, 5 device bytes held, 6 graph replays, 7 completed steps, 8 dynamic shared memory per CTA,
 * 9 total cells.  -1 for an unknown key. */
int64_t fdtdbath_batch_query(const fdtdbath_batch *batch, int32_t key);

/* Text of the last error of batch (or of the last failed batch create / plan when NULL). */
const char *fdtdbath_batch_last_error(const fdtdbath_batch *batch);

void fdtdbath_batch_destroy(fdtdbath_batch *batch);

/* Host-only planning (no GPU needed): pack the cavities for cluster_ctas CTAs of block_threads
 * threads (1..1024) per cluster, at most nclusters clusters and smem_per_cta bytes of dynamic
 * shared memory per CTA.  The packer bounds the work of the busiest thread (cell l of a CTA is
 * thread l mod block_threads's); block_threads = 1 balances whole CTAs.  Returns the number of
 * CTAs (nclusters_used * cluster_ctas, cluster-major) or a negative error; the optional outputs
 * receive per CTA its work units, cells and shared-memory bytes, and per cavity its cluster. */
int fdtdbath_batch_plan(const fdtdbath_cavity *cavities, int32_t ncav, double resolution, double courant,
                        int32_t precision, int32_t cluster_ctas, int32_t block_threads, int32_t nclusters,
                        int32_t smem_per_cta, int64_t *cta_work, int32_t *cta_ncell, int32_t *cta_smem,
                        int32_t *cav_cluster);

#ifdef __cplusplus
}
#endif

#endif /* FDTDBATH_H */
