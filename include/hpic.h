/*
 * hpic.h -- C-ABI of the GB300 fast-electron hybrid-PIC step.
 *
 * Method: Morris, Robinson & Ridgers, "Highly efficient conversion of laser
 * energy to hard X-rays in high intensity laser-solid simulations",
 * arXiv 2107.01723.  One step advances the hot electrons of one target
 * through the resistive fields of the cold solid and updates the solid:
 *   - relativistic push in E, B (Lorentz force; Sec. III.B, field loss),
 *   - ionisation drag, Eq. (5) (Sec. III.B),
 *   - Davies elastic scatter, Eq. (B4) (App. B),
 *   - optical-depth bremsstrahlung emission with photon tallies (App. B),
 *   - escape / reflux at the target faces (Sec. II.A, Table I),
 *   - hot-electron current deposit and the hybrid field solve
 *     E = eta (curl B / mu0 - j_h), dB/dt = -curl E, Eqs. (A1)-(A3),
 *   - Ohmic + ionisation heating, Eqs. (A7)-(A8), and the resistivity
 *     eta(T) of Eqs. (A4)-(A6),
 *   - injection of new hot electrons, Eq. (B1) and Sec. II.B.
 *
 * Conventions for every function:
 *   - Returns an hpic_status (0 = success).  Nothing aborts or throws across
 *     this boundary.  On failure hpic_last_error() describes the cause.
 *   - Host pointers are caller-owned; the library copies what it needs and
 *     keeps no host pointer after a call returns.  All device memory is
 *     allocated, owned and freed by the library.
 *   - All work is enqueued on the context's CUDA stream (the one passed at
 *     creation, or the legacy default stream if NULL).  hpic_step returns
 *     once the work is enqueued; every hpic_read_* call synchronises that
 *     stream before it returns.
 *   - A context may be used from one host thread at a time.
 *   - Units are SI at the interface (m, s, J, K, V/m, T, A/m^2, Ohm m),
 *     except particle momentum, given as u = p / (m_e c).
 *
 * Grid layout (Yee staggering, the reading used throughout): the target is
 * nx*ny*nz cubic cells of side dx.  Each vector component (E, B, j_h) is an
 * (nx+1)*(ny+1)*(nz+1) array of doubles, index i + (nx+1)*(j + (ny+1)*k),
 * located at (in cells) Ex (i+1/2, j, k), Ey (i, j+1/2, k), Ez (i, j, k+1/2),
 * Bx (i, j+1/2, k+1/2), By (i+1/2, j, k+1/2), Bz (i+1/2, j+1/2, k); entries
 * beyond a staggered extent are padding (zero).  Cell scalars (T, eta, drag
 * heat) are nx*ny*nz doubles, index i + nx*(j + ny*k).
 */
#ifndef HPIC_H
#define HPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HPIC_OK = 0,
  HPIC_EINVAL = -1,    /* an argument is out of range or inconsistent */
  HPIC_ENOMEM = -2,    /* a device or host allocation failed */
  HPIC_ECUDA = -3,     /* a CUDA call failed (message in hpic_last_error) */
  HPIC_ETIMEOUT = -4,  /* a bounded device wait gave up */
  HPIC_ESTATE = -5,    /* call not allowed in the context's current state */
  HPIC_ENONFINITE = -6 /* non-finite particle state was found and removed */
} hpic_status;

typedef enum { HPIC_FP64 = 0, HPIC_FP32_MIXED = 1 } hpic_precision;

/* physics switches for hpic_run_params.physics (bitmask) */
enum {
  HPIC_DRAG = 1,     /* ionisation drag, Eq. (5) */
  HPIC_SCATTER = 2,  /* Davies scatter, Eq. (B4) */
  HPIC_BREM = 4,     /* bremsstrahlung emission, App. B */
  HPIC_FIELDS = 8,   /* E from Eq. (A2) every step (else E is held) */
  HPIC_FARADAY = 16, /* B from Eq. (A3) every step (else B is held: the
                        paper's B = 0 test, Sec. III.A) */
  HPIC_HEATING = 32, /* T and eta update, Eqs. (A4)-(A8) */
  HPIC_ALL = 63,
  /* unbounded uniform medium: no field gather, no faces, nothing deposited
   * on the grid; drag, scatter and emission only (the emission benchmark) */
  HPIC_UNBOUNDED = 64,
  /* ionised-screening enhancement of the bremsstrahlung cross section,
   * F_sigma = 1 + ln(lambda_D/a_s) / ln(a_s m_e c/hbar) (Zstar/Z)^2 (App. B),
   * from the ion temperature of the electron's cell; lambda_D is the ion
   * Debye length, a_s = 1.4 a_B Z^(-1/3) */
  HPIC_FSIGMA = 128,
  /* electron-ion temperature equilibration (App. A): T_i is evolved and
   * relaxes with T_e at the rates Z*^2 e^4 n_i / t_c (electrons) and
   * Z*^3 e^4 n_i / t_c (ions), integrated exactly over each step with the
   * rates frozen at the start of the exchange */
  HPIC_EI_EQUIL = 256
};

/* grid codes for hpic_read_grid / hpic_write_grid */
enum {
  HPIC_GRID_T = 0, HPIC_GRID_ETA = 1,
  HPIC_GRID_EX = 2, HPIC_GRID_EY = 3, HPIC_GRID_EZ = 4,
  HPIC_GRID_BX = 5, HPIC_GRID_BY = 6, HPIC_GRID_BZ = 7,
  HPIC_GRID_JX = 8, HPIC_GRID_JY = 9, HPIC_GRID_JZ = 10,
  HPIC_GRID_HEAT = 11, /* drag heat (J) deposited per cell in the last step */
  HPIC_GRID_TI = 12    /* ion temperature (K), cell-centred */
};

/* One more element sharing every cell of a compound target (App. A). */
typedef struct {
  double Z, n_i_m3, I_ex_J, Zstar, A_ion;
} hpic_solid;

/* One target: a uniform solid filling the box (App. A): one element, or a
 * compound of it and up to three more (n_extra; e.g. CH plastic).  For a
 * compound the heating of Eq. (A7) uses n_e = sum Z n_i and the n_e-weighted
 * mean of 1/C (the paper's rule); the ionisation and bremsstrahlung stopping
 * powers and the emission rate add over the elements, the Davies scatter
 * variances add, and eta of Eqs. (A4)-(A6) takes sum Z* n_i, sum Z*^2 n_i and
 * the total ion density.  Compounds do not combine with HPIC_FSIGMA or
 * HPIC_EI_EQUIL. */
typedef struct {
  int32_t nx, ny, nz;   /* cells, each >= 2 */
  double dx_m;          /* cell side; must exceed c * dt */
  double Z;             /* atomic number */
  double n_i_m3;        /* ion number density */
  double I_ex_J;        /* mean excitation energy (the paper uses 11 eV * Z) */
  double Zstar;         /* ionisation state in eta, Eq. (A4) */
  double lnLambda;      /* Coulomb logarithm in Eq. (A5) */
  double eta_max_ohm_m; /* cap on eta */
  double lambda1;       /* cold-limit factor of Eq. (A6); 0 drops that limit */
  double lambda2;       /* multiplier on eta (App. A) */
  double T0_K;          /* initial background temperature (electrons and ions) */
  double A_ion;         /* ion mass in atomic mass units (e-i equilibration) */
  int32_t n_extra;      /* further elements of a compound, 0..3 */
  int32_t pad;
  hpic_solid extra[3];
} hpic_target_desc;

/* Laser and injection, Eq. (1), Eq. (B1), Sec. II.B and App. B.
 *
 * HPIC_ENV_FLAT: flat-top envelopes, a disc of radius spot_radius_m centred
 * at (0, spot_y, spot_z) for t < t_inj_s; n_macro electrons in all, each of
 * the weight N_real/n_macro of Eq. (B1).
 *
 * HPIC_ENV_GAUSS (the paper's own): f(r) = exp(-4 ln2 r^2/r_fwhm^2) at the
 * centre of each x = 0 face cell (r from the spot centre) and g(t) =
 * exp(-4 ln2 (t - t_pk)^2/t_fwhm^2) at mid-step t = (s + 1/2) dt, t_pk set so
 * that g(0) = g_min.  While g >= g_min every face cell with f >= f_min
 * injects per_cell macro-electrons per step, uniform over the cell's face,
 * each carrying its own weight N_cell/per_cell with N_cell = I0 f g dx^2 dt
 * eta_l2e / <eps> and the local mean energy <eps> = a0 sqrt(f g) m_e c^2
 * (Eq. (N_cell)); spot_radius_m, t_inj_s and n_macro are unused.
 *
 * Either way energies are exponential with the (local) mean and directions
 * uniform in solid angle inside the cone, whose half-angle is, with
 * moore_cap, the smaller of cone_half_angle_rad and atan(sqrt(2/(gamma-1)))
 * for each electron (Sec. II.B). */
enum { HPIC_ENV_FLAT = 0, HPIC_ENV_GAUSS = 1 };
typedef struct {
  double I0_Wm2;        /* peak intensity, W m^-2 (1e20 W/cm^2 = 1e24) */
  double lambda_m;      /* wavelength */
  double eta_l2e;       /* laser -> hot electron energy efficiency */
  double spot_radius_m;
  double spot_y_m, spot_z_m;
  double t_inj_s;       /* injection window */
  double cone_half_angle_rad; /* uniform in solid angle within this cone */
  int64_t n_macro;      /* macro-electrons over the whole window (< 2^32-1) */
  int32_t envelope;     /* HPIC_ENV_FLAT or HPIC_ENV_GAUSS */
  int32_t per_cell;     /* Gaussian: macro-electrons per injecting cell per step */
  double r_fwhm_m, t_fwhm_s; /* Gaussian: radial and temporal FWHM */
  double f_min, g_min;  /* Gaussian: inject where f >= f_min and g >= g_min */
  int32_t moore_cap;    /* 1: Moore-scaling cap on the cone half-angle */
  int32_t pad;
} hpic_laser_desc;

typedef struct {
  double dt_s;          /* time step */
  uint64_t seed;        /* Philox4x32-10 key */
  uint32_t target_index;/* fourth Philox counter word */
  int32_t precision;    /* hpic_precision */
  double kappa_esc;     /* escape energy kappa_esc a0 m_e c^2 (Sec. II.A) */
  double kappa_tnsa;    /* reflux |p| loss kappa_tnsa a0 m_e c (Sec. II.A) */
  double sigma_dtheta_rad; /* reflux scatter range +-sigma/2 (Sec. II.A) */
  double brem_boost;    /* cross-section boost B; photon weight w/B (Sec. II.B) */
  double k_min_J;       /* lowest photon energy modelled */
  double E_cut_J;       /* tracking cut: electrons below it are absorbed */
  int32_t n_Ebins, n_thbins; /* photon tally: log energy x polar angle */
  double tally_Emin_J, tally_Emax_J;
  double ce_threshold_J;/* X-ray threshold (1 MeV in the paper) */
  int32_t table_rows, table_cols; /* inverse-CDF photon table */
  double table_Emax_J;  /* top electron energy of the table */
  int32_t curlB_term;   /* 1: E = eta(curl B/mu0 - j_h) (Eq. A2); 0: E = -eta j_h */
  int32_t physics;      /* HPIC_* bitmask */
  int32_t sort_interval;/* cell sort inside every sort_interval-th step of
                           hpic_step (0 = never): the step writes the electrons
                           in the order of the cell each reaches
                           (sort_interval + 1)/2 steps after it at its
                           velocity (clamped to the grid), the middle of the
                           steps that order serves */
  int32_t max_history;  /* length of the per-step X-ray history */
} hpic_run_params;

/* Energy-budget and event tallies (all FP64).  Budget identity, closed by
 * construction: E_injected = E_live + W_field + E_drag + E_xray
 *                            + E_escaped + E_reflux. */
typedef struct {
  double E_injected, N_injected; /* injected energy (J) and real electrons */
  double W_field;       /* energy lost by electrons to E (J; gain < 0) */
  double E_drag;        /* ionisation heat incl. absorbed electrons (J) */
  double E_xray;        /* photon energy, all k >= k_min (J) */
  double E_xray_above;  /* photon energy with k >= ce_threshold (J) */
  double E_escaped;     /* energy of escaped electrons (J) */
  double E_reflux;      /* energy lost in reflux events (J) */
  double E_ohmic_grid;  /* sum eta j_h.j_h dt V over cells and steps (J) */
  double n_injected, n_escaped, n_refluxed, n_reflux_absorbed;
  double n_cut, n_emitted, particle_steps;
  double n_nonfinite;   /* particles removed for non-finite state */
  double E_live;        /* kinetic energy of live electrons now (J) */
  double E_B_field;     /* magnetic energy sum B^2/(2 mu0) V now (J) */
} hpic_tallies;

typedef struct hpic_ctx hpic_ctx;
typedef struct hpic_batch hpic_batch;

/* Create a context for one target on `device`, with work on `cuda_stream`
 * (a cudaStream_t, or NULL).  Builds the photon inverse-CDF table on the
 * device, sets T = T0 and eta = eta(T0) everywhere, E = B = 0, no electrons.
 * Errors: HPIC_EINVAL (dx <= c dt, a dimension < 2, bad bins or table),
 * HPIC_ENOMEM, HPIC_ECUDA.  *out is NULL on failure. */
int hpic_init_target(hpic_ctx **out, const hpic_target_desc *target,
                     const hpic_run_params *run, int device, void *cuda_stream);

/* Schedule injection (Eq. (B1), Sec. II.B): step s < t_inj/dt injects
 * floor((s+1) N/S) - floor(s N/S) electrons at x = 1e-6 dx, with energies
 * exponential of mean a0 m_e c^2, disc positions and cone directions
 * uniform; they first move in the next step.  Reserves device room for
 * n_macro more electrons.  Errors: HPIC_EINVAL, HPIC_ENOMEM, HPIC_ESTATE
 * (a laser was already scheduled). */
int hpic_inject_electrons(hpic_ctx *ctx, const hpic_laser_desc *laser);

/* Append n electrons uniform in the box, with directions uniform on the
 * sphere, kinetic energies exponential with mean mean_energy_J and fresh
 * optical depths (Philox blocks 10 and 11 at the current step; ids from the
 * id counter; weight: the laser's macro weight, or 1 without a laser).  The
 * bulk initial state of the emission benchmark.  Errors: HPIC_EINVAL,
 * HPIC_ENOMEM, HPIC_ECUDA. */
int hpic_seed_electrons(hpic_ctx *ctx, int64_t n, double mean_energy_J);

/* Advance n_steps >= 0 steps (asynchronous).  Errors: HPIC_EINVAL, HPIC_ECUDA. */
int hpic_step(hpic_ctx *ctx, int64_t n_steps);

/* Counting sort of the electrons by the cell they are in (4x4x4 cell tiles,
 * x-fastest); drops absorbed/escaped slots.  The sort inside every
 * sort_interval-th step of hpic_step is folded into that step: its keys come
 * from the state at the start of the step, one step further ahead, and the
 * push writes each electron to its sorted slot (the order only; electrons
 * absorbed or escaping in that step leave their slots there marked dead
 * until the next sort).  Asynchronous. */
int hpic_sort(hpic_ctx *ctx);

/* Tallies accumulated since creation or the last reset (synchronises). */
int hpic_read_tallies(hpic_ctx *ctx, hpic_tallies *out);
int hpic_reset_tallies(hpic_ctx *ctx);
/* Photon histograms, (n_Ebins + 2) rows (underflow, bins, overflow) x
 * n_thbins, row-major; energy-weighted (J) and number-weighted (photons).
 * Either pointer may be NULL.  Polar angle is measured from +x. */
int hpic_read_hist(hpic_ctx *ctx, double *energy_weighted, double *number_weighted);
/* Per-step X-ray energy above ce_threshold, max_history doubles. */
int hpic_read_history(hpic_ctx *ctx, double *out);

/* Number of doubles in grid `which` (see the layout above). */
int hpic_grid_len(const hpic_ctx *ctx, int which, int64_t *len);
int hpic_read_grid(hpic_ctx *ctx, int which, double *host_out);
/* Overwrite a grid from host doubles (state restore, tests).  Writing T or
 * eta does not recompute the other. */
int hpic_write_grid(hpic_ctx *ctx, int which, const double *host_in);

/* Live electrons (synchronises). */
int hpic_count_particles(hpic_ctx *ctx, int64_t *n);
/* Copy live electrons out in storage order: positions (m), u = p/(m_e c),
 * remaining optical depth tau, id.  Fails with HPIC_EINVAL if cap is less
 * than the live count; *n receives the count.  Any of the output pointers
 * may be NULL (that array is skipped).  The compaction and the conversion
 * to double run on the device in a scratch buffer the context owns (grown
 * to 8 bytes per electron slot, freed by hpic_destroy or
 * hpic_batch_destroy); HPIC_ENOMEM if it cannot be allocated.  This call
 * and hpic_load_particles / hpic_count_particles synchronise the stream.
 * The host arrays here and in hpic_load_particles may be page-locked
 * (cudaHostAlloc) or pageable; page-locked ones, allocated once and reused,
 * avoid the driver's staging copies and the page faults of fresh memory. */
int hpic_read_particles(hpic_ctx *ctx, double *x, double *y, double *z,
                        double *ux, double *uy, double *uz, double *tau,
                        uint32_t *id, int64_t cap, int64_t *n);
/* Replace the electron population with n host electrons (same units).
 * Positions must lie in [0, n*dx] on each axis (any finite position with
 * HPIC_UNBOUNDED).  The arrays are checked on the device before anything is
 * written, so on HPIC_EINVAL the population is unchanged; the upload uses
 * the context's transfer scratch (see hpic_read_particles).  Errors:
 * HPIC_EINVAL, HPIC_ENOMEM. */
/* Per-electron weights (real electrons per macro-electron) of the live
 * electrons, in the order hpic_read_particles returns them (same cap / n
 * semantics).  With the flat-top envelope every weight is the Eq. (B1) one. */
int hpic_read_weights(hpic_ctx *ctx, double *w, int64_t cap, int64_t *n);
/* Set the weights of the n electrons last loaded by hpic_load_particles (in
 * that order); HPIC_ESTATE unless the laser uses the Gaussian envelope (the
 * flat-top path keeps one weight for all). */
int hpic_load_weights(hpic_ctx *ctx, int64_t n, const double *w);

int hpic_load_particles(hpic_ctx *ctx, int64_t n, const double *x, const double *y,
                        const double *z, const double *ux, const double *uy,
                        const double *uz, const double *tau, const uint32_t *id);
/* Step counter (the Philox counter word) and the next injection id. */
int hpic_get_clock(hpic_ctx *ctx, int64_t *step, int64_t *next_id);
int hpic_set_clock(hpic_ctx *ctx, int64_t step, int64_t next_id);

/* Kernel timing of the particle push/collide/emit/deposit kernel: when
 * enabled, CUDA events bracket each of its launches on the context stream.
 * hpic_kernel_time returns the summed device time (ms), the launch count
 * and the particle-steps those launches processed, then clears them. */
int hpic_profile(hpic_ctx *ctx, int enable);
int hpic_kernel_time(hpic_ctx *ctx, double *ms, int64_t *launches, double *particle_steps);

/* Kernels launched by this context since creation (all kinds). */
int hpic_launch_count(const hpic_ctx *ctx, int64_t *launches);

/* Cell sort for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a service of this library.  Callers such as code
 * running inside a CUDA stream capture (allocation cannot be captured),
 * hosts with a device-memory budget fixed at start-up, or plug-ins whose
 * framework owns all device allocations cannot call cudaMalloc; this entry
 * point allocates nothing.  It sorts the caller's n electron slots
 * (in_soa: x, y, z in cells, i.e. position / dx, then ux, uy, uz, tau, all
 * float for HPIC_FP32_MIXED or double for HPIC_FP64, then uint32 ids; all
 * device pointers) into out_soa (same layout, room for n) in the order of
 * hpic_sort: 4x4x4 cell tiles, x-fastest; slots with id 0xFFFFFFFF are
 * dropped and the number kept is written to *n_live_dev (device int64).
 * Scratch comes from one fixed 8 MiB + 64 KiB device array inside the
 * library, which every GPU that loads the library holds until exit; hence
 * the limits n <= 1048576 and nti*ntj*ntk*64 <= 1048576 cells (each
 * dimension rounded up to a multiple of 4), beyond which it returns
 * HPIC_EINVAL with a message in hpic_last_error(NULL).  The first call on a
 * device looks up the scratch address on that device; make that call
 * before any stream capture.  That address is kept for the life of the
 * device's primary context: do not call this again in a process that has
 * reset the device (cudaDeviceReset), since the array may have moved.  Calls
 * share the scratch: calls that overlap on the GPU race, so serialise them.
 * No output array may overlap an input array (the sort reads one while it
 * writes the other): overlapping ranges give HPIC_EINVAL before any device
 * call.  Asynchronous on cuda_stream. */
int hpic_sort_cells_noalloc(int32_t nx, int32_t ny, int32_t nz, int32_t precision, int64_t n,
                            const void *const in_soa[8], void *const out_soa[8],
                            int64_t *n_live_dev, int device, void *cuda_stream);

/* Checkpoint and resume.  hpic_save writes the whole state of ctx (target,
 * run and laser descriptions, clock, every particle slot with weights, all
 * grids, tallies, histograms and history) to the file `path` (created or
 * truncated; HPIC_EINVAL if it cannot be written).  hpic_load creates a new
 * context on `device` / cuda_stream from such a file, as hpic_init_target and
 * hpic_inject_electrons would, then restores the state; stepping it continues
 * the saved run (random numbers are keyed on the saved clock and ids).  The
 * file is raw host memory of this ABI's structs (little-endian, natural
 * alignment); a file that is not a checkpoint, or is truncated, gives
 * HPIC_EINVAL with nothing created.  Works on batch targets too (the loaded
 * context is a single one). */
int hpic_save(hpic_ctx *ctx, const char *path);
int hpic_load(hpic_ctx **out, const char *path, int device, void *cuda_stream);

int hpic_destroy(hpic_ctx *ctx);
/* Last error of ctx, or of the last failed creation when ctx is NULL. */
const char *hpic_last_error(const hpic_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batches: many independent targets advanced together.
 *
 * The paper's scans (Sec. III: thickness, material and intensity) are many
 * independent runs of the step above.  A batch holds n_targets such runs of
 * uneven size on one GPU and advances all of them with one launch per kernel
 * kind per step: the particle kernel is persistent (a fixed grid of
 * blocks_per_sm blocks per SM walks the warp-sized tasks of every target),
 * the field kernels walk the concatenated grids, and the whole step is
 * replayed from a captured CUDA graph.  Physics per target is identical to
 * a single context made with the same target, laser and run parameters and
 * run.target_index + t: target t draws the same random numbers, so in FP64
 * its results match such a context to rounding (only the order of
 * floating-point atomic additions differs).
 *
 * Memory: every target gets n_macro + spare_slots particle slots, fixed at
 * creation, and its own grid, tallies and counters; all of it is one device
 * allocation owned by the batch.
 * ------------------------------------------------------------------------ */
#define HPIC_BATCH_MAX_TARGETS 256

typedef struct {
  int32_t blocks_per_sm;   /* persistent particle-kernel blocks per SM (1..5; FP64 1..2);
                              FP32 blocks hold 512 threads at 1..2 per SM, 384 at 3,
                              256 at 4..5; FP64 blocks 256 */
  int32_t sort_interval;   /* steps between cell sorts (0: never); keyed by the cell
                              reached (sort_interval + 1)/2 steps ahead */
  int32_t use_graph;       /* replay captured CUDA graphs (1) or launch directly (0) */
  int32_t reserved;
  double ms_per_step;      /* autotuner: measured time of the chosen setting */
} hpic_batch_tuning;

/* Create a batch of n_targets (1..HPIC_BATCH_MAX_TARGETS) targets sharing the
 * run parameters `run` (time step, precision, physics, tallies, table; the
 * run's sort_interval is the initial tuning).  lasers[t] schedules target t's
 * injection as hpic_inject_electrons does (lasers may be NULL: no injection).
 * target_index[t] is target t's fourth Philox counter word (NULL: the run's
 * target_index + t); a scan sharded over several batches keeps each target's
 * random numbers by passing its global index.  Work goes to cuda_stream, or
 * to a stream the batch creates if NULL (a captured graph needs a stream
 * other than the legacy default). */
int hpic_batch_init(hpic_batch **out, int32_t n_targets, const hpic_target_desc *targets,
                    const hpic_laser_desc *lasers, const hpic_run_params *run,
                    const uint32_t *target_index, int64_t spare_slots, int device,
                    void *cuda_stream);

/* Borrow target t's context.  On it the read/write calls work as on a
 * single context (hpic_read_tallies, hpic_read_hist, hpic_read_history,
 * hpic_read_grid, hpic_write_grid, hpic_read_particles,
 * hpic_count_particles, hpic_load_particles within the slots,
 * hpic_get_clock, hpic_set_clock, hpic_launch_count); the calls that step,
 * sort, inject, seed, profile or destroy return HPIC_ESTATE.  The handle
 * stays valid until hpic_batch_destroy. */
int hpic_batch_target(hpic_batch *b, int32_t t, hpic_ctx **out);

/* Advance every target by n steps (asynchronous on the batch stream). */
int hpic_batch_step(hpic_batch *b, int64_t n_steps);

/* Current tuning, and a manual override (validated; graphs re-captured). */
int hpic_batch_get_tuning(const hpic_batch *b, hpic_batch_tuning *out);
int hpic_batch_set_tuning(hpic_batch *b, const hpic_batch_tuning *in);

/* Autotuner: from a snapshot of the whole batch state, time trial_steps
 * steps (>= 1, rounded up to a multiple of 40) for every candidate
 * (blocks_per_sm 2..5 in FP32, 1..2 in FP64, x sort_interval in
 * {3, 5, 10, 20}, graphs on), restore the snapshot after each trial, and
 * keep the fastest.  The simulation is left exactly where it was.  Needs
 * device memory for one copy of the batch state; the result is written to
 * *out when out is not NULL. */
int hpic_batch_autotune(hpic_batch *b, int32_t trial_steps, hpic_batch_tuning *out);

/* Timing of the particle kernel, as hpic_profile / hpic_kernel_time (while
 * enabled the step is launched directly, not from a graph, so that events
 * can bracket the kernel).  particle_steps sums all targets. */
int hpic_batch_profile(hpic_batch *b, int enable);
int hpic_batch_kernel_time(hpic_batch *b, double *ms, int64_t *launches,
                           double *particle_steps);

/* Kernels launched by the batch (graph replays count their kernels). */
int hpic_batch_launch_count(const hpic_batch *b, int64_t *launches);

int hpic_batch_destroy(hpic_batch *b);
/* Last error of b, or of the last failed batch creation when b is NULL. */
const char *hpic_batch_last_error(const hpic_batch *b);

/* ------------------------------------------------------------------------
 * The paper's three-macro-electron estimate of the loss channels (Sec. III.B),
 * evaluated for many parameter sets at once, one GPU thread each (the
 * background heatmap of eta_e->gamma over intensity and Z).  Per set: a0
 * from Eq. (1), mean energy <eps> = a0 m_e c^2 <sqrt(fg)>, injected count
 * N_e = I0 <fg> (pi r_fwhm^2/4)(t_fwhm sqrt(ln10/ln2)) eta_l2e / <eps>; the
 * exponential spectrum is cut at eps_th and eps_esc = kappa_esc a0 m_e c^2
 * into a warm, an emitting and an escaping macro-electron (band count and
 * band energy); each is integrated by RK4 in its path length x through
 * d eps/dx = -(S_brem + S_ion + S_tnsa + S_field(x)), Eqs. (stop_brem),
 * (stop_ion), (stop_tnsa), (stop_field): the warm and emitting ones until
 * eps <= E_stop (the remainder counts as ionisation), the escaping one to
 * x = L_x (the remainder escapes).  Photons above eps_th are counted with
 * S_brem(eps - eps_th).  Each step is at most rel_step eps / S_total and
 * rel_step (x + r_fwhm/(2 tan theta_c)) long.  FP64 throughout.
 * ------------------------------------------------------------------------ */
enum {
  HPIC_MODEL_BREM = 1, HPIC_MODEL_ION = 2, HPIC_MODEL_TNSA = 4, HPIC_MODEL_FIELD = 8,
  HPIC_MODEL_ALL = 15
};
enum {  /* hpic_model_out.E */
  HPIC_MODEL_E_INJ = 0, HPIC_MODEL_E_BREM = 1, HPIC_MODEL_E_ION = 2, HPIC_MODEL_E_TNSA = 3,
  HPIC_MODEL_E_FIELD = 4, HPIC_MODEL_E_XRAY_ABOVE = 5, HPIC_MODEL_E_ESC = 6
};
typedef struct {
  double Z, n_i_m3, I_ex_J;         /* solid */
  double Lx_m, Ly_m, Lz_m;          /* target size */
  double I0_Wm2, lambda_m, eta_l2e; /* laser */
  double r_fwhm_m, t_fwhm_s;        /* injection envelope widths */
  double mean_fg, mean_sqrt_fg;     /* envelope means over the injecting cells */
  double kappa_esc, kappa_tnsa;     /* reflux constants (Sec. II.A) */
  double theta_c_rad, eta_avg_ohm_m;/* current cone half-angle, typical resistivity */
  double eps_th_J;                  /* X-ray threshold */
  double E_stop_J;                  /* a macro-electron has stopped below this */
  double rel_step;                  /* RK4 step bound, fraction (e.g. 0.01) */
  int32_t mechanisms;               /* HPIC_MODEL_* bitmask */
  int32_t pad;
} hpic_model_in;
typedef struct {
  double E[8];                      /* J, indexed by HPIC_MODEL_E_* */
  double N_e, a0;
  double N_band[3], eps_band[3];    /* warm, emitting, escaping: count, J per electron */
  double x_end[3];                  /* path length of each macro-electron (m) */
  int64_t steps;                    /* RK4 steps taken, all three */
} hpic_model_out;

/* n parameter sets from host memory in, results to host memory out
 * (caller-owned; synchronous).  Invalid sets (non-positive rel_step, sizes,
 * energies or densities) make the call return HPIC_EINVAL before any work. */
int hpic_model(int64_t n, const hpic_model_in *in, hpic_model_out *out, int device,
               void *cuda_stream);
/* The same on device arrays (in, out: n entries each on `device`),
 * enqueued on cuda_stream; allocates nothing and does not validate. */
int hpic_model_device(int64_t n, const hpic_model_in *in, hpic_model_out *out, int device,
                      void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
