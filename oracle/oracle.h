/*
 * FP64 CPU oracle for the fast-electron step of the 3D hybrid-PIC
 * bremsstrahlung method (Morris, Robinson & Ridgers, arXiv 2107.01723).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, serial reference the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library: every formula below is
 * written again from the paper, in SI units and double precision.
 *
 * Units: SI throughout (m, s, kg, J, K, V/m, T, A/m^2, Ohm m).  The only
 * exception is at the interface, where particle momentum is exchanged as
 * u = p / (m_e c) (dimensionless), so that both sides can be compared.
 *
 * Grid convention (Yee staggering; the paper names no grid, this is the
 * reading both sides use): the target is nx*ny*nz cubic cells of side dx.
 * Every vector component is stored in an (nx+1)*(ny+1)*(nz+1) array indexed
 * i + (nx+1)*(j + (ny+1)*k); its physical location is
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)   (also j_h)
 *   Bx (i, j+1/2, k+1/2)  By (i+1/2, j, k+1/2)  Bz (i+1/2, j+1/2, k)
 * in units of dx; entries past a staggered extent are padding and stay 0.
 * Cell-centred scalars (T, eta, drag heat) are nx*ny*nz, index i+nx*(j+ny*k).
 */
#ifndef HPIC_ORACLE_H
#define HPIC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* physics switches (bitmask) */
enum {
  ORC_DRAG = 1,     /* continuous ionisation drag, Eq. (5) */
  ORC_SCATTER = 2,  /* Davies angular scatter, Eq. (B4) */
  ORC_BREM = 4,     /* optical-depth bremsstrahlung emission, App. B */
  ORC_FIELDS = 8,   /* E from Ohm's law with return current, Eq. (A2) */
  ORC_FARADAY = 16, /* B update, Eq. (A3); clear to hold B fixed */
  ORC_HEATING = 32, /* temperature and resistivity update, Eqs. (A4)-(A8) */
  ORC_ALL = 63,
  /* unbounded uniform medium: no fields are gathered, no faces, no current
   * or heat deposited on the grid (collisions and emission only) */
  ORC_UNBOUNDED = 64,
  /* ionised-screening enhancement F_sigma of the bremsstrahlung cross
   * section (App. B), from the ion temperature of the electron's cell */
  ORC_FSIGMA = 128,
  /* electron-ion temperature equilibration (App. A); T_i is evolved */
  ORC_EI = 256
};

/* grid component codes */
enum {
  ORC_T = 0, ORC_ETA = 1, ORC_EX = 2, ORC_EY = 3, ORC_EZ = 4,
  ORC_BX = 5, ORC_BY = 6, ORC_BZ = 7, ORC_JX = 8, ORC_JY = 9, ORC_JZ = 10,
  ORC_HEAT = 11, ORC_TI = 12
};

/* one more element sharing every cell with the target's own (a compound
 * solid, App. A), at its own ion density */
typedef struct {
  double Z, n_i, I_ex, Zstar, A_ion;
} orc_solid;

typedef struct {
  int32_t nx, ny, nz;
  double dx;          /* cell side (m) */
  double Z;           /* atomic number */
  double n_i;         /* ion number density (m^-3) */
  double I_ex;        /* mean excitation energy (J) */
  double Zstar;       /* conduction ionisation state for eta */
  double lnLambda;    /* Coulomb logarithm for eta */
  double eta_max;     /* resistivity cap (Ohm m) */
  double lambda1;     /* cold-limit fit parameter (0 = no cold limit) */
  double lambda2;     /* resistivity multiplier */
  double T0;          /* initial background temperature, electrons and ions (K) */
  double A_ion;       /* ion mass in atomic mass units (e-i equilibration) */
  int32_t n_extra;    /* further elements of a compound (0..3) */
  int32_t pad;
  orc_solid extra[3];
} orc_target;

typedef struct {
  double I0;          /* peak intensity (W m^-2) */
  double lambda;      /* wavelength (m) */
  double eta_l2e;     /* laser -> hot-electron efficiency */
  double spot_r;      /* injection disc radius (m) */
  double spot_y, spot_z; /* disc centre on the x = 0 face (m) */
  double t_inj;       /* injection duration (s) */
  double cone_half;   /* injection cone half-angle (rad) */
  int64_t n_macro;    /* flat-top: macro-electrons over the whole injection */
  int32_t envelope;   /* ORC_ENV_FLAT or ORC_ENV_GAUSS */
  int32_t per_cell;   /* Gaussian: macro-electrons per injecting cell per step */
  double r_fwhm, t_fwhm; /* Gaussian: radial and temporal full widths at half maximum */
  double f_min, g_min;   /* Gaussian: inject where f(r) >= f_min and g(t) >= g_min */
  int32_t moore_cap;  /* 1: cone half-angle min(cone_half, atan(sqrt(2/(gamma-1)))) */
  int32_t pad;
} orc_laser;

enum { ORC_ENV_FLAT = 0, ORC_ENV_GAUSS = 1 };

typedef struct {
  double dt;          /* time step (s) */
  uint64_t seed;      /* Philox key */
  uint32_t target_index; /* fourth counter word */
  double kappa_esc, kappa_tnsa, sigma_dtheta; /* reflux constants */
  double brem_boost;  /* cross-section multiplier B, photon weight w/B */
  double k_min;       /* lowest photon energy modelled (J) */
  double E_cut;       /* tracking cut (J) */
  int32_t n_E, n_theta;          /* photon tally bins */
  double tally_E_min, tally_E_max; /* log energy bin range (J) */
  double ce_threshold;           /* X-ray threshold (J) */
  int32_t table_rows, table_cols; /* inverse-CDF table shape */
  double table_E_max;            /* top electron energy of the table (J) */
  int32_t curlB_term;            /* 1: E = eta(curl B/mu0 - j_h), 0: E = -eta j_h */
  int32_t physics;               /* ORC_* bitmask */
  int32_t max_history;           /* length of the per-step X-ray history */
} orc_run;

typedef struct {
  double E_injected, N_injected;
  double W_field;       /* energy lost by electrons to E (positive = loss) */
  double E_drag;        /* ionisation heat, including cut remainders */
  double E_xray, E_xray_above;
  double E_escaped, E_reflux;
  double E_ohmic_grid;  /* sum of eta j_h.j_h dt V over cells */
  double n_injected, n_escaped, n_refluxed, n_reflux_absorbed;
  double n_cut, n_emitted, particle_steps;
} orc_tallies;

typedef struct orc_sim orc_sim;

/* ---- whole-step simulation ---- */
orc_sim *orc_create(const orc_target *t, const orc_laser *l, const orc_run *r);
void orc_destroy(orc_sim *s);
/* advance n steps; returns 0 */
int orc_step(orc_sim *s, int64_t n);
/* field solve and heating on the current grids only (no particles, clock
 * unchanged): exposes Eqs. (A2)-(A8) to the pins */
void orc_fields(orc_sim *s);
/* append n electrons uniform in the box, isotropic, kinetic energy
 * exponential with mean `mean_eps` (J), fresh optical depths; Philox
 * blocks 10 and 11 at the current step, ids from the id counter */
void orc_seed(orc_sim *s, int64_t n, double mean_eps);
int64_t orc_n_particles(const orc_sim *s);
/* particles in storage order; x in m, u = p/(m_e c); tau = remaining optical depth */
void orc_get_particles(const orc_sim *s, double *x, double *y, double *z,
                       double *ux, double *uy, double *uz, double *tau,
                       uint32_t *id);
void orc_set_particles(orc_sim *s, int64_t n, const double *x, const double *y,
                       const double *z, const double *ux, const double *uy,
                       const double *uz, const double *tau, const uint32_t *id);
int64_t orc_grid_len(const orc_sim *s, int which);
void orc_get_grid(const orc_sim *s, int which, double *out);
void orc_set_grid(orc_sim *s, int which, const double *in);
void orc_get_tallies(const orc_sim *s, orc_tallies *out);
void orc_reset_tallies(orc_sim *s);
/* histograms are (n_E + 2) rows (underflow, n_E bins, overflow) x n_theta */
void orc_get_hist(const orc_sim *s, double *energy_weighted, double *number_weighted);
void orc_get_history(const orc_sim *s, double *out);
void orc_get_clock(const orc_sim *s, int64_t *step, int64_t *n_injected_ids);
void orc_set_clock(orc_sim *s, int64_t step, int64_t n_injected_ids);
double orc_live_energy(const orc_sim *s);   /* sum w * kinetic energy (J) */
double orc_field_energy(const orc_sim *s);  /* sum B^2/(2 mu0) dx^3 (J) */
double orc_weight(const orc_sim *s);        /* flat-top macro-electron weight */
/* per-electron weights (real electrons per macro-electron), storage order */
void orc_get_weights(const orc_sim *s, double *w);
void orc_set_weights(orc_sim *s, int64_t n, const double *w);
double orc_a0_of(const orc_sim *s);

/* ---- the three-macro-electron estimate of the loss channels (Sec. III.B) ---- */
enum {
  ORC_MODEL_BREM = 1, ORC_MODEL_ION = 2, ORC_MODEL_TNSA = 4, ORC_MODEL_FIELD = 8,
  ORC_MODEL_ALL = 15
};
enum {  /* orc_model_out.E */
  ORC_MODEL_E_INJ = 0, ORC_MODEL_E_BREM = 1, ORC_MODEL_E_ION = 2, ORC_MODEL_E_TNSA = 3,
  ORC_MODEL_E_FIELD = 4, ORC_MODEL_E_XRAY_ABOVE = 5, ORC_MODEL_E_ESC = 6
};
typedef struct {
  double Z, n_i, I_ex;            /* solid */
  double Lx, Ly, Lz;              /* target size (m) */
  double I0, lambda, eta_l2e;     /* peak intensity (W m^-2), wavelength (m), absorption */
  double r_fwhm, t_fwhm;          /* envelope widths (m, s) */
  double mean_fg, mean_sqrt_fg;   /* <fg> and <sqrt(fg)> over the injecting cells */
  double kappa_esc, kappa_tnsa;   /* reflux constants */
  double theta_c, eta_avg;        /* current cone half-angle (rad), typical resistivity */
  double eps_th;                  /* X-ray threshold (J) */
  double E_stop;                  /* a macro-electron has stopped below this (J) */
  double rel_step;                /* RK4 step: rel_step eps / S_total long */
  int32_t mechanisms;             /* ORC_MODEL_* bitmask */
  int32_t pad;
} orc_model_in;
typedef struct {
  double E[8];                    /* J, indexed by ORC_MODEL_E_* */
  double N_e, a0;                 /* injected electrons, Eq. (1) */
  double N_band[3], eps_band[3];  /* warm, emitting, escaping: count, energy per electron (J) */
  double x_end[3];                /* path length of each macro-electron (m) */
} orc_model_out;
void orc_model(const orc_model_in *m, orc_model_out *out);

/* ---- single formulas, for the pins ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t x);
double orc_a0(double I0_Wm2, double lambda_m);
/* A compound's stopping powers, cross sections, scatter variances and
 * heat capacities combine its elements as documented in physics.c. */
double orc_stop_ion(const orc_target *t, double eps_k);   /* J/m */
double orc_stop_brem(const orc_target *t, double eps_k);  /* J/m, Eq. (4) */
double orc_dsigma_dk(const orc_target *t, double eps_k, double k); /* m^2/J */
double orc_sigma_tot(const orc_target *t, double k_min, double eps_k); /* m^2, per target ion */
/* sum over the elements of n_i sigma_tot (1/m): the emission rate per length */
double orc_brem_rate(const orc_target *t, double k_min, double eps_k);
void orc_brem_table(const orc_target *t, double k_min, double E_max, int rows,
                    int cols, double *v);
double orc_brem_sample(const double *v, int rows, int cols, double k_min,
                       double E_max, double eps_k, double r);
double orc_davies_sigma(const orc_target *t, double p_SI, double dt); /* rad */
double orc_photon_theta(double gamma, double u);
double orc_heat_capacity(double T_K, double Z);
/* the temperature rise of Eq. (A7) for a deposited energy density rho
 * (J/m^3); a compound uses sum Z n_i and the n_e-weighted mean of 1/C */
double orc_temperature_rise(const orc_target *t, double T_K, double rho);
double orc_resistivity(const orc_target *t, double T_K);
/* F_sigma of the bremsstrahlung cross section at ion temperature T_i (K) */
double orc_f_sigma(const orc_target *t, double Ti_K);
/* e-i equilibration rates (1/s): dT_e/dt = (T_i - T_e) rate_e,
 * dT_i/dt = (T_e - T_i) rate_i */
void orc_ei_rates(const orc_target *t, double Te_K, double Ti_K, double *rate_e,
                  double *rate_i);
void orc_rotate(const double d[3], double theta, double phi, double out[3]);
/* energy row and polar column of a photon of energy k (J) at polar angle
 * theta (rad, from +x) in the run's photon tallies; the step's own tally
 * uses it */
void orc_tally_bin(const orc_run *r, double k, double theta, int *row, int *col);
void orc_boris(double u[3], const double E[3], const double B[3], double dt);

#ifdef __cplusplus
}
#endif
#endif
