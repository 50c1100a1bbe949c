/*
 * pic_oracle.h -- FP64 CPU oracle of the explicit 1D3V electrostatic PIC-MCC step.
 *
 * TEST INFRASTRUCTURE.  This is the oracle: a plain, slow, single-threaded
 * restatement of the method that the CUDA library is checked against.  Only
 * the tests, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs may load it.  It shares no code, header, table or constant generator
 * with the CUDA library, and the library never calls it.
 *
 * The method (paper §1): particles move in the field computed on a mesh from
 * their own charge; explicit leapfrog; Boris pusher with a static B;
 * null-collision Monte Carlo against tabulated cross sections; walls with
 * secondary emission; Poisson's equation.  The paper prints no equations for
 * any of these; every reading taken where it is silent is listed in the
 * design notes and repeated at the function that implements it.
 *
 * Units: SI, except energies of cross-section tables (eV) and positions, which
 * are kept in cell units xi = x/dx (cell index + offset) so that a state
 * written by the GPU as (int32 cell, fp32 offset) converts to FP64 exactly.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#define OR_MAX_SPECIES 2
#define OR_MAX_PROC 4
#define OR_NGRID 1000          /* cross-section grid: 1000 log points (1e-3..1e3 eV) */
#define OR_EEPF_BINS 240       /* 0..60 eV in 0.25 eV bins */
#define OR_IFEDF_BINS 256      /* ion energy at the electrodes: 256 bins on [0, ifedf_emax_ev) */

enum { OR_ELASTIC = 0, OR_EXCITATION = 1, OR_IONIZATION = 2, OR_ISO = 3, OR_CX = 4 };

typedef struct {
    int32_t periodic;          /* 1 = periodic box, 0 = two absorbing electrodes */
    int32_t n_cells;
    double length;             /* m */
    double dt;                 /* s */
    double gas_density;        /* m^-3 */
    double gas_temp;           /* K */
    double gas_mass;           /* kg */
    double B[3];               /* T, static and uniform */
    double E_ext[3];           /* V/m, static and uniform, added to the mesh field */
    int32_t n_harm;            /* electrode voltage harmonics at x = 0 */
    double harm_freq[4], harm_amp[4], harm_phase[4];
    double see_gamma;          /* secondary electrons per ion reaching a wall */
    double see_temp_ev;
    double bg_charge;          /* immobile uniform charge density, C/m^3 */
    double const_nu_e;         /* >0: constant-frequency electron-neutral model, 1/s */
    int32_t n_species;         /* species 0 = electrons, species 1 = ions */
    double q[OR_MAX_SPECIES], m[OR_MAX_SPECIES], w[OR_MAX_SPECIES];  /* C, kg, particles/m^2 */
    uint64_t seed;
    int32_t diag_interval;     /* energy moments / EEPF every diag_interval steps (0 = never) */
    int32_t rewind;            /* 1 = velocities loaded at t=0 are pushed back dt/2 before the first step */
    int32_t circuit;           /* electrode at x = 0: 0 = driven by V(t), 1 = V(t) through a series capacitor,
                                  2 = driven by the current density J(t) (the harmonics in A/m^2) */
    double cap;                /* that capacitor, F/m^2 (0 = floating electrode) */
    double ifedf_emax_ev;      /* > 0: histogram the energy of ions reaching each electrode */
    int32_t no_field;          /* 1: no Poisson solve; the particles feel only E_ext (swarm runs) */
    double axial_len;          /* > 0: virtual axial length (m); a particle whose axial excursion reaches it
                                  is renewed (paper §3.6, after Lafleur, Baalrud and Chabert) */
    double renew_temp_ev[OR_MAX_SPECIES];      /* Maxwellian of the renewed particles */
    double renew_drift[OR_MAX_SPECIES][3];     /* and its drift, m/s */
} or_params;

typedef struct or_case or_case;

/* per-step counters (cumulative since the last or_reset_moments) */
typedef struct {
    int64_t n_steps;           /* steps accumulated into the moment sums */
    int64_t n_diag;            /* diagnostic steps accumulated */
    int64_t absorbed[OR_MAX_SPECIES][2];   /* per species, per wall (0: x=0, 1: x=L) */
    int64_t see_emitted;
    int64_t candidates[OR_MAX_SPECIES];
    int64_t collisions[OR_MAX_SPECIES][OR_MAX_PROC];
    int64_t ionizations;
    int64_t step;              /* completed steps since load */
    int64_t renewed[OR_MAX_SPECIES];   /* axial renewals */
} or_counters;

or_case *or_create(const or_params *p);
void     or_destroy(or_case *c);
/* Load one process's raw cross-section table (energy eV, sigma m^2, n points,
 * ascending energy).  Processes are summed in load order. */
int  or_load_xsec(or_case *c, int sp, int kind, double threshold_ev,
                  const double *energy_ev, const double *sigma_m2, int n);
int  or_load_particles(or_case *c, int sp, int64_t n, const double *xi,
                       const double *vx, const double *vy, const double *vz,
                       const uint32_t *id);
int  or_load_profile(or_case *c, int sp, int64_t n, const double *density, const double *temp_ev,
                     const double drift[3], uint32_t id_base);
int  or_step(or_case *c, int64_t n_steps);
int64_t or_count(const or_case *c, int sp);
/* margin/event: per particle, the smallest normalised distance of any
 * discrete decision of the last step to its threshold, and that step's event
 * (0 none, 1 null candidate, 2+k process k, -1 absorbed).  Either may be NULL. */
int  or_get_particles(const or_case *c, int sp, double *xi, double *vx, double *vy,
                      double *vz, uint32_t *id, double *margin, int32_t *event);
/* Diagnostic of the last step, same order as or_get_particles: an electron's
 * speed (m/s) just before a collision that took a threshold energy from it
 * (excitation or ionization), and for the electron an ionization ejects, its
 * parent's; 0 for every other particle.  A test uses it to scale the
 * comparison of the energy left after the loss, which cancels against the
 * threshold and carries the rounding of the energy before it. */
int  or_get_loss_speed(const or_case *c, int sp, double *v);
/* Diagnostic of the last step, same order: the length in cells of the move
 * that placed the particle (its own |v_x| dt/dx; for an ionization product
 * its parent's; for a secondary electron its distance from the wall).  The
 * FP32 rounding of a position grows with it. */
int  or_get_move(const or_case *c, int sp, double *d);
/* axial excursion z (m) of each particle, same order as or_get_particles */
int  or_get_axial(const or_case *c, int sp, double *z);
/* collision clock 2 k + c of each particle, same order as or_get_particles */
int  or_get_clock(const or_case *c, int sp, int32_t *clk);
/* -ln(u) in FP32 (the gap arithmetic of the collision clock) */
float or_neg_log_u32(float u);
/* clock state 2 k + c of a fresh gap from uniform u with lam = numax dt (FP32) */
int32_t or_clock_state(float u, float lam, double *margin);
/* phi, E: n_nodes; R: n_nodes int64 raw deposit of species sp */
int  or_get_field(const or_case *c, double *phi, double *E);
int  or_get_deposit(const or_case *c, int sp, int64_t *R);
int  or_get_numax(const or_case *c, int sp, double *numax);
int  or_get_nu_table(const or_case *c, int sp, int k, double *nu);  /* OR_NGRID values */
void or_get_counters(const or_case *c, or_counters *out);
/* moment sums since the last reset (any pointer may be NULL):
 *   dens[sp*n_nodes + i]  : sum over steps of the number density (m^-3)
 *   phi_sum[i]            : sum over steps of phi
 *   en[sp*n_nodes + i]    : sum over diagnostic steps of sum_p w eps W_i / vol_i (eV m^-3)
 *   dens_diag[...]        : the density on those diagnostic steps
 *   eepf[OR_EEPF_BINS]    : counts of electrons in the central 10 % of the gap
 *   ke[sp]                : kinetic energy per area (J/m^2) summed over diagnostic steps
 *   pw[sp]                : sum_p q w v_x E_x(mesh) (W/m^2) summed over diagnostic steps */
int  or_get_moments(const or_case *c, double *dens, double *phi_sum, double *en,
                    double *dens_diag, double *eepf, double *ke, double *pw);
void or_reset_moments(or_case *c);
/* ion energy histogram at each electrode since the last reset:
 * out[wall * OR_IFEDF_BINS + b], b = floor(eps / ifedf_emax_ev * OR_IFEDF_BINS) */
int  or_get_ifedf(const or_case *c, double *out);
/* charge per area of the electrode at x = 0 with its capacitor plate (series
 * capacitor circuit), C/m^2 */
double or_get_electrode_charge(const or_case *c);
/* field energy per area (J/m^2) after each step since load, n_out values */
int64_t or_get_field_energy(const or_case *c, double *out, int64_t max_n);

/* primitives exposed for the pins */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform(uint32_t r);
void or_deposit(int n_cells, int periodic, int64_t n, const double *xi, int64_t *R);
int  or_poisson(int n_cells, int periodic, double dx, const double *rho,
                double phi_left, double *phi);
void or_boris(double qm, double h, const double E[3], const double B[3], double v[3]);
int64_t or_sort_by_cell(int n_cells, int64_t n, const int32_t *cell, int64_t *perm);

#endif
