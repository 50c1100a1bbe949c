/*
 * pic1d3v.h -- C ABI of the B300 (sm_103a) explicit 1D3V electrostatic
 * PIC-MCC particle step.
 *
 * The method is the one the paper states in §1: charged super-particles move
 * in the electric field computed on a mesh from their own charge (explicit
 * leapfrog, Boris pusher with a static imposed B), collide with the neutral
 * gas by the null-collision Monte Carlo method against tabulated cross
 * sections, are absorbed at the electrodes with secondary electron emission,
 * and Poisson's equation is solved on the mesh every step.  A case is set up
 * with the quantities the paper's dialog asks for (§1: gas, pressure, gap,
 * voltage waveform, magnetic field, walls and secondary emission).
 *
 * Conventions for every call:
 *   - Returns a pic_status; calls never abort, exit or trap on the device.
 *   - Work is enqueued on the case's stream; errors raised by device work
 *     (capacity overflow, non-finite field, a device wait that gave up)
 *     surface at the next call that synchronises (pic_read_*, pic_sync).
 *   - Host pointers are read during the call only; the library keeps copies.
 *   - A pic_case is not thread-safe; distinct cases are independent.
 *   - pic_last_error() gives a human-readable message for the calling thread.
 *
 * Particle layout (species s, slot k): SoA, int32 cell[k] in [0, n_cells),
 * float32 offset[k] in [0, 1) (position x = (cell + offset) dx), float32
 * vx, vy, vz (m/s), uint32 id (keys the counter-based random numbers).
 * Species 0 are electrons, species 1 ions.
 */
#ifndef PIC1D3V_H
#define PIC1D3V_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = 1,      /* bad argument or descriptor */
    PIC_ENOMEM = 2,      /* device allocation failed */
    PIC_ECUDA = 3,       /* a CUDA runtime call failed (message in pic_last_error) */
    PIC_ECAPACITY = 4,   /* particles exceeded a species' capacity; the overflow was not stored */
    PIC_ENUMERIC = 5,    /* the field solve produced a non-finite value */
    PIC_ETIMEOUT = 6,    /* a bounded device wait gave up */
    PIC_ESTATE = 7       /* call not valid in the current state (e.g. step before load) */
} pic_status;

/* collision process kinds (cumulative sums follow the load order) */
enum { PIC_ELASTIC = 0, PIC_EXCITATION = 1, PIC_IONIZATION = 2, PIC_ISO = 3, PIC_CX = 4 };

#define PIC_DESC_VERSION 2u
#define PIC_MAX_PROC 4
#define PIC_NGRID 1000          /* cross-section grid: 1000 energies log-spaced on [1e-3, 1e3] eV */
#define PIC_EEPF_BINS 240       /* 0..60 eV in 0.25 eV bins */
#define PIC_IFEDF_BINS 256      /* ion energy at each electrode: bins of ifedf_emax_ev / 256 */

/* Case descriptor: versioned plain data, SI units (paper §1's dialog). */
typedef struct {
    uint32_t struct_size;         /* sizeof(pic_case_desc) */
    uint32_t version;             /* PIC_DESC_VERSION */
    int32_t periodic;             /* 1: periodic box; 0: electrodes at x = 0 (driven) and x = L (grounded) */
    int32_t n_cells;              /* 2 .. 4096 */
    double length_m;
    double dt_s;
    double gas_density_m3;        /* N = p / (k_B T_gas) */
    double gas_temp_k;
    double gas_mass_kg;
    double B_T[3];                /* static uniform magnetic field */
    double E_ext_V_per_m[3];      /* static uniform imposed field, added to the mesh field */
    int32_t n_harm;               /* V(t) = sum_h amp_h cos(2 pi f_h t + phase_h) at x = 0 (paper §3.3 form) */
    double harm_freq_hz[4], harm_amp_v[4], harm_phase_rad[4];
    double see_gamma;             /* electrons emitted per ion reaching an electrode */
    double see_temp_ev;           /* temperature of the emitted electrons */
    double background_charge_C_per_m3;   /* immobile uniform charge (paper §3.1 immobile ions) */
    double const_nu_e_per_s;      /* > 0: constant-frequency electron-neutral elastic model instead of tables */
    int32_t n_species;            /* 1 (electrons) or 2 (electrons, ions) */
    double charge_C[2], mass_kg[2], weight_per_m2[2];
    int64_t capacity[2];          /* particle slots per species; 0 = 2x the first load (min 65536) */
    uint64_t seed;                /* Philox key */
    int32_t sort_interval;        /* steps between counting sorts by cell (which also compact); 0 = chosen by
                                     the library's autotuner from timed steps (see pic_step) */
    int32_t diag_interval;        /* energy moments / EEPF every diag_interval steps; 0 = never */
    int32_t rewind;               /* 1: velocities given to pic_load_particles are at t = 0 and are
                                     pushed back by dt/2 before the first step (leapfrog start) */
    int32_t field_history;        /* field-energy history length kept on the device; 0 = 65536 */
    int32_t circuit;              /* electrode at x = 0: 0 = held at V(t); 1 = V(t) through a series
                                     blocking capacitor (bounded cases).  Electrode and capacitor plate
                                     form one conductor whose charge Q changes only by the particles it
                                     absorbs and the secondary electrons it emits; each step
                                     phi_0 (C + eps0/L) = Q + C V + (eps0/dx) phi_p(1) + rho_0 dx/2, phi_p
                                     the potential for phi_0 = 0 (paper §3.3 reports the DC self-bias such
                                     a capacitor develops).  At load the capacitor is uncharged. */
                                  /* 2 = the current density J(t) is imposed on it instead (the harmonics
                                     read as A/m^2, into the electrode; paper §3.2 drives Godyak's
                                     discharges this way): Q also gains J(t^{n+1}) dt each step and
                                     phi_0 eps0/L = Q + (eps0/dx) phi_p(1) + rho_0 dx/2; phi_0 = 0 at load. */
    double blocking_cap_F_per_m2; /* C of circuit 1 (0 = floating electrode) */
    double ifedf_emax_ev;         /* > 0: histogram the energy of the ions reaching each electrode,
                                     PIC_IFEDF_BINS bins on [0, ifedf_emax_ev) (paper §3.3's ion
                                     flux-energy distributions); energies beyond are not counted */
    int32_t no_field;             /* 1: no Poisson solve, the particles feel only E_ext (swarm runs of the
                                     paper's §4); densities and counters are still accumulated */
    double axial_length_m;        /* > 0: axial renewal (paper §3.6, after Lafleur, Baalrud and Chabert):
                                     every particle carries its axial excursion z, advanced by v_z dt
                                     after the push; when |z| reaches this length the particle keeps its
                                     position, takes a new velocity from the renewal Maxwellian below
                                     and z = 0, before the collision test.  Single cases only (not in a
                                     batch); the step then always loads its particles directly. */
    double renew_temp_ev[2];      /* renewal Maxwellian per species: temperature (eV) */
    double renew_drift_m_per_s[2][3];   /* and drift */
    void *stream;                 /* cudaStream_t to enqueue on; NULL = a stream owned by the case */
    /* optional device allocator (e.g. a framework's caching allocator); NULL = cudaMalloc */
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *ctx);
    void *alloc_ctx;
} pic_case_desc;

typedef struct pic_case pic_case;

/* Create a case on the current CUDA device.  Copies the descriptor.
 * Errors: PIC_EINVAL (sizes, version, a floating-point field that is not finite),
 *         PIC_ENOMEM, PIC_ECUDA. */
pic_status pic_create_case(const pic_case_desc *desc, pic_case **out);

/* Load one collision process of one species from a raw table (paper §1:
 * tabulated cross sections, LXCat format): n points of energy (eV,
 * ascending) and cross section (m^2).  The table is sampled onto the
 * 1000-point log grid by linear interpolation in energy (constant beyond
 * its ends, zero below threshold_ev); the collision frequency
 * nu = N sigma g is tabulated there (g: electron speed; for ions the
 * relative speed at centre-of-mass energy eps) and interpolated linearly in
 * ln(eps) during the step.  At most PIC_MAX_PROC processes per species.
 * Errors: PIC_EINVAL (species, kind, n < 1, too many processes, tables
 * combined with the constant-frequency model). */
pic_status pic_load_xsec_table(pic_case *c, int species, int kind, double threshold_ev,
                               const double *energy_ev, const double *sigma_m2, int n);

/* Replace the particles of one species with n particles in the layout above
 * (id may be NULL: ids 0..n-1).  on_device != 0: the pointers are device
 * pointers.  The case restarts at step 0; the next pic_step first solves the
 * field of the loaded state at t = 0 and, if desc.rewind, pushes the
 * velocities back by dt/2.  Errors: PIC_EINVAL (a cell outside [0,n_cells)
 * or offset outside [0,1) is reported by the next synchronising call as
 * PIC_EINVAL), PIC_ECAPACITY (n above capacity). */
pic_status pic_load_particles(pic_case *c, int species, int64_t n, const int32_t *cell,
                              const float *offset, const float *vx, const float *vy,
                              const float *vz, const uint32_t *id, int on_device);

/* Load n particles of a species in SI units (paper §1's statement of the
 * problem: positions along the gap, three velocity components), replacing
 * the species' particles and restarting the case at step 0 like
 * pic_load_particles.  x_m[k] in [0, L) (m); v_m_per_s is n x 3, row-major
 * (vx, vy, vz of particle k at 3k .. 3k+2, m/s); id may be NULL (ids
 * 0..n-1).  on_device = 1: the arrays are device pointers, else host.  The
 * library converts on the device: xi = x * (1/dx) in FP64, cell = floor(xi),
 * offset = xi - cell rounded to FP32 (an offset that rounds up to 1 moves to
 * offset 0 of the next cell; in the last cell it stays just below 1),
 * velocities rounded to FP32.  A position outside [0, L) or not finite is
 * reported as PIC_EINVAL by the next synchronising call after the first
 * step (the same validation as pic_load_particles).  The caller keeps
 * ownership of its arrays.  Errors: PIC_EINVAL, PIC_ECAPACITY (n above the
 * species capacity), PIC_ENOMEM, PIC_ECUDA. */
pic_status pic_load_particles_si(pic_case *c, int species, int64_t n, const double *x_m,
                                 const double *v_m_per_s, const uint32_t *id, int on_device);

/* Load n particles of one species sampled on the GPU from profiles at the
 * nodes (n_nodes values each): number density (m^-3), giving the count per
 * cell through the linear (CIC) density between nodes, and temperature (eV)
 * of an isotropic Maxwellian, plus a drift velocity (m/s, may be NULL).  This
 * is how a case starts from given profiles (a uniform plasma, or profiles
 * predicted by the learned warm start).  Particle k gets id id_base + k and
 * its draws come from Philox under the case seed, counter
 * (id, 0xFFFFFFFF, species << 16 | 0x100 + j, 1), j = 0, 1: word 0 picks the
 * cell (u <= cumulative mass, FP64), word 1 the offset (inverse of the linear
 * density in the cell), words 2..5 three Gaussian components (Box-Muller).
 * Replaces the species' particles, like pic_load_particles.  Scratch for the
 * profile tables comes from the stream-ordered allocator.  Errors: PIC_EINVAL
 * (negative profile, zero total density with n > 0), PIC_ECAPACITY. */
pic_status pic_load_profile(pic_case *c, int species, int64_t n, const double *density,
                            const double *temp_ev, const double drift_m_per_s[3], uint32_t id_base);

/* Enqueue n_steps time steps (paper §1 scheme; step order in the design
 * notes) on the case stream.  Returns after enqueueing; steps are replayed
 * from a CUDA graph of up to 16 steps when no sort falls inside it.  With
 * desc.sort_interval = 0, the first call that has 50 steps to run after the
 * first step runs them as the autotuner (this call then synchronises once):
 * one sort and 32 steps that fit the growth of the step time, giving per
 * species the sort interval K minimising (sort time)/K + mean step time,
 * then 18 steps that time six launch shapes of the step kernel per species
 * (see pic_read_tuning).  The choice is kept per case shape for the process and,
 * if the environment variable PIC1D3V_TUNE_CACHE names a file, in that file
 * (one line per shape: key K0 K1 threads0 stages0 threads1 stages1).  Errors:
 * PIC_ESTATE (no particles loaded), PIC_ECUDA (launch failure). */
pic_status pic_step(pic_case *c, int64_t n_steps);

/* Wait for the case stream and report any error raised by device work.  The
 * device error word is sticky: the same status is reported again until
 * pic_clear_error or the next load. */
pic_status pic_sync(pic_case *c);

/* Wait for the case stream and clear its device error word, so that a case
 * whose step reported PIC_ETIMEOUT or PIC_ECAPACITY can go on (the step that
 * raised it is not repeated). */
pic_status pic_clear_error(pic_case *c);

/* Polls of a staging barrier (the bulk copy of the node field and the
 * collision tables into a step kernel's shared memory) before the step gives
 * up on it and raises PIC_ETIMEOUT; default 2^22.  A wait that gives up still
 * waits (bounded) for the copy it issued before the CTA leaves, so no copy
 * is left writing into shared memory.  For tests of the timeout path: 0 makes
 * every such wait give up at once.  Applies to this case's later steps. */
pic_status pic_set_wait_limit(pic_case *c, uint32_t polls);

/* Live particle count per species (synchronises). */
pic_status pic_count(pic_case *c, int64_t n_alive[2]);

/* Copy the live particles of a species to host buffers of max_n entries
 * (order unspecified).  *n_out = live count; PIC_ECAPACITY if max_n is
 * smaller (nothing beyond max_n written).  Any output pointer may be NULL. */
pic_status pic_read_particles(pic_case *c, int species, int64_t max_n, int64_t *n_out,
                              int32_t *cell, float *offset, float *vx, float *vy, float *vz,
                              uint32_t *id);

/* Collision clock of the live particles of a species, in the order
 * pic_read_particles gives them (paper §4's free flights, §1's null-collision
 * method): clock = 2 k + c, k the steps left before the particle's next
 * collision candidate; c = 1 when that step only ends a gap longer than
 * 131071 steps and draws a fresh one.  Each gap is
 * floor(-ln(u) / (numax dt)), evaluated in FP32, u uniform from word 0 of
 * the particle's block-0 draw of the step that drew it (block 6 at load or
 * creation).  0 for a species without collisions.  *n_out = live count;
 * PIC_ECAPACITY if max_n is smaller. */
pic_status pic_read_clock(pic_case *c, int species, int64_t max_n, int64_t *n_out, uint32_t *clock);

/* Axial excursion z (m) of the live particles of a species, in the order
 * pic_read_particles gives them (desc.axial_length_m > 0; PIC_ESTATE
 * otherwise).  *n_out = live count; PIC_ECAPACITY if max_n is smaller. */
pic_status pic_read_axial(pic_case *c, int species, int64_t max_n, int64_t *n_out, float *z);

/* Copy the FP64 potential and field at the nodes (n_nodes = n_cells for a
 * periodic case, n_cells + 1 otherwise) and, if rho_raw is not NULL, the
 * raw fixed-point deposit of each species (int64, units of 2^-32 particle,
 * n_species x n_nodes) of the last step.  Any pointer may be NULL. */
pic_status pic_read_field(pic_case *c, double *phi, double *E, int64_t *rho_raw);

/* Moment sums accumulated since the last reset (paper §1 diagnostics:
 * density and potential profiles, EEPF, currents).  Caller-owned buffers;
 * any array pointer may be NULL.  Sums over steps: divide by n_steps
 * (n_diag for the diagnostic-step sums). */
typedef struct {
    uint32_t struct_size;          /* sizeof(pic_moments) */
    int32_t n_nodes;               /* out */
    int64_t step;                  /* out: completed steps since load */
    int64_t n_steps, n_diag;       /* out: steps / diagnostic steps in the sums */
    int64_t n_alive[2];            /* out */
    int64_t absorbed[2][2];        /* out: per species, per electrode (x = 0, x = L) */
    int64_t see_emitted, ionizations;
    int64_t candidates[2];         /* out: null-collision candidates */
    int64_t collisions[2][PIC_MAX_PROC];
    double ke_sum[2];              /* out: kinetic energy per area (J/m^2), diagnostic steps */
    double pw_sum[2];              /* out: sum q w v_x E_x(mesh) (W/m^2), diagnostic steps */
    double *dens_sum;              /* [n_species * n_nodes] number density (m^-3), every step */
    double *phi_sum;               /* [n_nodes] potential (V), every step */
    double *en_sum;                /* [n_species * n_nodes] sum w eps (eV m^-3), diagnostic steps */
    double *dens_diag_sum;         /* [n_species * n_nodes] density on diagnostic steps */
    double *eepf;                  /* [PIC_EEPF_BINS] electron counts in the central 10 % of the gap */
    double *field_energy;          /* [field_energy_cap] field energy per area (J/m^2) per step: the
                                      oldest entries the ring of desc.field_history still holds, in
                                      step order (NULL or cap 0: none is copied) */
    int64_t field_energy_cap;      /* in */
    int64_t field_energy_n;        /* out: entries written */
    int32_t reset;                 /* in: nonzero = clear the sums after reading */
    int32_t sort_interval;         /* out: steps between sorts in use (chosen by the autotuner when
                                      desc.sort_interval = 0) */
    double *ifedf;                 /* [2 * PIC_IFEDF_BINS] ion counts per energy bin, electrode x = 0 then
                                      x = L (desc.ifedf_emax_ev > 0) */
    double electrode_charge;       /* out: charge per area of the electrode at x = 0 and its capacitor
                                      plate (circuit 1), C/m^2 */
    int64_t renewed[2];            /* out: axial renewals per species (desc.axial_length_m > 0) */
} pic_moments;

pic_status pic_read_moments(pic_case *c, pic_moments *out);

/* Launch configuration in use, per species, and what the autotuner measured
 * (no counterpart in the paper: a property of this implementation).  With
 * desc.sort_interval = 0 the autotuner picks, per species, the sort interval
 * and the step kernel's launch shape: CTA size (256, 512 or 1024 threads)
 * and particle tiles in flight through shared memory (0 = each thread loads
 * its own particles; 1 or 2 = bulk-copy pipeline); otherwise (1024, 0) and
 * desc.sort_interval stand.  shape_ms[s][k] is the fastest of three timed
 * step-kernel launches of candidate k = (1024,0), (512,0), (256,0), (1024,1),
 * (512,1), (512,2) (the tuner keeps the least); sort_ms
 * the time of one sort; slope_ms the growth of the step-kernel time per step
 * that the tuner extends beyond its timing window (the fitted slope of the
 * window's second half less two standard errors, not below zero; all zero
 * until the autotuner has run, and
 * when its choice came from the cache).  `stages` reports the buffers in use
 * (fewer than chosen when shared memory is short).  Does not synchronise.
 * Errors: PIC_EINVAL (NULL argument or struct_size mismatch). */
typedef struct {
    uint32_t struct_size;          /* in: sizeof(pic_tuning) */
    int32_t tuned;                 /* 1 once the autotuner (or its cache) has chosen */
    int32_t sort_interval[2];
    int32_t threads[2];
    int32_t stages[2];
    int32_t grid[2];               /* CTAs of the last step launch (0 before the first step) */
    float shape_ms[2][6];
    float sort_ms[2];
    float slope_ms[2];
} pic_tuning;

pic_status pic_read_tuning(pic_case *c, pic_tuning *out);

/* Set the step kernel's launch shape for one species by hand (no counterpart
 * in the paper): threads = 256, 512 or 1024 per CTA, stages = particle tiles in
 * flight through shared memory, 0 (each thread loads its own particles) to
 * 4 (fewer are used when shared memory is short).  Results do not depend on
 * the shape.  With desc.sort_interval = 0 an autotuner that has not run yet
 * still chooses later.  Errors: PIC_EINVAL (bad species, threads or stages). */
pic_status pic_set_step_shape(pic_case *c, int species, int threads, int stages);

/* Checkpoint and resume (paper §1: the program saves a run and resumes it).
 * The state between two steps (particles of both species including slots of
 * absorbed particles not yet compacted, the control block with the step
 * counter, drive phases and circuit charge, the field, the moment sums and
 * the sort and launch settings) goes into one caller-owned host buffer.
 * Random numbers are drawn from (id, step) counters, so a case restored into
 * a case created from the same descriptor continues bit-identically to an
 * uninterrupted run.
 *   pic_checkpoint_size: bytes needed now.
 *   pic_checkpoint_save: synchronises, writes the state (bytes >= size).
 *   pic_checkpoint_load: restores into c; c's descriptor must match the saved
 *   one in cells, species, charges, masses, weights, dt, length and seed.
 * Errors: PIC_EINVAL (NULL, buffer too small, not a checkpoint, descriptor
 * mismatch), PIC_ECAPACITY (saved particles exceed c's capacity), PIC_ECUDA. */
pic_status pic_checkpoint_size(pic_case *c, uint64_t *bytes);
pic_status pic_checkpoint_save(pic_case *c, void *host, uint64_t bytes);
pic_status pic_checkpoint_load(pic_case *c, const void *host, uint64_t bytes);

/* Free everything the case owns.  Safe on NULL. */
pic_status pic_destroy(pic_case *c);

/* Per-kernel timing of the step (CUDA events on the case stream around each
 * launch) and launch counts.  pic_profile(c, 1) clears the records and starts
 * recording events; pic_profile(c, 0) stops recording (launch counts are
 * always kept).  pic_profile_read synchronises and returns one entry per
 * kernel class ("particle_step", "field_solve", "sort", "init"). */
typedef struct {
    char name[32];
    int64_t launches;      /* launches since the last pic_profile(c, 1) */
    int64_t timed;         /* launches bracketed by events */
    double total_ms;       /* summed event time of the timed launches */
} pic_kernel_stat;

pic_status pic_profile(pic_case *c, int enable);
pic_status pic_profile_read(pic_case *c, pic_kernel_stat *out, int max_entries, int *n_out);

const char *pic_status_str(pic_status s);
const char *pic_last_error(void);

/* ---------------------------------------------------------------------------
 * Kernel-level entry points (device pointers, enqueued on `stream`, a
 * cudaStream_t or NULL for the default stream).  They expose single steps of
 * the method for unit checks and for callers that manage their own particles.
 * ------------------------------------------------------------------------- */

/* Philox4x32-10 (Salmon et al., SC'11), the counter-based generator that keys
 * every random draw of the step on (particle id, step, stream word): for
 * i < n, out[4i..4i+3] = Philox(key, counter_i) with counter_i =
 * (ctr[4i], ctr[4i+1], ctr[4i+2], ctr[4i+3]).  ctr, out: device, 4n uint32. */
pic_status pic_philox(uint64_t seed, int64_t n, const uint32_t *ctr, uint32_t *out, void *stream);

/* Linear (cloud-in-cell) charge assignment in fixed point (paper §1: the
 * field is computed on the mesh from the particles' own charge): each of the
 * n particles adds 2^32 - f to node cell and f to node cell+1 (periodic: node
 * n_cells is node 0), f = floor(offset 2^32); particles with a cell outside
 * [0, n_cells) or an offset outside [0, 1) are skipped.  R: device int64[n_nodes],
 * accumulated into (not cleared).  Integer sums: bit-reproducible. */
pic_status pic_deposit(int32_t n_cells, int32_t periodic, int64_t n, const int32_t *cell,
                       const float *offset, int64_t *R, void *stream);

/* Counting sort of particles by cell (the periodic sort of the step, as a
 * stand-alone operation): the n input particles (SoA, device) with a cell in
 * [0, n_cells) are written to the output arrays grouped by ascending cell;
 * the others (absorbed: cell < 0, or cell >= n_cells) are dropped.  The order
 * inside one cell is unspecified.  *n_live (device int64, may be NULL)
 * receives the number written.  Inputs and outputs must not overlap.  Scratch
 * (per-cell counts and cursors, 12 B per cell) comes from the stream-ordered
 * allocator (cudaMallocAsync / cudaFreeAsync on `stream`).
 * Errors: PIC_EINVAL (n_cells outside [1, 4096], n < 0, NULL array), PIC_ECUDA. */
pic_status pic_sort_by_cell(int32_t n_cells, int64_t n, const int32_t *cell, const float *offset,
                            const float *vx, const float *vy, const float *vz, const uint32_t *id,
                            int32_t *cell_out, float *offset_out, float *vx_out, float *vy_out,
                            float *vz_out, uint32_t *id_out, int64_t *n_live, void *stream);

/* ---------------------------------------------------------------------------
 * Batched sweep: n independent cases (a parameter sweep of the paper's cases:
 * different pressures, voltages, gaps, cell and particle counts) stepped
 * together.  Each case is an ordinary pic_case created from descs[i] on the
 * batch's stream (descs[0].stream, or one the batch creates); use
 * pic_batch_case(b, i) with the per-case calls to load tables and particles
 * and to read results.  pic_batch_step runs every case's steps with the
 * particles of all cases split into work items (slices of 16384 to 262144
 * particles of one case and species, largest first): either one persistent
 * launch whose CTAs take items from an atomic counter, or a grid of one CTA
 * per item, one launch per species and table of up to 256 cases (the items
 * and the cases' push constants in the kernel parameter); then the field
 * solves, one cluster per case of as few CTAs as its grid needs, one launch
 * per cluster size.  The steps are replayed from CUDA graphs between sorts;
 * every sort_interval steps every case is sorted, one launch per sort kernel
 * and species for all cases.  descs[0].sort_interval > 0 fixes the interval;
 * 0 lets the batch's autotuner choose it and the launch shape, during the
 * first pic_batch_step of at least 44 steps after the first step (12 steps,
 * two per shape, then one sort and 32 timed steps, all part of the run:
 * results do not depend on the choices; see pic_batch_tuning).  All cases must share the boundary kind, the number of species and
 * the collision model of each species (none, tables, or constant frequency
 * for electrons).  Results equal stepping each case alone.
 * Errors: PIC_EINVAL (mixed cases), PIC_ESTATE (a case without particles).
 * ------------------------------------------------------------------------- */
typedef struct pic_batch pic_batch;
pic_status pic_batch_create(const pic_case_desc *descs, int n_cases, pic_batch **out);
/* Borrowed handle of case i (owned by the batch; NULL if out of range). */
pic_case *pic_batch_case(pic_batch *b, int i);
pic_status pic_batch_step(pic_batch *b, int64_t n_steps);
pic_status pic_batch_sync(pic_batch *b);
/* Kernel launches the batch has enqueued (for launch accounting). */
int64_t pic_batch_launches(const pic_batch *b);
/* Particle tiles the batch's step kernel keeps in flight through shared
 * memory (0 = each thread loads its own particles, the default; 1-4 = bulk
 * copies; fewer are used when shared memory is short).  Takes effect at the
 * next pic_batch_step; results do not depend on it.  Errors: PIC_EINVAL. */
pic_status pic_batch_set_stages(pic_batch *b, int stages);
/* Cases with at least `particles` live particles (both species, counted when
 * the batch plans its step) run the single-case step kernels inside the
 * batch's graph instead of the shared batch kernels; every case's field
 * solve stays in the batched launches.  0 = every case in the batch kernels
 * (the default).  Results do not depend on it.  Errors: PIC_EINVAL. */
pic_status pic_batch_set_own_threshold(pic_batch *b, int64_t particles);
/* The batch's launch choices: *shape (the persistent kernel, CTAs taking work
 * items from a counter: 0: 512-thread CTAs, one per SM, chunks of one
 * particle with three in flight; 1: two 512-thread CTAs per SM, chunks of
 * two, one ahead; 2: 1024-thread CTAs, chunks of two, one ahead; 3:
 * 640-thread CTAs, chunks of two, one ahead; or one CTA per work item, the
 * items and the cases' push constants in the kernel parameter, up to 256
 * cases and one species per launch: 4: 1024-thread CTAs, 5: 640-thread
 * CTAs), *sort_interval, *tuned (1 once the autotuner ran), and its
 * measurements: shape_ms[6] (fastest step of each shape over two rounds) and *sort_ms (one
 * batched sort).  Any output pointer may be NULL. */
pic_status pic_batch_tuning(pic_batch *b, int *shape, int *sort_interval, int *tuned, float *shape_ms,
                            float *sort_ms, float *step_ms);
/* (step_ms[32]: the 32 steps the autotuner timed after its sort, in order.) */
/* Run the autotuner again at the next pic_batch_step of at least 44 steps
 * (the discharge of a sweep changes over its first RF cycles, and with it the
 * cost of lost cell order). */
pic_status pic_batch_retune(pic_batch *b);
/* Leave case i out of the batch's steps (frozen != 0) or take it back (0):
 * a frozen case keeps its state, takes no work item, no sort and no field
 * solve, so that cases that have reached what the caller waits for (a steady
 * state, say) stop costing GPU time while the others go on.  Takes effect at
 * the next pic_batch_step (the batch re-plans).  Errors: PIC_EINVAL. */
pic_status pic_batch_freeze(pic_batch *b, int i, int frozen);
/* Fix the launch shape of the batch kernel (0 to 5, as pic_batch_tuning
 * describes them); the autotuner then does not run (with sort_interval 0 the
 * interval stays 64).  Results do not depend on it.  Errors: PIC_EINVAL. */
pic_status pic_batch_set_shape(pic_batch *b, int shape);
pic_status pic_batch_destroy(pic_batch *b);

/* ---------------------------------------------------------------------------
 * Learned warm start (a network that maps a case's parameters to initial
 * profiles, so that a run starts near its steady state): a 3-layer MLP
 * n_in -> n_hidden (GELU) -> n_hidden (GELU) -> n_out, trained and evaluated
 * on the GPU.  Every product takes BF16-rounded operands on the tensor cores
 * (mma m16n8k16) with FP32 accumulation; master weights, gradients and Adam
 * moments are FP32.  Inputs are scaled to [-1, 1] by [in_lo, in_hi], outputs
 * standardised by (out_mean, out_sd); the loss is the mean squared error of
 * the standardised outputs.  Parameters are packed W1 (n_in x n_hidden,
 * row-major), b1, W2, b2, W3, b3.  Host arrays are row-major, n rows.
 * ------------------------------------------------------------------------- */
typedef struct pic_mlp pic_mlp;
/* Glorot-uniform weights from `seed`, zero biases, identity normalisation. */
pic_status pic_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, pic_mlp **out);
pic_status pic_mlp_set_normalization(pic_mlp *m, const float *in_lo, const float *in_hi,
                                     const float *out_mean, const float *out_sd);
int64_t pic_mlp_param_count(const pic_mlp *m);
pic_status pic_mlp_get_params(pic_mlp *m, float *params);
pic_status pic_mlp_set_params(pic_mlp *m, const float *params);   /* also clears the Adam state */
/* Loss and its gradient (packed like the parameters) on n samples. */
pic_status pic_mlp_gradients(pic_mlp *m, const float *X, const float *Y, int n, float *grads, float *loss);
/* `epochs` full-batch Adam steps (lr; beta 0.9, 0.999; eps 1e-8); loss_curve
 * (may be NULL) receives the loss before each step. */
pic_status pic_mlp_train(pic_mlp *m, const float *X, const float *Y, int n, int epochs, float lr,
                         float *loss_curve);
/* One Adam step (the update pic_mlp_train applies: beta 0.9, 0.999, eps 1e-8,
 * bias-corrected, step counter shared with pic_mlp_train) with the given
 * host gradient, packed like the parameters. */
pic_status pic_mlp_adam_step(pic_mlp *m, const float *grads, float lr);
/* Outputs in physical units (normalisation undone). */
pic_status pic_mlp_predict(pic_mlp *m, const float *X, int n, float *Y);
/* Train the warm-start network on n_cases converged runs (paper §2: a run
 * resumed from a converged state answers in minutes; the network stands in
 * for a converged state of a case it has not seen).  params is n_cases x
 * n_params; ne, ni (m^-3) and te (eV) are n_cases x n_points, on points
 * spanning [0, L].  The targets are [log10 max(ne, 1e6), log10 max(ni, 1e6),
 * te] (n_out = 3 n_points, the layout pic_warmstart_load reads); inputs are
 * scaled by [in_lo, in_hi] (n_params each); outputs are standardised by the
 * targets' mean and deviation (+1e-3) over the cases; then `epochs`
 * full-batch Adam steps at lr, loss_curve (may be NULL) receiving the loss
 * before each.  Errors: PIC_EINVAL (sizes that do not match the network, a
 * negative or non-finite profile, in_hi <= in_lo), PIC_ECUDA. */
pic_status pic_warmstart_train(pic_mlp *m, const double *params, const double *ne, const double *ni,
                               const double *te, int n_cases, int n_params, int n_points,
                               const double *in_lo, const double *in_hi, int epochs, float lr,
                               float *loss_curve);
pic_status pic_mlp_destroy(pic_mlp *m);
/* Warm start of a case from the network: predict, for the n_params case
 * parameters, the profiles [log10 n_e (m^-3), log10 n_i (m^-3), T_e (eV)] at
 * n_points points spanning [0, L] (n_out = 3 n_points), interpolate them
 * linearly to the nodes, and load each species with pic_load_profile:
 * count = integral of its density / its weight (capped at max_per_species when
 * that is > 0), electrons at the predicted T_e, ions at ion_temp_ev. */
pic_status pic_warmstart_load(pic_case *c, pic_mlp *m, const double *params, int n_params, int n_points,
                              double ion_temp_ev, uint32_t id_base, int64_t max_per_species);
/* The tensor-core product the MLP uses, on device FP32 arrays:
 * C(i,j) = sum_k A(i,k) B(k,j), A(i,k) = A[i*ar + k*ac], B(k,j) = B[k*br + j*bc],
 * C row-major with leading dimension ldc; operands rounded to BF16. */
pic_status pic_gemm_bf16(const float *A, int ar, int ac, const float *B, int br, int bc, float *C, int ldc,
                         int M, int N, int K, void *stream);

/* Allocation-free variant of pic_sort_by_cell.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * while they run (a fixed device-memory budget set at start-up, a plug-in
 * whose host program owns the device heap, or code that cannot take the
 * device-wide synchronisation cudaMalloc/cudaFree can imply).  Same arguments,
 * layout and result as pic_sort_by_cell; the scratch (12 B per cell) is one
 * fixed device array inside the library, sized for PIC_NOALLOC_MAX_CELLS
 * cells, which every device that loads the library keeps until the process
 * exits.  No cudaMalloc, cudaFree or allocating library routine is called.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress, once per device, with the device current); make
 *     that first call before any stream capture.  The address is kept for the
 *     life of the process: it does not survive cudaDeviceReset (which loads
 *     the library's device code again), so do not call this entry point on a
 *     device after resetting it.
 *   - Every call on a device shares the one array: calls whose GPU work can
 *     overlap (different streams without ordering, or concurrent host threads)
 *     race on it.  Serialise them.
 *   - Errors: PIC_EINVAL (n_cells outside [1, PIC_NOALLOC_MAX_CELLS], n < 0,
 *     NULL array), PIC_ECUDA (message in pic_last_error). */
#define PIC_NOALLOC_MAX_CELLS 4096
pic_status pic_sort_by_cell_noalloc(int32_t n_cells, int64_t n, const int32_t *cell, const float *offset,
                                    const float *vx, const float *vy, const float *vz, const uint32_t *id,
                                    int32_t *cell_out, float *offset_out, float *vx_out, float *vy_out,
                                    float *vz_out, uint32_t *id_out, int64_t *n_live, void *stream);

#ifdef __cplusplus
}
#endif
#endif
