/*
 * pic_oracle.c -- FP64 CPU oracle of the explicit 1D3V ES PIC-MCC step.
 *
 * TEST INFRASTRUCTURE (see pic_oracle.h): loaded only by the tests, by
 * __graft_entry__.smoke() and by bench.py's CPU legs.  Plain loops, one
 * particle at a time, in the step order stated at or_step().  Nothing here is
 * blocked, fused or reordered for speed.
 *
 * Parity status of each part and what pins it (tests/test_oracle_*.py):
 *   Philox4x32-10 ........ pinned: Triton's Philox run by its CPU interpreter
 *   deposit (CIC) ........ pinned: charge conservation, single-particle weights
 *   Poisson .............. pinned: dense LU (numpy), parabola, periodic sine mode
 *   Boris ................ pinned: |v| invariance, exact rotation angle, ExB drift
 *   leapfrog + CIC field . pinned: cold plasma frequency; Landau root (scipy wofz)
 *   null-collision MCC ... pinned: constant-nu decay exp(-nu t), binomial counts,
 *                          exponential free flights, elastic/inelastic energy balance
 *   walls and SEE ........ pinned: binomial emission counts, flux balance
 *   ionization append .... pinned: one electron + one ion per event, energy balance
 *   moments .............. pinned: uniform-plasma density, Maxwellian Te
 */
#include "pic_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ELEM 1.602176634e-19      /* C */
#define EPS0 8.8541878128e-12     /* F/m */
#define KBOLTZ 1.380649e-23       /* J/K */
#define TWO32 4294967296.0
#define GRID_EMIN 1e-3
#define GRID_EMAX 1e3

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers: */
/* as easy as 1, 2, 3").  Each round: two 32x32->64 products of the even      */
/* counter words with the round multipliers, the high halves xor'ed with the  */
/* odd words and the key, the words permuted; the key is bumped by the Weyl   */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A 32-bit word to a uniform in (0,1): the top 23 bits, centred in their
 * interval, ((r >> 9) + 1/2) 2^-23.  The result has at most 24 significant
 * bits, so it is the same number in FP32 and FP64. */
double or_uniform(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* The draw of block `blk` for particle `id` of species `sp` during step `n`:
 * counter (id, n, sp<<16 | blk, 0), key (seed_lo, seed_hi). */
static void draw(const or_case *c, uint32_t id, int64_t n, int sp, uint32_t blk, uint32_t out[4]);

enum { BLK_MCC = 0, BLK_AUX = 1, BLK_NEWION = 2, BLK_SEE = 3, BLK_SEE_V = 4, BLK_RENEW = 5, BLK_GAP = 6,
       BLK_CHILD = 0xFFFF };

/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, cap;
    double *xi, *vx, *vy, *vz;
    uint32_t *id;
    double *margin;
    int32_t *event;
    double *z;                 /* axial excursion (m), used with axial renewal */
    int32_t *clk;              /* collision clock: 2 k + c (see or_clock_state) */
    double *vloss;             /* diagnostic: speed before the last step's energy-loss collision */
    double *xmove;             /* diagnostic: cells of the last step's move that placed the particle */
} species_t;

typedef struct {
    int kind;
    double thr;
    double nu[OR_NGRID];       /* collision frequency at the grid energies, 1/s */
} proc_t;

struct or_case {
    or_params p;
    int n_nodes;
    double dx;
    species_t sp[OR_MAX_SPECIES];
    species_t pend[OR_MAX_SPECIES];   /* particles created during the current step */
    int n_proc[OR_MAX_SPECIES];
    proc_t proc[OR_MAX_SPECIES][OR_MAX_PROC];
    double numax[OR_MAX_SPECIES];
    double *phi, *E, *rho;
    int64_t *R[OR_MAX_SPECIES];
    int initialised;
    int64_t step;
    or_counters cnt;
    double *dens, *phi_sum, *en, *dens_diag, eepf[OR_EEPF_BINS], ke[OR_MAX_SPECIES], pw[OR_MAX_SPECIES];
    double *fe_hist; int64_t fe_n, fe_cap;
    double q_el;                      /* series-capacitor circuit: charge of electrode 0 + plate, C/m^2 */
    int64_t st_abs0[OR_MAX_SPECIES];  /* this step: particles absorbed at x = 0 */
    int64_t st_see0;                  /* this step: secondary electrons emitted at x = 0 */
    double ifedf[2 * OR_IFEDF_BINS];
};

static void draw(const or_case *c, uint32_t id, int64_t n, int sp, uint32_t blk, uint32_t out[4])
{
    uint32_t ctr[4] = { id, (uint32_t)n, ((uint32_t)sp << 16) | blk, 0u };
    uint32_t key[2] = { (uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32) };
    or_philox4x32_10(ctr, key, out);
}

static int sp_reserve(species_t *s, int64_t cap)
{
    if (cap <= s->cap) return 0;
    int64_t nc = s->cap ? s->cap : 1024;
    while (nc < cap) nc *= 2;
#define GROW(f, T) do { void *q = realloc(s->f, (size_t)nc * sizeof(T)); if (!q) return -1; s->f = q; } while (0)
    GROW(xi, double); GROW(vx, double); GROW(vy, double); GROW(vz, double);
    GROW(id, uint32_t); GROW(margin, double); GROW(event, int32_t); GROW(z, double); GROW(clk, int32_t);
    GROW(vloss, double); GROW(xmove, double);
#undef GROW
    s->cap = nc;
    return 0;
}

static int sp_push(species_t *s, double xi, double vx, double vy, double vz, uint32_t id)
{
    if (sp_reserve(s, s->n + 1)) return -1;
    int64_t k = s->n++;
    s->xi[k] = xi; s->vx[k] = vx; s->vy[k] = vy; s->vz[k] = vz; s->id[k] = id;
    s->margin[k] = INFINITY; s->event[k] = 0; s->z[k] = 0.0; s->clk[k] = 0; s->vloss[k] = 0.0; s->xmove[k] = 0.0;
    return 0;
}

static void sp_free(species_t *s)
{
    free(s->xi); free(s->vx); free(s->vy); free(s->vz); free(s->id); free(s->margin); free(s->event); free(s->z);
    free(s->clk); free(s->vloss); free(s->xmove);
    memset(s, 0, sizeof(*s));
}

or_case *or_create(const or_params *p)
{
    if (!p || p->n_cells < 2 || p->n_species < 1 || p->n_species > OR_MAX_SPECIES || p->dt <= 0 || p->length <= 0)
        return NULL;
    if (p->circuit < 0 || p->circuit > 2 || (p->circuit >= 1 && (p->periodic || !(p->cap >= 0))))
        return NULL;
    or_case *c = calloc(1, sizeof(*c));
    if (!c) return NULL;
    c->p = *p;
    c->n_nodes = p->periodic ? p->n_cells : p->n_cells + 1;
    c->dx = p->length / p->n_cells;
    int nn = c->n_nodes;
    c->phi = calloc(nn, sizeof(double)); c->E = calloc(nn, sizeof(double)); c->rho = calloc(nn, sizeof(double));
    c->phi_sum = calloc(nn, sizeof(double));
    c->dens = calloc((size_t)nn * OR_MAX_SPECIES, sizeof(double));
    c->en = calloc((size_t)nn * OR_MAX_SPECIES, sizeof(double));
    c->dens_diag = calloc((size_t)nn * OR_MAX_SPECIES, sizeof(double));
    for (int s = 0; s < OR_MAX_SPECIES; ++s) c->R[s] = calloc(nn, sizeof(int64_t));
    if (p->const_nu_e > 0) c->numax[0] = p->const_nu_e;
    return c;
}

void or_destroy(or_case *c)
{
    if (!c) return;
    for (int s = 0; s < OR_MAX_SPECIES; ++s) { sp_free(&c->sp[s]); sp_free(&c->pend[s]); free(c->R[s]); }
    free(c->phi); free(c->E); free(c->rho); free(c->phi_sum); free(c->dens); free(c->en); free(c->dens_diag);
    free(c->fe_hist);
    free(c);
}

/* ------------------------------------------------------------------------ */
/* Cross sections (paper §1: tabulated cross sections in the LXCat format).    */
/* Reading: the raw table is sampled, by linear interpolation in energy, onto  */
/* a grid of OR_NGRID energies log-spaced on [1e-3, 1e3] eV (held constant     */
/* beyond its ends, zero below the threshold of an inelastic process); the    */
/* collision frequency nu_k = N sigma_k(eps) g(eps) is stored at the grid      */
/* energies, with g the electron speed, or for ions the relative speed at the  */
/* centre-of-mass energy eps; between grid energies nu_k is linear in ln eps.  */
/* ------------------------------------------------------------------------ */
static double grid_energy(int i)
{
    return GRID_EMIN * exp((double)i * log(GRID_EMAX / GRID_EMIN) / (OR_NGRID - 1));
}

static double raw_sigma(const double *e, const double *s, int n, double eps)
{
    if (eps <= e[0]) return s[0];
    if (eps >= e[n - 1]) return s[n - 1];
    int k = 0;
    while (k + 1 < n && e[k + 1] < eps) ++k;
    double t = (eps - e[k]) / (e[k + 1] - e[k]);
    return s[k] + t * (s[k + 1] - s[k]);
}

/* reduced mass of the pair that defines the energy axis of species sp */
static double pair_mass(const or_case *c, int sp)
{
    double m = c->p.m[sp];
    if (sp == 0) return m;                 /* electrons: the atom is at rest */
    return m * c->p.gas_mass / (m + c->p.gas_mass);
}

static void update_numax(or_case *c, int sp)
{
    double best = 0;
    for (int i = 0; i < OR_NGRID; ++i) {
        double tot = 0;
        for (int k = 0; k < c->n_proc[sp]; ++k) tot += c->proc[sp][k].nu[i];
        if (tot > best) best = tot;
    }
    c->numax[sp] = best;
}

int or_load_xsec(or_case *c, int sp, int kind, double thr, const double *e, const double *s, int n)
{
    if (!c || sp < 0 || sp >= c->p.n_species || n < 1 || c->n_proc[sp] >= OR_MAX_PROC) return -1;
    if (sp == 0 && c->p.const_nu_e > 0) return -1;
    proc_t *pr = &c->proc[sp][c->n_proc[sp]++];
    pr->kind = kind;
    pr->thr = thr;
    double mu = pair_mass(c, sp);
    for (int i = 0; i < OR_NGRID; ++i) {
        double eps = grid_energy(i);
        double sig = (eps < thr) ? 0.0 : raw_sigma(e, s, n, eps);
        double g = sqrt(2.0 * eps * ELEM / mu);
        pr->nu[i] = c->p.gas_density * sig * g;
    }
    update_numax(c, sp);
    return 0;
}

/* nu_k(eps) between grid energies: linear in ln eps; zero below threshold */
static double nu_at(const proc_t *pr, double eps)
{
    if (eps < pr->thr) return 0.0;
    double s;
    if (eps <= GRID_EMIN) s = 0.0;
    else if (eps >= GRID_EMAX) s = OR_NGRID - 1;
    else s = log(eps / GRID_EMIN) / (log(GRID_EMAX / GRID_EMIN) / (OR_NGRID - 1));
    int i = (int)floor(s);
    if (i > OR_NGRID - 2) i = OR_NGRID - 2;
    double t = s - i;
    return (1.0 - t) * pr->nu[i] + t * pr->nu[i + 1];
}

/* ------------------------------------------------------------------------ */
int or_load_particles(or_case *c, int sp, int64_t n, const double *xi, const double *vx,
                      const double *vy, const double *vz, const uint32_t *id)
{
    if (!c || sp < 0 || sp >= c->p.n_species || n < 0) return -1;
    species_t *s = &c->sp[sp];
    for (int64_t k = 0; k < n; ++k) {
        if (!(xi[k] >= 0 && xi[k] < c->p.n_cells)) return -2;
        if (sp_push(s, xi[k], vx[k], vy[k], vz[k], id[k])) return -3;
    }
    c->initialised = 0;
    c->step = 0;
    c->fe_n = 0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Charge assignment.  Reading: linear (cloud-in-cell) weighting, held as an   */
/* integer count in units of 2^-32 particle: a particle at offset delta in     */
/* cell j gives node j the weight 2^32 - f and node j+1 the weight f, with     */
/* f = floor(delta * 2^32).  Periodic: node n_cells is node 0.                 */
/* ------------------------------------------------------------------------ */
void or_deposit(int n_cells, int periodic, int64_t n, const double *xi, int64_t *R)
{
    for (int64_t k = 0; k < n; ++k) {
        double j = floor(xi[k]);
        double delta = xi[k] - j;
        int64_t f = (int64_t)floor(delta * TWO32);
        int jn = (int)j + 1;
        if (periodic && jn == n_cells) jn = 0;
        R[(int)j] += ((int64_t)1 << 32) - f;
        R[jn] += f;
    }
}

/* node volume per unit area: dx, and dx/2 at an electrode */
static double node_vol(const or_case *c, int i)
{
    if (!c->p.periodic && (i == 0 || i == c->n_nodes - 1)) return 0.5 * c->dx;
    return c->dx;
}

/* ------------------------------------------------------------------------ */
/* Poisson's equation (paper §1), second-order differences:                    */
/*   (phi_{i-1} - 2 phi_i + phi_{i+1}) / dx^2 = -rho_i / eps0.                 */
/* Bounded: phi_0 = phi_left, phi_N = 0, Thomas algorithm on nodes 1..N-1.     */
/* Periodic: the mean of rho is removed, phi_0 is fixed at 0 and the same      */
/* Dirichlet system is solved on nodes 1..N-1 (the equation at node 0 then    */
/* holds because sum(rho) = 0); the mean of phi is removed at the end.         */
/* ------------------------------------------------------------------------ */
static void thomas(int m, const double *d, double *x)
{
    /* solves x_{i-1} - 2 x_i + x_{i+1} = d_i, i = 0..m-1, with x_{-1} = x_m = 0 */
    double *cp = malloc(sizeof(double) * (m > 0 ? m : 1));
    double *dp = malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int i = 0; i < m; ++i) {
        double a = (i > 0) ? 1.0 : 0.0, b = -2.0, cc = (i < m - 1) ? 1.0 : 0.0;
        double den = b - a * (i > 0 ? cp[i - 1] : 0.0);
        cp[i] = cc / den;
        dp[i] = (d[i] - a * (i > 0 ? dp[i - 1] : 0.0)) / den;
    }
    for (int i = m - 1; i >= 0; --i) x[i] = dp[i] - (i < m - 1 ? cp[i] * x[i + 1] : 0.0);
    free(cp); free(dp);
}

int or_poisson(int n_cells, int periodic, double dx, const double *rho, double phi_left, double *phi)
{
    int N = n_cells;
    double k2 = dx * dx / EPS0;
    if (!periodic) {
        int m = N - 1;
        double *d = malloc(sizeof(double) * m);
        for (int i = 1; i <= m; ++i) d[i - 1] = -rho[i] * k2;
        d[0] -= phi_left;                       /* phi_N = 0 adds nothing */
        thomas(m, d, phi + 1);
        phi[0] = phi_left;
        phi[N] = 0.0;
        free(d);
    } else {
        double mean = 0;
        for (int i = 0; i < N; ++i) mean += rho[i];
        mean /= N;
        int m = N - 1;
        double *d = malloc(sizeof(double) * m);
        for (int i = 1; i <= m; ++i) d[i - 1] = -(rho[i] - mean) * k2;
        thomas(m, d, phi + 1);
        phi[0] = 0.0;
        double pm = 0;
        for (int i = 0; i < N; ++i) pm += phi[i];
        pm /= N;
        for (int i = 0; i < N; ++i) phi[i] -= pm;
        free(d);
    }
    return 0;
}

/* E = -dphi/dx at the nodes.  Interior: central difference.  Periodic: the
 * same with wrap-around.  Electrode nodes (reading): Gauss's law over the
 * half cell next to the wall, E_0 = -(phi_1-phi_0)/dx - rho_0 dx/(2 eps0) and
 * E_N = -(phi_N-phi_{N-1})/dx + rho_N dx/(2 eps0). */
static void field_from_phi(or_case *c)
{
    int N = c->p.n_cells, nn = c->n_nodes;
    double dx = c->dx;
    if (c->p.periodic) {
        for (int i = 0; i < nn; ++i) {
            int ip = (i + 1) % nn, im = (i - 1 + nn) % nn;
            c->E[i] = -(c->phi[ip] - c->phi[im]) / (2.0 * dx);
        }
    } else {
        for (int i = 1; i < N; ++i) c->E[i] = -(c->phi[i + 1] - c->phi[i - 1]) / (2.0 * dx);
        c->E[0] = -(c->phi[1] - c->phi[0]) / dx - c->rho[0] * dx / (2.0 * EPS0);
        c->E[N] = -(c->phi[N] - c->phi[N - 1]) / dx + c->rho[N] * dx / (2.0 * EPS0);
    }
}

/* electrode voltage at x = 0, V(t) = sum_h A_h cos(2 pi f_h t + theta_h)
 * (paper §1 "voltage waveform"; the two-harmonic form of §3.3) */
static double drive_voltage(const or_case *c, double t)
{
    double v = 0;
    for (int h = 0; h < c->p.n_harm && h < 4; ++h)
        v += c->p.harm_amp[h] * cos(2.0 * M_PI * c->p.harm_freq[h] * t + c->p.harm_phase[h]);
    return v;
}

/* Series blocking capacitor (reading; paper §3.3 reports the DC self-bias
 * such a capacitor develops).  A capacitor of `cap` F/m^2 sits between the
 * source V(t) and the electrode at x = 0.  Electrode and capacitor plate form
 * one isolated conductor whose charge Q per area changes only by the charge
 * of the particles it absorbs and of the secondary electrons it emits.  The
 * plate carries cap (phi_0 - V) and the electrode surface sigma = eps0 E_0,
 * E_0 being the electrode field of Gauss's law over the half cell, so
 *   Q = eps0 E_0 + cap (phi_0 - V).
 * Poisson's solution with phi_N = 0 is linear in phi_0: phi = phi_p + phi_0
 * (1 - i/N), phi_p solving it for phi_0 = 0.  With E_0 = -(phi_1 - phi_0)/dx
 * - rho_0 dx / (2 eps0) this gives
 *   phi_0 (cap + eps0/L) = Q + cap V + (eps0/dx) phi_p[1] + rho_0 dx/2.
 * cap -> infinity is the voltage drive, cap = 0 a floating electrode.  At
 * load the capacitor is uncharged: phi_0 = V(0) and Q = eps0 E_0. */
static double circuit_phi0(const or_case *c, double V)
{
    double L = c->p.length, dx = c->dx;
    return (c->q_el + c->p.cap * V + (EPS0 / dx) * c->phi[1] + 0.5 * c->rho[0] * dx) / (c->p.cap + EPS0 / L);
}

/* Current-source drive (reading; paper §3.2 runs Godyak's discharges with the
 * current imposed): circuit 2 imposes J(t) = sum_h A_h cos(2 pi f_h t +
 * theta_h) (A/m^2, into the electrode) on the electrode at x = 0.  Its charge
 * then changes by J(t^{n+1}) dt each step besides the absorbed and emitted
 * particles, and phi_0 follows from the relation above with no capacitor
 * (cap = 0): phi_0 eps0/L = Q + (eps0/dx) phi_p[1] + rho_0 dx/2.  At load the
 * electrode is at phi_0 = 0 and Q = eps0 E_0. */
static double drive_current(const or_case *c, double t) { return drive_voltage(c, t); }

/* deposit every species, form rho, solve for phi and E at time t */
static void solve_field(or_case *c, double t)
{
    int nn = c->n_nodes, N = c->p.n_cells;
    for (int s = 0; s < c->p.n_species; ++s) {
        memset(c->R[s], 0, sizeof(int64_t) * nn);
        or_deposit(c->p.n_cells, c->p.periodic, c->sp[s].n, c->sp[s].xi, c->R[s]);
    }
    for (int i = 0; i < nn; ++i) {
        double r = c->p.bg_charge;
        for (int s = 0; s < c->p.n_species; ++s)
            r += c->p.q[s] * c->p.w[s] * ((double)c->R[s][i] / TWO32) / node_vol(c, i);
        c->rho[i] = r;
    }
    if (c->p.no_field) {                                         /* swarm: only the imposed field */
        memset(c->phi, 0, sizeof(double) * nn);
        memset(c->E, 0, sizeof(double) * nn);
        return;
    }
    if (!c->p.periodic && c->p.circuit >= 1 && c->initialised) {
        or_poisson(N, 0, c->dx, c->rho, 0.0, c->phi);            /* phi_p */
        double phi0 = circuit_phi0(c, c->p.circuit == 1 ? drive_voltage(c, t) : 0.0);
        for (int i = 0; i <= N; ++i) c->phi[i] += phi0 * (1.0 - (double)i / N);
        c->phi[0] = phi0;
        c->phi[N] = 0.0;
    } else {
        double phi_left = (c->p.periodic || c->p.circuit == 2) ? 0.0 : drive_voltage(c, t);
        or_poisson(c->p.n_cells, c->p.periodic, c->dx, c->rho, phi_left, c->phi);
    }
    field_from_phi(c);
    if (!c->p.periodic && c->p.circuit >= 1 && !c->initialised) c->q_el = EPS0 * c->E[0];
}

/* ------------------------------------------------------------------------ */
/* Boris pusher (paper §1), one velocity update over a time h:                 */
/* half electric kick, rotation about B by the angle 2 atan(qBh/2m), half kick.*/
/* ------------------------------------------------------------------------ */
void or_boris(double qm, double h, const double E[3], const double B[3], double v[3])
{
    double a = 0.5 * qm * h;
    double vm[3] = { v[0] + a * E[0], v[1] + a * E[1], v[2] + a * E[2] };
    double t[3] = { a * B[0], a * B[1], a * B[2] };
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3] = { 2 * t[0] / (1 + t2), 2 * t[1] / (1 + t2), 2 * t[2] / (1 + t2) };
    double vp[3] = { vm[0] + (vm[1] * t[2] - vm[2] * t[1]),
                     vm[1] + (vm[2] * t[0] - vm[0] * t[2]),
                     vm[2] + (vm[0] * t[1] - vm[1] * t[0]) };
    double vq[3] = { vm[0] + (vp[1] * s[2] - vp[2] * s[1]),
                     vm[1] + (vp[2] * s[0] - vp[0] * s[2]),
                     vm[2] + (vp[0] * s[1] - vp[1] * s[0]) };
    v[0] = vq[0] + a * E[0];
    v[1] = vq[1] + a * E[1];
    v[2] = vq[2] + a * E[2];
}

/* linear gather of the mesh field at xi, plus the imposed field */
static void gather(const or_case *c, double xi, double E[3])
{
    int j = (int)floor(xi);
    double d = xi - j;
    int jn = j + 1;
    if (c->p.periodic && jn == c->n_nodes) jn = 0;
    E[0] = (1.0 - d) * c->E[j] + d * c->E[jn] + c->p.E_ext[0];
    E[1] = c->p.E_ext[1];
    E[2] = c->p.E_ext[2];
}

/* ------------------------------------------------------------------------ */
/* Scattering kinematics (readings: isotropic scattering; electrons scatter    */
/* on an atom at rest with the elastic recoil loss (2m/M)(1-cos chi) eps;      */
/* ions scatter isotropically in the centre-of-mass frame; charge exchange     */
/* gives the ion the velocity of its gas partner; ionization shares the        */
/* energy above threshold uniformly between the two electrons).               */
/* ------------------------------------------------------------------------ */
static void iso_dir(double ucos, double uphi, double n[3])
{
    double ct = 1.0 - 2.0 * ucos;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * M_PI * uphi;
    n[0] = st * cos(ph); n[1] = st * sin(ph); n[2] = ct;
}

static void box_muller(double a, double b, double *n0, double *n1)
{
    double r = sqrt(-2.0 * log(a));
    *n0 = r * cos(2.0 * M_PI * b);
    *n1 = r * sin(2.0 * M_PI * b);
}

static double fminabs(double m, double v) { v = fabs(v); return v < m ? v : m; }

/* ------------------------------------------------------------------------ */
/* Null-collision clock (paper §4: free flights between collisions; §1's      */
/* null-collision method).  With P = 1 - exp(-numax dt) the chance that a      */
/* step is a collision candidate, the number G of non-candidate steps before   */
/* the next candidate is geometric, P(G >= g) = exp(-g numax dt), and          */
/* G = floor(-ln(u) / (numax dt)) for u uniform has exactly that law.  So     */
/* instead of a uniform draw every step, each particle draws G once per        */
/* candidate and counts it down.  A clock holds 2 k + c: k more non-candidate  */
/* steps; at the step where k is 0 the particle is a candidate (c = 0), or,    */
/* for a gap longer than OR_CLOCK_MAX steps (c = 1), that step is one more     */
/* non-candidate step after which a fresh gap is drawn (the geometric law is   */
/* memoryless, so this splits one long gap exactly).  The gap is evaluated in  */
/* FP32 with every operation rounded once (IEEE), so that any implementation   */
/* of these operations obtains the same integers.                              */
/* ------------------------------------------------------------------------ */
#define OR_CLOCK_MAX 131071

/* -ln(u) for u in (0, 1), FP32: u = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(s), s = (m - 1)/(m + 1), by the series 2 s (1 + s^2/3 + s^4/5
 * + ... + s^10/11) (Abramowitz and Stegun 4.1.27; |s| < 0.172, so the first
 * omitted term is below 1e-10 relative). */
float or_neg_log_u32(float u)
{
    uint32_t b;
    memcpy(&b, &u, sizeof b);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    uint32_t mb = (b & 0x7FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &mb, sizeof m);
    if (m > 1.41421354f) { m = m * 0.5f; e += 1; }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float q = 1.0f / 11.0f;
    q = fmaf(q, s2, 1.0f / 9.0f);
    q = fmaf(q, s2, 1.0f / 7.0f);
    q = fmaf(q, s2, 1.0f / 5.0f);
    q = fmaf(q, s2, 1.0f / 3.0f);
    q = fmaf(q, s2, 1.0f);
    const float lnm = (s + s) * q;
    return -fmaf((float)e, 0.693147182f, lnm);
}

/* clock state 2 k + c for a fresh gap from the uniform u (FP32 arithmetic) */
int32_t or_clock_state(float u, float lam, double *margin)
{
    const float x = or_neg_log_u32(u) / lam;
    if (margin) {
        *margin = fminabs(*margin, (x - nearbyintf(x)) / fmax(x, 1.0));
        *margin = fminabs(*margin, (x - (float)(OR_CLOCK_MAX + 1)) / (OR_CLOCK_MAX + 1.0));
    }
    if (x >= (float)(OR_CLOCK_MAX + 1)) return 2 * OR_CLOCK_MAX + 1;
    return 2 * (int32_t)floorf(x);
}

static float clock_lambda(const or_case *c, int sp) { return (float)(c->numax[sp] * c->p.dt); }

/* the clock of a particle created (or loaded) during step c->step */
static int32_t first_clock(const or_case *c, int sp, uint32_t id)
{
    if (!(c->numax[sp] > 0)) return 0;
    uint32_t r[4];
    draw(c, id, c->step, sp, BLK_GAP, r);
    return or_clock_state((float)or_uniform(r[0]), clock_lambda(c, sp), NULL);
}

/* append a particle created in this step to the pending list, with its clock */
static void push_new(or_case *c, int sp, double xi, double vx, double vy, double vz, uint32_t id,
                     double vloss, double xmove)
{
    species_t *pd = &c->pend[sp];
    if (sp_push(pd, xi, vx, vy, vz, id)) return;
    pd->clk[pd->n - 1] = first_clock(c, sp, id);
    pd->vloss[pd->n - 1] = vloss;
    pd->xmove[pd->n - 1] = xmove;
}

/* Count the clock down one step.  Returns 1 if this step is a collision
 * candidate; then, or at the end of a long gap, a fresh gap is drawn from
 * word 0 of the step's block-0 draw, which is returned in r. */
static int clock_tick(or_case *c, int sp, int64_t k, uint32_t r[4], double *margin)
{
    species_t *s = &c->sp[sp];
    const int32_t st = s->clk[k];
    if (st >= 2) { s->clk[k] = st - 2; return 0; }
    draw(c, s->id[k], c->step, sp, BLK_MCC, r);
    s->clk[k] = or_clock_state((float)or_uniform(r[0]), clock_lambda(c, sp), margin);
    return (st & 1) ? 0 : 1;
}

/* one electron collision test; returns event code, updates v and margin */
static int collide_electron(or_case *c, int64_t k, double *margin)
{
    species_t *s = &c->sp[0];
    double m = c->p.m[0];
    uint32_t r[4];
    if (!clock_tick(c, 0, k, r, margin)) return 0;
    double u1 = or_uniform(r[1]);
    c->cnt.candidates[0]++;
    double v2 = s->vx[k] * s->vx[k] + s->vy[k] * s->vy[k] + s->vz[k] * s->vz[k];
    double eps = 0.5 * m * v2 / ELEM;
    double x = u1 * c->numax[0];
    int proc = -1, kind = OR_ELASTIC;
    double thr = 0;
    if (c->p.const_nu_e > 0) {
        proc = 0;                               /* every candidate collides */
    } else {
        double cum = 0;
        for (int q = 0; q < c->n_proc[0]; ++q) {
            const proc_t *pr = &c->proc[0][q];
            if (pr->thr > 0) *margin = fminabs(*margin, (eps - pr->thr) / pr->thr);
            cum += nu_at(pr, eps);
            *margin = fminabs(*margin, (x - cum) / c->numax[0]);
            if (proc < 0 && x < cum) { proc = q; kind = pr->kind; thr = pr->thr; }
        }
        if (proc < 0) return 1;                 /* null collision */
    }
    c->cnt.collisions[0][proc]++;
    double speed = sqrt(v2);
    if (kind == OR_EXCITATION || kind == OR_IONIZATION) s->vloss[k] = speed;
    double n[3];
    iso_dir(or_uniform(r[2]), or_uniform(r[3]), n);
    if (kind == OR_ELASTIC) {
        double cchi = speed > 0 ? (s->vx[k] * n[0] + s->vy[k] * n[1] + s->vz[k] * n[2]) / speed : 1.0;
        double epsn = eps * (1.0 - 2.0 * m / c->p.gas_mass * (1.0 - cchi));
        double sp = sqrt(2.0 * epsn * ELEM / m);
        s->vx[k] = sp * n[0]; s->vy[k] = sp * n[1]; s->vz[k] = sp * n[2];
    } else if (kind == OR_EXCITATION) {
        double epsn = fmax(0.0, eps - thr);
        double sp = sqrt(2.0 * epsn * ELEM / m);
        s->vx[k] = sp * n[0]; s->vy[k] = sp * n[1]; s->vz[k] = sp * n[2];
    } else if (kind == OR_IONIZATION) {
        uint32_t a[4], b[4], ids[4];
        draw(c, s->id[k], c->step, 0, BLK_AUX, a);
        draw(c, s->id[k], c->step, 0, BLK_NEWION, b);
        draw(c, s->id[k], c->step, 0, BLK_CHILD, ids);
        double avail = fmax(0.0, eps - thr);
        double eej = or_uniform(a[0]) * avail;
        double esc = avail - eej;
        double sp = sqrt(2.0 * esc * ELEM / m);
        s->vx[k] = sp * n[0]; s->vy[k] = sp * n[1]; s->vz[k] = sp * n[2];
        double ne[3];
        iso_dir(or_uniform(a[1]), or_uniform(a[2]), ne);
        double spe = sqrt(2.0 * eej * ELEM / m);
        push_new(c, 0, s->xi[k], spe * ne[0], spe * ne[1], spe * ne[2], ids[0], speed, s->xmove[k]);
        if (c->p.n_species > 1) {
            double g0, g1, g2, g3;
            box_muller(or_uniform(b[0]), or_uniform(b[1]), &g0, &g1);
            box_muller(or_uniform(b[2]), or_uniform(b[3]), &g2, &g3);
            double vt = sqrt(KBOLTZ * c->p.gas_temp / c->p.m[1]);
            push_new(c, 1, s->xi[k], vt * g0, vt * g1, vt * g2, ids[1], 0.0, s->xmove[k]);
        }
        c->cnt.ionizations++;
    }
    return 2 + proc;
}

static int collide_ion(or_case *c, int64_t k, double *margin)
{
    species_t *s = &c->sp[1];
    double m = c->p.m[1], M = c->p.gas_mass;
    uint32_t r[4], a[4];
    if (!clock_tick(c, 1, k, r, margin)) return 0;
    double u1 = or_uniform(r[1]);
    c->cnt.candidates[1]++;
    /* gas partner drawn from the Maxwellian at the gas temperature */
    draw(c, s->id[k], c->step, 1, BLK_AUX, a);
    double g0, g1, g2, g3;
    box_muller(or_uniform(a[0]), or_uniform(a[1]), &g0, &g1);
    box_muller(or_uniform(a[2]), or_uniform(a[3]), &g2, &g3);
    double vt = sqrt(KBOLTZ * c->p.gas_temp / M);
    double vg[3] = { vt * g0, vt * g1, vt * g2 };
    double gr[3] = { s->vx[k] - vg[0], s->vy[k] - vg[1], s->vz[k] - vg[2] };
    double g2n = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    double mu = m * M / (m + M);
    double eps = 0.5 * mu * g2n / ELEM;
    double x = u1 * c->numax[1];
    double cum = 0;
    int proc = -1, kind = OR_ISO;
    for (int q = 0; q < c->n_proc[1]; ++q) {
        const proc_t *pr = &c->proc[1][q];
        if (pr->thr > 0) *margin = fminabs(*margin, (eps - pr->thr) / pr->thr);
        cum += nu_at(pr, eps);
        *margin = fminabs(*margin, (x - cum) / c->numax[1]);
        if (proc < 0 && x < cum) { proc = q; kind = pr->kind; }
    }
    if (proc < 0) return 1;
    c->cnt.collisions[1][proc]++;
    if (kind == OR_CX) {
        s->vx[k] = vg[0]; s->vy[k] = vg[1]; s->vz[k] = vg[2];
    } else {
        double n[3];
        iso_dir(or_uniform(r[2]), or_uniform(r[3]), n);
        double gm = sqrt(g2n);
        double vc[3] = { (m * s->vx[k] + M * vg[0]) / (m + M), (m * s->vy[k] + M * vg[1]) / (m + M),
                         (m * s->vz[k] + M * vg[2]) / (m + M) };
        double f = M / (m + M) * gm;
        s->vx[k] = vc[0] + f * n[0]; s->vy[k] = vc[1] + f * n[1]; s->vz[k] = vc[2] + f * n[2];
    }
    return 2 + proc;
}

/* Secondary emission (paper §1 "walls and secondary emission").  Reading: an
 * ion reaching a wall releases an electron with probability gamma; the
 * electron leaves the wall with a flux-weighted half-Maxwellian velocity at
 * see_temp_ev (normal component Rayleigh, tangential components Gaussian),
 * placed a random fraction of one step's flight into the gap. */
static void emit_secondary(or_case *c, uint32_t ion_id, int wall, double *margin)
{
    uint32_t r[4], b[4], ids[4];
    draw(c, ion_id, c->step, 1, BLK_SEE, r);
    double u = or_uniform(r[0]);
    *margin = fminabs(*margin, u - c->p.see_gamma);
    if (u >= c->p.see_gamma) return;
    draw(c, ion_id, c->step, 1, BLK_SEE_V, b);
    draw(c, ion_id, c->step, 1, BLK_CHILD, ids);
    double vth = sqrt(c->p.see_temp_ev * ELEM / c->p.m[0]);
    double vn = vth * sqrt(-2.0 * log(or_uniform(r[1])));
    double t0, t1;
    box_muller(or_uniform(b[0]), or_uniform(b[1]), &t0, &t1);
    double d = or_uniform(r[2]) * vn * c->p.dt / c->dx;     /* cells from the wall */
    double N = c->p.n_cells;
    if (d >= N) d = 0.5 * N;
    double xi = wall == 0 ? d : N - d;
    if (xi >= N) xi = nextafter(N, 0.0);
    double vx = wall == 0 ? vn : -vn;
    push_new(c, 0, xi, vx, vth * t0, vth * t1, ids[0], 0.0, d);
    c->cnt.see_emitted++;
    if (wall == 0) c->st_see0++;
}

/* Axial renewal (paper §3.6: a periodic azimuthal box holds the ECDI only if
 * particles are renewed after a virtual axial transit, the method of
 * Lafleur, Baalrud and Chabert).  Reading: each particle carries its axial
 * excursion z, advanced by v_z dt after the push; when |z| reaches
 * axial_len the particle keeps its azimuthal position and gets a new
 * velocity from the species' renewal Maxwellian (temperature and drift), and
 * z = 0.  It happens before the collision test of the step.  Draws: Philox
 * block BLK_RENEW, words 0-1 and 2-3 through Box-Muller (x, y; z). */
static void renew(or_case *c, int s, int64_t k)
{
    species_t *sp = &c->sp[s];
    uint32_t r[4];
    draw(c, sp->id[k], c->step, s, BLK_RENEW, r);
    double g0, g1, g2, g3;
    box_muller(or_uniform(r[0]), or_uniform(r[1]), &g0, &g1);
    box_muller(or_uniform(r[2]), or_uniform(r[3]), &g2, &g3);
    double vt = sqrt(c->p.renew_temp_ev[s] * ELEM / c->p.m[s]);
    sp->vx[k] = c->p.renew_drift[s][0] + vt * g0;
    sp->vy[k] = c->p.renew_drift[s][1] + vt * g1;
    sp->vz[k] = c->p.renew_drift[s][2] + vt * g2;
    c->cnt.renewed[s]++;
}

/* ------------------------------------------------------------------------ */
/* Leapfrog start (reading): the first step solves the field of the loaded     */
/* state at t = 0 and pushes the velocities back by dt/2 with a Boris step.   */
/* ------------------------------------------------------------------------ */
static void initialise(or_case *c)
{
    for (int s = 0; s < c->p.n_species; ++s)                 /* every loaded particle's first gap */
        for (int64_t k = 0; k < c->sp[s].n; ++k) c->sp[s].clk[k] = first_clock(c, s, c->sp[s].id[k]);
    solve_field(c, 0.0);
    if (c->p.rewind) {
        for (int s = 0; s < c->p.n_species; ++s) {
            species_t *sp = &c->sp[s];
            double qm = c->p.q[s] / c->p.m[s];
            for (int64_t k = 0; k < sp->n; ++k) {
                double E[3], v[3] = { sp->vx[k], sp->vy[k], sp->vz[k] };
                gather(c, sp->xi[k], E);
                or_boris(qm, -0.5 * c->p.dt, E, c->p.B, v);
                sp->vx[k] = v[0]; sp->vy[k] = v[1]; sp->vz[k] = v[2];
            }
        }
    }
    c->initialised = 1;
}

static int is_diag_step(const or_case *c)
{
    return c->p.diag_interval > 0 && ((c->step + 1) % c->p.diag_interval) == 0;
}

/* CIC weights of a position onto its two nodes, as fractions */
static void cic(const or_case *c, double xi, int *j, int *jn, double *w0, double *w1)
{
    *j = (int)floor(xi);
    double d = xi - *j;
    *jn = *j + 1;
    if (c->p.periodic && *jn == c->n_nodes) *jn = 0;
    *w0 = 1.0 - d; *w1 = d;
}

/* ------------------------------------------------------------------------ */
/* One time step n -> n+1.  Order (state x^n, v^{n-1/2}, E^n on entry):        */
/*   1 gather E^n at x^n; 2 Boris v^{n-1/2} -> v^{n+1/2}; 3 x^{n+1} = x^n +    */
/*   v_x dt; 4 walls: absorb, secondary emission; 5 null-collision MCC with    */
/*   v^{n+1/2} at x^{n+1}; 6 append the particles created in 4-5 (they are     */
/*   not moved or collided in the step that creates them); 7 deposit rho^{n+1}*/
/*   of all particles; 8 Poisson at t^{n+1} with V(t^{n+1}); 9 E^{n+1};        */
/*   10 moments.                                                               */
/* ------------------------------------------------------------------------ */
static int one_step(or_case *c)
{
    const or_params *p = &c->p;
    int N = p->n_cells, nn = c->n_nodes;
    double dtdx = p->dt / c->dx;
    int diag = is_diag_step(c);
    for (int s = 0; s < p->n_species; ++s) c->pend[s].n = 0;

    for (int s = 0; s < p->n_species; ++s) {
        species_t *sp = &c->sp[s];
        double qm = p->q[s] / p->m[s];
        int64_t keep = 0;
        for (int64_t k = 0; k < sp->n; ++k) {
            double margin = INFINITY;
            int event = 0;
            sp->vloss[k] = 0.0;
            double E[3], v[3] = { sp->vx[k], sp->vy[k], sp->vz[k] };
            gather(c, sp->xi[k], E);                                 /* 1 */
            or_boris(qm, p->dt, E, p->B, v);                         /* 2 */
            sp->vx[k] = v[0]; sp->vy[k] = v[1]; sp->vz[k] = v[2];
            double xn = sp->xi[k] + v[0] * dtdx;                     /* 3 */
            sp->xmove[k] = fabs(v[0] * dtdx);
            margin = fminabs(margin, xn - floor(xn + 0.5));
            int absorbed = -1;
            if (p->periodic) {                                       /* x modulo the box, any distance */
                xn -= N * floor(xn / N);
                if (xn >= N) xn -= N;                                /* rounding of a tiny negative xn */
            } else if (xn < 0) {
                absorbed = 0;
            } else if (xn >= N) {
                absorbed = 1;
            }
            if (diag)                                                /* J.E with the mesh field */
                c->pw[s] += p->q[s] * p->w[s] * v[0] * (E[0] - p->E_ext[0]);
            if (absorbed >= 0) {                                     /* 4 */
                c->cnt.absorbed[s][absorbed]++;
                if (absorbed == 0) c->st_abs0[s]++;
                if (s == 1 && p->ifedf_emax_ev > 0) {                /* ion energy at the electrode */
                    double eps = 0.5 * p->m[1] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / ELEM;
                    double b = floor(eps / p->ifedf_emax_ev * OR_IFEDF_BINS);
                    if (b >= 0 && b < OR_IFEDF_BINS) c->ifedf[absorbed * OR_IFEDF_BINS + (int)b] += 1.0;
                }
                if (s == 1 && p->see_gamma > 0) emit_secondary(c, sp->id[k], absorbed, &margin);
                continue;
            }
            sp->xi[k] = xn;
            if (p->axial_len > 0) {                                  /* axial renewal */
                double zn = sp->z[k] + v[2] * p->dt;
                margin = fminabs(margin, (fabs(zn) - p->axial_len) / p->axial_len);
                if (fabs(zn) >= p->axial_len) {
                    renew(c, s, k);
                    zn = 0.0;
                    event = -2;
                }
                sp->z[k] = zn;
            }
            if (c->numax[s] > 0) {                                   /* 5, 6 */
                if (s == 0) event = collide_electron(c, k, &margin);
                else event = collide_ion(c, k, &margin);
            }
            /* compact in place */
            sp->xi[keep] = sp->xi[k]; sp->vx[keep] = sp->vx[k]; sp->vy[keep] = sp->vy[k];
            sp->vz[keep] = sp->vz[k]; sp->id[keep] = sp->id[k]; sp->z[keep] = sp->z[k];
            sp->margin[keep] = margin; sp->event[keep] = event; sp->clk[keep] = sp->clk[k];
            sp->vloss[keep] = sp->vloss[k]; sp->xmove[keep] = sp->xmove[k];
            ++keep;
        }
        sp->n = keep;
    }
    for (int s = 0; s < p->n_species; ++s) {                          /* 6 */
        species_t *pd = &c->pend[s];
        for (int64_t k = 0; k < pd->n; ++k) {
            if (sp_push(&c->sp[s], pd->xi[k], pd->vx[k], pd->vy[k], pd->vz[k], pd->id[k])) return -1;
            c->sp[s].clk[c->sp[s].n - 1] = pd->clk[k];
            c->sp[s].vloss[c->sp[s].n - 1] = pd->vloss[k];
            c->sp[s].xmove[c->sp[s].n - 1] = pd->xmove[k];
        }
    }
    if (p->circuit >= 1) {                                           /* charge reaching electrode 0 */
        double dq = p->q[0] * p->w[0] * (double)c->st_abs0[0];
        if (p->n_species > 1) dq += p->q[1] * p->w[1] * (double)c->st_abs0[1];
        dq -= p->q[0] * p->w[0] * (double)c->st_see0;                 /* an emitted electron leaves it */
        if (p->circuit == 2) dq += p->dt * drive_current(c, (double)(c->step + 1) * p->dt);
        c->q_el += dq;
    }
    c->st_abs0[0] = c->st_abs0[1] = 0;
    c->st_see0 = 0;
    solve_field(c, (double)(c->step + 1) * p->dt);                    /* 7, 8, 9 */
    /* 10: moments.  Every step: density and potential.  Diagnostic steps:
     * energy moment, EEPF, kinetic energy over every particle alive after
     * the append (v^{n+1/2} at x^{n+1}), and the density of that step. */
    for (int s = 0; s < p->n_species; ++s)
        for (int i = 0; i < nn; ++i) {
            double d = p->w[s] * ((double)c->R[s][i] / TWO32) / node_vol(c, i);
            c->dens[s * nn + i] += d;
            if (diag) c->dens_diag[s * nn + i] += d;
        }
    if (diag) {
        for (int s = 0; s < p->n_species; ++s) {
            species_t *sp = &c->sp[s];
            for (int64_t k = 0; k < sp->n; ++k) {
                double v2 = sp->vx[k] * sp->vx[k] + sp->vy[k] * sp->vy[k] + sp->vz[k] * sp->vz[k];
                double eps = 0.5 * p->m[s] * v2 / ELEM;
                int j, jn; double w0, w1;
                cic(c, sp->xi[k], &j, &jn, &w0, &w1);
                c->en[s * nn + j] += p->w[s] * eps * w0 / node_vol(c, j);
                c->en[s * nn + jn] += p->w[s] * eps * w1 / node_vol(c, jn);
                c->ke[s] += 0.5 * p->m[s] * p->w[s] * v2;
                if (s == 0 && sp->xi[k] >= 0.45 * N && sp->xi[k] < 0.55 * N) {
                    int b = (int)floor(eps / 0.25);
                    if (b < OR_EEPF_BINS) c->eepf[b] += 1.0;
                }
            }
        }
    }
    for (int i = 0; i < nn; ++i) c->phi_sum[i] += c->phi[i];
    c->cnt.n_steps++;
    if (diag) c->cnt.n_diag++;
    double fe = 0;
    for (int i = 0; i < nn; ++i) fe += 0.5 * EPS0 * c->E[i] * c->E[i] * node_vol(c, i);
    if (c->fe_n == c->fe_cap) {
        int64_t nc = c->fe_cap ? 2 * c->fe_cap : 4096;
        double *q = realloc(c->fe_hist, sizeof(double) * nc);
        if (!q) return -1;
        c->fe_hist = q; c->fe_cap = nc;
    }
    c->fe_hist[c->fe_n++] = fe;
    c->step++;
    c->cnt.step = c->step;
    return 0;
}

int or_step(or_case *c, int64_t n_steps)
{
    if (!c) return -1;
    if (!c->initialised) initialise(c);
    for (int64_t i = 0; i < n_steps; ++i)
        if (one_step(c)) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
int64_t or_count(const or_case *c, int sp) { return (c && sp >= 0 && sp < OR_MAX_SPECIES) ? c->sp[sp].n : -1; }

int or_get_particles(const or_case *c, int sp, double *xi, double *vx, double *vy, double *vz,
                     uint32_t *id, double *margin, int32_t *event)
{
    if (!c || sp < 0 || sp >= c->p.n_species) return -1;
    const species_t *s = &c->sp[sp];
    size_t n = (size_t)s->n;
    if (xi) memcpy(xi, s->xi, n * sizeof(double));
    if (vx) memcpy(vx, s->vx, n * sizeof(double));
    if (vy) memcpy(vy, s->vy, n * sizeof(double));
    if (vz) memcpy(vz, s->vz, n * sizeof(double));
    if (id) memcpy(id, s->id, n * sizeof(uint32_t));
    if (margin) memcpy(margin, s->margin, n * sizeof(double));
    if (event) memcpy(event, s->event, n * sizeof(int32_t));
    return 0;
}

int or_get_loss_speed(const or_case *c, int sp, double *v)
{
    if (!c || sp < 0 || sp >= c->p.n_species || !v) return -1;
    memcpy(v, c->sp[sp].vloss, (size_t)c->sp[sp].n * sizeof(double));
    return 0;
}

int or_get_move(const or_case *c, int sp, double *d)
{
    if (!c || sp < 0 || sp >= c->p.n_species || !d) return -1;
    memcpy(d, c->sp[sp].xmove, (size_t)c->sp[sp].n * sizeof(double));
    return 0;
}

int or_get_clock(const or_case *c, int sp, int32_t *clk)
{
    if (!c || sp < 0 || sp >= c->p.n_species || !clk) return -1;
    memcpy(clk, c->sp[sp].clk, (size_t)c->sp[sp].n * sizeof(int32_t));
    return 0;
}

int or_get_axial(const or_case *c, int sp, double *z)
{
    if (!c || sp < 0 || sp >= c->p.n_species || !z) return -1;
    memcpy(z, c->sp[sp].z, (size_t)c->sp[sp].n * sizeof(double));
    return 0;
}

int or_get_field(const or_case *c, double *phi, double *E)
{
    if (!c) return -1;
    if (phi) memcpy(phi, c->phi, sizeof(double) * c->n_nodes);
    if (E) memcpy(E, c->E, sizeof(double) * c->n_nodes);
    return 0;
}

int or_get_deposit(const or_case *c, int sp, int64_t *R)
{
    if (!c || sp < 0 || sp >= c->p.n_species) return -1;
    memcpy(R, c->R[sp], sizeof(int64_t) * c->n_nodes);
    return 0;
}

int or_get_numax(const or_case *c, int sp, double *numax)
{
    if (!c || sp < 0 || sp >= OR_MAX_SPECIES) return -1;
    *numax = c->numax[sp];
    return 0;
}

int or_get_nu_table(const or_case *c, int sp, int k, double *nu)
{
    if (!c || sp < 0 || sp >= OR_MAX_SPECIES || k < 0 || k >= c->n_proc[sp]) return -1;
    memcpy(nu, c->proc[sp][k].nu, sizeof(double) * OR_NGRID);
    return 0;
}

void or_get_counters(const or_case *c, or_counters *out) { *out = c->cnt; }

int or_get_moments(const or_case *c, double *dens, double *phi_sum, double *en, double *dens_diag,
                   double *eepf, double *ke, double *pw)
{
    if (!c) return -1;
    size_t nn = (size_t)c->n_nodes;
    if (dens) memcpy(dens, c->dens, sizeof(double) * nn * OR_MAX_SPECIES);
    if (phi_sum) memcpy(phi_sum, c->phi_sum, sizeof(double) * nn);
    if (en) memcpy(en, c->en, sizeof(double) * nn * OR_MAX_SPECIES);
    if (dens_diag) memcpy(dens_diag, c->dens_diag, sizeof(double) * nn * OR_MAX_SPECIES);
    if (eepf) memcpy(eepf, c->eepf, sizeof(double) * OR_EEPF_BINS);
    if (ke) memcpy(ke, c->ke, sizeof(double) * OR_MAX_SPECIES);
    if (pw) memcpy(pw, c->pw, sizeof(double) * OR_MAX_SPECIES);
    return 0;
}

void or_reset_moments(or_case *c)
{
    size_t nn = (size_t)c->n_nodes;
    memset(c->dens, 0, sizeof(double) * nn * OR_MAX_SPECIES);
    memset(c->phi_sum, 0, sizeof(double) * nn);
    memset(c->en, 0, sizeof(double) * nn * OR_MAX_SPECIES);
    memset(c->dens_diag, 0, sizeof(double) * nn * OR_MAX_SPECIES);
    memset(c->eepf, 0, sizeof(c->eepf));
    memset(c->ifedf, 0, sizeof(c->ifedf));
    memset(c->ke, 0, sizeof(c->ke));
    memset(c->pw, 0, sizeof(c->pw));
    int64_t step = c->cnt.step;
    memset(&c->cnt, 0, sizeof(c->cnt));
    c->cnt.step = step;
}

/* Loading from node profiles: n particles of species sp, ids id_base + k.
 * Cell: the j with cdf[j] <= u < cdf[j+1], cdf the normalised cumulative mass
 * (n_j + n_{j+1})/2 of the linear density between nodes (node N = node 0 when
 * periodic).  Offset: inverse of the linear density a(1-d) + b d on [0, 1),
 * d = u' (a+b) / (a + sqrt(a^2 + u' (b^2 - a^2))).  Velocity: isotropic
 * Maxwellian at the linearly interpolated temperature plus the drift.
 * Draws: Philox counter (id, 0xFFFFFFFF, sp << 16 | 0x100 + j, 1). */
int or_load_profile(or_case *c, int sp, int64_t n, const double *density, const double *temp_ev,
                    const double drift[3], uint32_t id_base)
{
    if (!c || sp < 0 || sp >= c->p.n_species || n < 0) return -1;
    int N = c->p.n_cells;
    double *cdf = calloc((size_t)N + 1, sizeof(double));
    double *dn = malloc(sizeof(double) * ((size_t)N + 1)), *tn = malloc(sizeof(double) * ((size_t)N + 1));
    for (int j = 0; j <= N; ++j) {
        int jj = (c->p.periodic && j == N) ? 0 : j;
        dn[j] = density[jj];
        tn[j] = temp_ev[jj];
    }
    for (int j = 0; j < N; ++j) cdf[j + 1] = cdf[j] + 0.5 * (density[j] + density[(c->p.periodic && j + 1 == N) ? 0 : j + 1]);
    double total = cdf[N];
    for (int j = 1; j < N; ++j) cdf[j] /= total;
    cdf[N] = 1.0;
    uint32_t key[2] = { (uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32) };
    species_t *s = &c->sp[sp];
    s->n = 0;
    for (int64_t k = 0; k < n; ++k) {
        uint32_t id = id_base + (uint32_t)k;
        uint32_t ctr[4] = { id, 0xFFFFFFFFu, ((uint32_t)sp << 16) | 0x100u, 1u }, r[4], r2[4];
        or_philox4x32_10(ctr, key, r);
        ctr[2] = ((uint32_t)sp << 16) | 0x101u;
        or_philox4x32_10(ctr, key, r2);
        double u = or_uniform(r[0]);
        int j = 0;
        while (j + 1 < N && cdf[j + 1] <= u) ++j;
        double a = dn[j], b = dn[j + 1], u2 = or_uniform(r[1]);
        double den = a + sqrt(fmax(a * a + u2 * (b * b - a * a), 0.0));
        double d = den > 0 ? u2 * (a + b) / den : u2;
        double T = (1.0 - d) * tn[j] + d * tn[j + 1];
        double vt = sqrt(fmax(T, 0.0) * ELEM / c->p.m[sp]);
        double g0, g1, g2, g3;
        box_muller(or_uniform(r[2]), or_uniform(r[3]), &g0, &g1);
        box_muller(or_uniform(r2[0]), or_uniform(r2[1]), &g2, &g3);
        double dr[3] = { drift ? drift[0] : 0, drift ? drift[1] : 0, drift ? drift[2] : 0 };
        if (sp_push(s, j + d, vt * g0 + dr[0], vt * g1 + dr[1], vt * g2 + dr[2], id)) { free(cdf); free(dn); free(tn); return -3; }
    }
    free(cdf); free(dn); free(tn);
    c->initialised = 0;
    c->step = 0;
    c->fe_n = 0;
    return 0;
}

/* Counting sort by cell (the periodic reordering of the particle arrays):
 * the indices of the particles whose cell lies in [0, n_cells), grouped by
 * ascending cell and, inside a cell, in input order.  Returns how many. */
int64_t or_sort_by_cell(int n_cells, int64_t n, const int32_t *cell, int64_t *perm)
{
    int64_t *start = calloc((size_t)n_cells + 1, sizeof(int64_t));
    if (!start) return -1;
    for (int64_t k = 0; k < n; ++k)
        if (cell[k] >= 0 && cell[k] < n_cells) start[cell[k] + 1]++;
    for (int j = 0; j < n_cells; ++j) start[j + 1] += start[j];
    int64_t kept = start[n_cells];
    for (int64_t k = 0; k < n; ++k)
        if (cell[k] >= 0 && cell[k] < n_cells) perm[start[cell[k]]++] = k;
    free(start);
    return kept;
}

int or_get_ifedf(const or_case *c, double *out)
{
    if (!c || !out) return -1;
    memcpy(out, c->ifedf, sizeof(c->ifedf));
    return 0;
}

double or_get_electrode_charge(const or_case *c) { return c ? c->q_el : 0.0; }

int64_t or_get_field_energy(const or_case *c, double *out, int64_t max_n)
{
    int64_t n = c->fe_n < max_n ? c->fe_n : max_n;
    if (out) memcpy(out, c->fe_hist, sizeof(double) * (size_t)n);
    return c->fe_n;
}
