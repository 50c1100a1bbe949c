// pic_device.cuh -- device-side types and helpers of the 1D3V PIC-MCC step.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

constexpr int kMaxProc = 4;
constexpr int kNGrid = 1000;            // cross-section grid, log-spaced on [1e-3, 1e3] eV
constexpr float kGridEmin = 1e-3f;
constexpr int kEepfBins = 240;          // 0..60 eV, 0.25 eV bins
constexpr int kIfedfBins = 256;         // ion energy at each electrode
constexpr int kStepThreads = 1024;     // largest CTA of the particle step
constexpr int kBatchMaxThreads = 1024; // largest CTA of the batched (many-case) particle step
constexpr int kMaxStages = 4;          // particle tiles in flight per CTA (bulk-copy pipeline)
// Copies of each species' raw deposit: CTA b adds its histogram into copy
// b mod kDepositCopies, spreading the int64 atomics of hundreds of CTAs over
// more L2 lines; the field solve sums the copies (exact: integers).
constexpr int kDepositCopies = 8;
constexpr int kFieldThreads = 576;      // >= nodes per CTA of the cluster (4097 / 8 = 513)
constexpr int kFieldCluster = 8;       // CTAs (SMs) sharing one field solve

// device error word bits
constexpr unsigned kErrCapacity = 1u;
constexpr unsigned kErrNumeric = 2u;
constexpr unsigned kErrTimeout = 4u;
constexpr unsigned kErrLoad = 8u;

// Random-draw blocks: counter word 2 is (species << 16) | block.
constexpr uint32_t kBlkMcc = 0, kBlkAux = 1, kBlkNewIon = 2, kBlkSee = 3, kBlkSeeV = 4, kBlkRenew = 5,
                   kBlkGap = 6, kBlkChild = 0xFFFF;

// Cell word of a particle: bits 0-12 the cell index, bits 13-30 its collision
// clock 2 k + c (k non-candidate steps left, c = 1 when that gap was cut at
// kClockMax steps and a fresh one follows), -1 for an absorbed particle.
constexpr int kCellBits = 13;
constexpr int32_t kCellMask = (1 << kCellBits) - 1;
constexpr int kClockMax = 131071;

struct SpeciesBufs {                    // one half of a species' ping-pong storage
    int32_t *cell;
    float *off, *vx, *vy, *vz;
    uint32_t *id;
    float *z;                           // axial excursion (only with axial renewal, else null)
};

// Device-resident control block: counts, step, errors, event counters.
struct Ctrl {
    unsigned long long n_total[2];      // slots in use (append counter)
    unsigned long long n_active[2];     // slots the current step processes
    int32_t cur[2];                     // current ping-pong half per species
    long long step;                     // completed steps since load
    unsigned int err;
    unsigned int pad;
    unsigned long long absorbed[2][2];
    unsigned long long see, iz;
    unsigned long long cand[2];
    unsigned long long coll[2][kMaxProc];
    unsigned long long n_dead[2];       // absorbed slots not yet compacted
    unsigned long long fe_n;            // field-energy history entries written
    unsigned long long n_steps_acc, n_diag_acc;
    double drive_c[4], drive_s[4];      // cos, sin of 2 pi f_h t + theta_h at the next field solve
    double q_el;                        // series capacitor: charge per area of electrode 0 + plate
    unsigned long long st_abs0[2];      // this step: particles absorbed at x = 0 per species
    unsigned long long st_see0;         // this step: secondary electrons emitted at x = 0
    unsigned long long renewed[2];      // axial renewals per species
};

// Constants of the push and of the collision clock, per species; with the
// case's imposed field and Philox key they form CasePush, which a step kernel
// reads from its kernel parameter (constant bank) in the particle loop.
struct SpPush {
    float c_e;                          // q dt / (2 m): half electric kick per V/m
    float cEy, cEz;                     // c_e * E_ext_y, c_e * E_ext_z
    float tB[3], sB[3];                 // Boris rotation vectors t = (q dt / 2m) B, s = 2t/(1+t^2)
    float lam;                          // numax dt in FP32: the collision clock's gap unit (0 = no MCC)
    int rot;                            // 0: B = 0 (no rotation), 1: B along y only, 2: general B
};
struct CasePush {
    float ex_ext;                       // imposed field along x
    uint32_t key0, key1;                // Philox key
    SpPush sp[2];
};

struct SpConst {
    float m_over_2e;                    // eps[eV] = m/(2e) |v|^2
    float v_of_sqrt_eps;                // |v| = sqrt(2e/m) sqrt(eps)
    float numax;
    int nproc;
    int kind[kMaxProc];
    float thr[kMaxProc];
    float recoil;                       // 2 m / M_gas
    float vt_gas;                       // sqrt(k T_gas / M_gas)
    float mfrac, Mfrac;                 // m/(m+M), M/(m+M)
    float mu_over_2e;                   // centre-of-mass energy eps = mu/(2e) |g|^2
    float vt_newion;                    // sqrt(k T_gas / m_ion)
    double q, m, w;
    int mcc;                            // 0 none, 1 tables, 2 constant frequency
    int stages;                         // particle tiles in flight through shared memory (0 = direct loads)
    float renew_vt, renew_drift[3];     // axial renewal Maxwellian: sqrt(kT/m), drift
};

struct StepConst {
    int n_cells, n_nodes, periodic, n_species;
    float dtdx;                         // dt / dx
    CasePush push;
    float see_gamma, see_vth, see_dtdx;
    float eepf_lo, eepf_hi;             // cells: central 10 % of the gap
    float inv_dlog;                     // 1 / (ln(emax/emin)/(NGRID-1)) for the ln-eps interpolation
    int diag_interval;
    unsigned wait_polls;                // polls of a staging mbarrier before a step gives up (kErrTimeout)
    double dx, dt, eps0;
    double vol_interior, vol_wall;
    double bg_charge;
    int n_harm;
    double harm_f[4], harm_a[4], harm_p[4];
    SpConst sp[2];
    const float *nu_tab[2];             // [nproc][kNGrid] per species
    float2 *E32p;                       // [n_cells, padded to 16 B]: (E_c, E_{c+1}) in FP32 for the gather
    double *E, *phi;                    // [n_nodes]
    unsigned long long *R[2];           // [kDepositCopies][r_stride] raw fixed-point deposit (copies summed)
    int r_stride;                       // words between copies (n_cells + 1 rounded up to 16)
    unsigned long long *R_last;         // [2][n_nodes] deposit of the last solve (read-back)
    SpeciesBufs buf[2][2];              // [species][half]
    unsigned long long cap[2];
    Ctrl *ctrl;
    unsigned long long *Rsum, *Rdiag;   // [2][n_nodes] raw deposit summed over steps / diagnostic steps
    double *phi_sum, *en_sum;           // [n_nodes], [2][n_nodes]
    double cq[2];                       // (dx/eps0) q_s w_s 2^-32: Poisson source per raw unit (interior)
    double rho_wall[2];                 // q_s w_s 2^-32 / (dx/2): charge density per raw unit at a wall node
    double bg_r;                        // bg dx^2 / eps0
    double inv_dx, inv_2dx, half_dx_eps0, fe_c;   // 1/dx, 1/(2dx), dx/(2 eps0), eps0 dx / 2
    double inv_n;                       // 1 / n_cells
    double v_init;                      // electrode voltage at t = 0
    double rot_c[4], rot_s[4];          // cos, sin of 2 pi f_h dt (one step of each harmonic's phase)
    double *ke_sum, *pw_sum;            // [2]
    unsigned long long *eepf;           // [kEepfBins]
    double *fe_hist;                    // [fe_cap][kFieldCluster] partial field energies per cluster rank
    long long fe_cap;
    unsigned int *sort_count;           // [n_cells]
    unsigned long long *sort_cursor;    // [n_cells]
    // electrode circuit (series capacitor) and ion energy histograms
    int circuit;                        // 0 = electrode 0 at V(t), 1 = V(t) through a capacitor, 2 = J(t)
    int no_field;                       // 1: E = 0 on the mesh (only E_ext acts)
    float axial_len, dt_f;              // axial renewal length (0 = off), dt in FP32
    double c_blk, eps0_L, inv_cap_eps0_L; // blocking capacitance C, eps0/L, 1/(C + eps0/L)
    double qw[2];                       // q_s w_s: charge per area of one particle
    double r0c[2], bg_half;             // rho_0 dx/2 = sum r0c_s R_s[0] + bg_half
    float ifedf_scale;                  // bins per eV (0 = no histogram)
    unsigned long long *ifedf;          // [2][kIfedfBins]
};

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while the previous kernel of the stream runs;
// grid_dep_wait() blocks until that kernel has completed and its writes are
// visible, grid_dep_launch() lets the next kernel start launching.  Both are
// no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds; each forms
// the 64-bit products of counter words 0 and 2 with the round multipliers,
// xors the high halves with words 1 and 3 and the key, and permutes; the key
// advances by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;   // one wide multiply each
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// 32-bit word -> uniform in (0,1): ((r >> 9) + 1/2) 2^-23, exact in FP32.
__device__ __forceinline__ float u01(uint32_t r)
{
    return __fmaf_rn((float)(r >> 9), 1.0f / 8388608.0f, 0.5f / 8388608.0f);
}

__device__ __forceinline__ uint4 draw(const StepConst &P, uint32_t id, uint32_t step, int sp, uint32_t blk)
{
    return philox4x32_10(make_uint4(id, step, ((uint32_t)sp << 16) | blk, 0u), P.push.key0, P.push.key1);
}

// Null-collision clock (paper §4 free flights; §1 null-collision method).
// The number G of non-candidate steps before a particle's next collision
// candidate is geometric with P(G >= g) = exp(-g numax dt), and
// G = floor(-ln(u) / (numax dt)) has that law for u uniform, so each particle
// draws G once per candidate instead of testing a uniform every step.  The
// gap is evaluated in FP32 with every operation rounded once (IEEE), so that
// the result is the same integer on any conforming implementation.
//
// -ln(u) for u in (0, 1): u = m 2^e, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s)
// with s = (m - 1)/(m + 1), summed as 2 s (1 + s^2/3 + ... + s^10/11)
// (Abramowitz and Stegun 4.1.27; |s| < 0.172).
__device__ __forceinline__ float neg_log_u32(float u)
{
    const uint32_t b = __float_as_uint(u);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
    if (m > 1.41421354f) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float q = 1.0f / 11.0f;
    q = __fmaf_rn(q, s2, 1.0f / 9.0f);
    q = __fmaf_rn(q, s2, 1.0f / 7.0f);
    q = __fmaf_rn(q, s2, 1.0f / 5.0f);
    q = __fmaf_rn(q, s2, 1.0f / 3.0f);
    q = __fmaf_rn(q, s2, 1.0f);
    const float lnm = __fmul_rn(__fadd_rn(s, s), q);
    return -__fmaf_rn((float)e, 0.693147182f, lnm);
}

// Clock state 2 k + c of a fresh gap drawn from the uniform u (lam = numax dt)
__device__ __forceinline__ uint32_t clock_state(float u, float lam)
{
    const float x = __fdiv_rn(neg_log_u32(u), lam);
    if (x >= (float)(kClockMax + 1)) return 2u * kClockMax + 1u;
    return 2u * (uint32_t)floorf(x);
}

// isotropic unit vector from two uniforms: cos(theta) = 1 - 2u, phi = 2 pi u'
__device__ __forceinline__ float3 iso_dir(float ucos, float uphi)
{
    const float ct = 1.0f - 2.0f * ucos;
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float s, c;
    sincospif(2.0f * uphi, &s, &c);
    return make_float3(st * c, st * s, ct);
}

// Box-Muller pair
__device__ __forceinline__ float2 box_muller(float a, float b)
{
    const float r = sqrtf(-2.0f * logf(a));
    float s, c;
    sincospif(2.0f * b, &s, &c);
    return make_float2(r * c, r * s);
}

} // namespace pic
