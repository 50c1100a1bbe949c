// pic_api.cu -- host runtime behind the C ABI of include/pic1d3v.h.
#include "pic1d3v.h"
#include "pic_device.cuh"
#include "particle_step.cuh"
#include "field_sort.cuh"
#include "sort_interval.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace pic;

namespace {

constexpr double kElem = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kBoltz = 1.380649e-23;
constexpr double kEmin = 1e-3, kEmax = 1e3;

thread_local std::string g_err;

pic_status fail(pic_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

#define CU(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(PIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Longest CUDA graph of steps replayed by pic_step; graphs of every length
// 1..kGraphSteps are kept so that a run of steps cut short by a sort or by
// the end of the call still replays a graph.
constexpr int kGraphSteps = 16;

struct Proc {
    int kind;
    double thr;
    std::vector<double> nu;   // collision frequency at the grid energies (FP64)
};

} // namespace

struct pic_case {
    pic_case_desc d{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 0;
    int n_nodes = 0;
    StepConst P{};
    std::vector<std::pair<void *, size_t>> allocs;
    void *h_stage = nullptr;                    // pinned host staging of pic_read_moments
    size_t h_stage_bytes = 0;
    std::vector<Proc> proc[2];
    float *d_nu[2] = {nullptr, nullptr};
    unsigned long long *R_last = nullptr;
    bool loaded[2] = {false, false};
    bool need_init = true;
    long long host_step = 0;
    // per species: sort interval and launch shape of the step kernel, fixed
    // (descriptor, defaults) or chosen by the autotuner
    bool autotune = false, tuned = false;
    int sort_k[2] = {16, 16};
    long long since_sort[2] = {0, 0};
    int step_threads[2] = {1024, 1024};
    int step_stages[2] = {0, 0};                // particle tiles in flight (0 = direct loads)
    float tune_shape_ms[2][6] = {};             // autotuner measurements, reported by pic_read_tuning
    float tune_sort_ms[2] = {}, tune_slope_ms[2] = {};
    // CUDA graphs of k = 1..kGraphSteps steps (no sort), replayed by pic_step,
    // and the kernel arguments they captured (a change drops them)
    cudaGraphExec_t graph[kGraphSteps + 1] = {};
    StepConst graph_P{};
    int step_grid[2] = {0, 0};
    unsigned step_smem[2] = {0, 0};
    int step_grid_threads[2] = {0, 0}, step_grid_stages[2] = {-1, -1};   // shape the cached grid was computed for
    unsigned field_smem = 0;
    // profiling: per kernel class, launch counts and event pairs
    static constexpr int kClasses = 4;
    bool prof = false;
    long long launches[kClasses] = {0, 0, 0, 0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    std::vector<std::pair<int, size_t>> ev_used;   // (class, pool index)

    void *dalloc(size_t bytes)
    {
        void *p = nullptr;
        if (d.alloc) p = d.alloc(bytes, d.alloc_ctx);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (p) allocs.push_back({p, bytes});
        return p;
    }
    void dfree(void *p)
    {
        for (size_t i = 0; i < allocs.size(); ++i)
            if (allocs[i].first == p) {
                if (d.free) d.free(p, allocs[i].second, d.alloc_ctx);
                else cudaFree(p);
                allocs.erase(allocs.begin() + i);
                return;
            }
    }
};

namespace {

enum { KC_STEP = 0, KC_FIELD = 1, KC_SORT = 2, KC_INIT = 3 };
const char *kClassName[4] = {"particle_step", "field_solve", "sort", "init"};

// Bracket one launch (or launch group) of class k with events when profiling.
struct Timed {
    pic_case *c;
    int k;
    size_t idx = (size_t)-1;
    Timed(pic_case *c_, int k_, int n_launches) : c(c_), k(k_)
    {
        c->launches[k] += n_launches;
        if (!c->prof) return;
        idx = c->ev_used.size();
        if (idx >= c->ev_pool.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            c->ev_pool.push_back({a, b});
        }
        c->ev_used.push_back({k, idx});
        cudaEventRecord(c->ev_pool[idx].first, c->stream);
    }
    ~Timed()
    {
        if (idx != (size_t)-1) cudaEventRecord(c->ev_pool[idx].second, c->stream);
    }
};

double grid_energy(int i) { return kEmin * std::exp((double)i * std::log(kEmax / kEmin) / (kNGrid - 1)); }

// LXCat-style linear interpolation of a raw table, held constant beyond its ends
double sample_table(const double *e, const double *s, int n, double eps)
{
    if (eps <= e[0]) return s[0];
    if (eps >= e[n - 1]) return s[n - 1];
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (e[mid] < eps) lo = mid; else hi = mid;
    }
    return s[lo] + (eps - e[lo]) / (e[hi] - e[lo]) * (s[hi] - s[lo]);
}

double reduced_mass(const pic_case *c, int sp)
{
    const double m = c->d.mass_kg[sp];
    return sp == 0 ? m : m * c->d.gas_mass_kg / (m + c->d.gas_mass_kg);
}

// Species constants of the step (FP64 on the host, rounded to FP32 once).
void fill_species(pic_case *c, int sp)
{
    SpConst &S = c->P.sp[sp];
    SpPush &H = c->P.push.sp[sp];
    const pic_case_desc &d = c->d;
    const double q = d.charge_C[sp], m = d.mass_kg[sp], dt = d.dt_s, M = d.gas_mass_kg;
    const double ce = q * dt / (2.0 * m);
    double t[3], tt = 0;
    for (int k = 0; k < 3; ++k) { t[k] = ce * d.B_T[k]; tt += t[k] * t[k]; }
    H.c_e = (float)ce;
    for (int k = 0; k < 3; ++k) { H.tB[k] = (float)t[k]; H.sB[k] = (float)(2.0 * t[k] / (1.0 + tt)); }
    H.rot = (H.tB[0] == 0.0f && H.tB[1] == 0.0f && H.tB[2] == 0.0f) ? 0
            : (H.tB[0] == 0.0f && H.tB[2] == 0.0f)                  ? 1
                                                                    : 2;
    H.cEy = (float)(ce * d.E_ext_V_per_m[1]);
    H.cEz = (float)(ce * d.E_ext_V_per_m[2]);
    S.m_over_2e = (float)(m / (2.0 * kElem));
    S.v_of_sqrt_eps = (float)std::sqrt(2.0 * kElem / m);
    S.recoil = M > 0 ? (float)(2.0 * m / M) : 0.0f;
    S.vt_gas = M > 0 ? (float)std::sqrt(kBoltz * d.gas_temp_k / M) : 0.0f;
    S.mfrac = (float)(m / (m + M));
    S.Mfrac = (float)(M / (m + M));
    S.mu_over_2e = (float)(reduced_mass(c, sp) / (2.0 * kElem));
    S.vt_newion = d.n_species > 1 ? (float)std::sqrt(kBoltz * d.gas_temp_k / d.mass_kg[1]) : 0.0f;
    S.q = q; S.m = m; S.w = d.weight_per_m2[sp];
    S.renew_vt = (float)std::sqrt(d.renew_temp_ev[sp] * kElem / m);
    for (int k = 0; k < 3; ++k) S.renew_drift[k] = (float)d.renew_drift_m_per_s[sp][k];
    double numax = 0.0;
    S.nproc = (int)c->proc[sp].size();
    for (int k = 0; k < kMaxProc; ++k) {
        S.kind[k] = k < S.nproc ? c->proc[sp][k].kind : 0;
        S.thr[k] = k < S.nproc ? (float)c->proc[sp][k].thr : 0.0f;
    }
    if (sp == 0 && d.const_nu_e_per_s > 0) {
        S.mcc = 2;
        numax = d.const_nu_e_per_s;
        S.nproc = 1;
        S.kind[0] = PIC_ELASTIC;
    } else if (S.nproc > 0) {
        S.mcc = 1;
        for (int i = 0; i < kNGrid; ++i) {
            double tot = 0;
            for (auto &p : c->proc[sp]) tot += p.nu[i];
            numax = std::max(numax, tot);
        }
    } else {
        S.mcc = 0;
    }
    S.numax = (float)numax;
    H.lam = S.mcc != 0 ? (float)(numax * dt) : 0.0f;
}

pic_status upload_tables(pic_case *c, int sp)
{
    const auto &pr = c->proc[sp];
    if (pr.empty()) return PIC_OK;
    if (!c->d_nu[sp]) {
        c->d_nu[sp] = (float *)c->dalloc(sizeof(float) * kNGrid * kMaxProc);
        if (!c->d_nu[sp]) return fail(PIC_ENOMEM, "table allocation failed");
    }
    std::vector<float> h(kNGrid * pr.size());
    for (size_t k = 0; k < pr.size(); ++k)
        for (int i = 0; i < kNGrid; ++i) h[k * kNGrid + i] = (float)pr[k].nu[i];
    CU(cudaMemcpyAsync(c->d_nu[sp], h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->P.nu_tab[sp] = c->d_nu[sp];
    return PIC_OK;
}

// Launch with programmatic stream serialization: the kernel may begin while
// the stream's previous kernel finishes (it orders itself with
// griddepcontrol; see k_particle_step and k_field).
template <typename... KArgs, typename... Args>
cudaError_t launch_programmatic(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Dynamic shared memory a step kernel may use: the device's opt-in maximum
// per block less a margin for the kernels' static shared memory (at most
// StepShared + one StepConst).  The cap is a property of the kernel, shared
// by every case: each instantiation sets it once.
constexpr int kStaticSmemMargin = 4096;
int step_smem_limit(int device)
{
    static std::once_flag once;
    static int lim = 0;
    std::call_once(once, [&] {
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) optin = 0;
        lim = std::max(0, optin - kStaticSmemMargin);
    });
    return lim;
}

// One flag per kernel instantiation (the caller is itself a template).
template <typename K>
cudaError_t allow_max_step_smem(K k, std::once_flag &once, cudaError_t &err, int device)
{
    std::call_once(once, [&] {
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, step_smem_limit(device));
    });
    return err;
}

// Tile buffers that fit next to the tables: `want`, fewer if shared memory is short.
int fit_stages(int n_cells, int nproc, int threads, int want, int narr, int qcap, unsigned apcap, int ccap,
               int limit)
{
    int st = std::max(0, std::min(want, kMaxStages));
    while (st > 0 && StepSmem(n_cells, nproc, threads, st, narr, qcap, apcap, ccap).total > (unsigned)limit) --st;
    return st;
}

// The variants (direct loads, bulk-copy tiles, axial renewal with direct
// loads) are separate kernels, so that each carries only its own state.
template <int SP, bool PER, int MCC, bool STAGED, bool AXIAL = false>
cudaError_t launch_step_k(pic_case *c, int stages)
{
    auto k = k_particle_step<SP, PER, MCC, STAGED, AXIAL>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    cudaError_t e = allow_max_step_smem(k, once, attr_err, c->device);
    if (e != cudaSuccess) return e;
    const int nproc = MCC == 1 ? c->P.sp[SP].nproc : 0;
    constexpr int narr = step_arrays(SP, PER, MCC);
    constexpr int qcap = draw_queue_cap(MCC, STAGED ? 4 : kDirectChunk);
    // each warp's draw queue grows the CTA's shared memory: a CTA that does
    // not fit next to the tables of the largest grids is halved
    const unsigned apcap = append_cap(c->P);
    constexpr int ccap = child_queue_cap(SP, MCC);
    int threads = c->step_threads[SP];
    while (threads > 64 && StepSmem(c->d.n_cells, nproc, threads, stages, narr, qcap, apcap, ccap).total >
                               (unsigned)step_smem_limit(c->device))
        threads /= 2;
    const unsigned smem = StepSmem(c->d.n_cells, nproc, threads, stages, narr, qcap, apcap, ccap).total;
    if (c->step_smem[SP] != smem || c->step_grid[SP] == 0 || c->step_grid_threads[SP] != threads ||
        c->step_grid_stages[SP] != stages) {
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
        if (e != cudaSuccess) return e;
        c->step_grid[SP] = std::max(1, occ) * c->num_sms;
        c->step_smem[SP] = smem;
        c->step_grid_threads[SP] = threads;
        c->step_grid_stages[SP] = stages;
    }
    c->P.sp[SP].stages = stages;
    Timed t(c, KC_STEP, 1);
    e = launch_programmatic(k, dim3(c->step_grid[SP]), dim3(threads), smem, c->stream, c->P);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int SP, bool PER, int MCC>
cudaError_t launch_step_t(pic_case *c)
{
    if (c->P.axial_len > 0.0f) return launch_step_k<SP, PER, MCC, false, true>(c, 0);
    const int nproc = MCC == 1 ? c->P.sp[SP].nproc : 0;
    const int stages = fit_stages(c->d.n_cells, nproc, c->step_threads[SP], c->step_stages[SP],
                                  step_arrays(SP, PER, MCC), draw_queue_cap(MCC, 4), append_cap(c->P),
                                  child_queue_cap(SP, MCC), step_smem_limit(c->device));
    return stages > 0 ? launch_step_k<SP, PER, MCC, true>(c, stages) : launch_step_k<SP, PER, MCC, false>(c, 0);
}

template <int SP>
cudaError_t launch_step_sp(pic_case *c)
{
    const int mcc = c->P.sp[SP].mcc;
    if (c->d.periodic) {
        if (mcc == 0) return launch_step_t<SP, true, 0>(c);
        if (mcc == 1) return launch_step_t<SP, true, 1>(c);
        return launch_step_t<SP, true, 2>(c);
    }
    if (mcc == 0) return launch_step_t<SP, false, 0>(c);
    if (mcc == 1) return launch_step_t<SP, false, 1>(c);
    return launch_step_t<SP, false, 2>(c);
}

cudaError_t launch_field(pic_case *c, int mode)
{
    Timed t(c, mode == 0 ? KC_INIT : KC_FIELD, 1);
    cudaError_t e = launch_programmatic(k_field, dim3(kFieldCluster), dim3(field_threads_for(c->d.n_cells, kFieldCluster)),
                                        c->field_smem, c->stream, c->P, mode);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// The scatter's shared memory passes the default 48 KB above about 600
// cells: each scatter kernel is allowed the size of the largest grid once.
template <typename K>
cudaError_t allow_scatter_smem(K k, std::once_flag &once, cudaError_t &err)
{
    std::call_once(once, [&] {
        err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem(4096));
    });
    return err;
}
template <bool CLOCK>
cudaError_t allow_cells_scatter()
{
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    return allow_scatter_smem(k_cells_scatter<CLOCK>, once, err);
}
cudaError_t allow_batch_scatter()
{
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    return allow_scatter_smem(k_batch_cells_scatter, once, err);
}

cudaError_t launch_sort(pic_case *c, int sp)
{
    const int N = c->d.n_cells;
    const long long cap = (long long)c->P.cap[sp];
    Timed t(c, KC_SORT, 4);
    SortHalves H{{c->P.buf[sp][0], c->P.buf[sp][1]}};
    const int32_t *cur = &c->P.ctrl->cur[sp];
    const unsigned long long *n = &c->P.ctrl->n_active[sp];
    const int gc = (int)std::min<long long>(c->num_sms * 4, std::max<long long>(1, cap / 1024));
    k_cells_count<true><<<gc, 512, N * sizeof(unsigned), c->stream>>>(H, cur, n, 0, N, c->P.sort_count);
    k_cells_scan<<<1, 1024, N * sizeof(double), c->stream>>>(c->P.sort_count, N, c->P.sort_cursor);
    const int gs = (int)std::min<long long>(c->num_sms, std::max<long long>(1, (cap + 2047) / 2048));   // one wave
    cudaError_t e = allow_cells_scatter<true>();
    if (e != cudaSuccess) return e;
    k_cells_scatter<true><<<gs, kScatterThreads, scatter_smem(N), c->stream>>>(H, cur, n, 0, N, c->P.sort_cursor);
    k_sort_finish<<<4, 256, 0, c->stream>>>(c->P, sp, c->P.sort_cursor + N);
    return cudaGetLastError();
}

pic_status device_error(pic_case *c)
{
    Ctrl h;
    CU(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (h.err & kErrLoad) return fail(PIC_EINVAL, "loaded particle outside the grid (cell or offset)");
    if (h.err & kErrCapacity) return fail(PIC_ECAPACITY, "particle capacity exceeded during a step");
    if (h.err & kErrNumeric) return fail(PIC_ENUMERIC, "non-finite potential or field");
    if (h.err & kErrTimeout) return fail(PIC_ETIMEOUT, "a bounded device wait gave up");
    return PIC_OK;
}

pic_status alloc_species(pic_case *c, int sp, long long need)
{
    long long cap = c->d.capacity[sp] > 0 ? c->d.capacity[sp] : std::max<long long>(2 * need, 65536);
    if (need > cap) return fail(PIC_ECAPACITY, "load exceeds the species capacity");
    if ((long long)c->P.cap[sp] >= cap && c->P.buf[sp][0].cell) return PIC_OK;
    for (int h = 0; h < 2; ++h) {
        SpeciesBufs &B = c->P.buf[sp][h];
        c->dfree(B.cell); c->dfree(B.off); c->dfree(B.vx); c->dfree(B.vy); c->dfree(B.vz); c->dfree(B.id);
        c->dfree(B.z);
        B.z = nullptr;
    }
    const long long slots = (cap + 3) / 4 * 4 + 4;   // float4 access never leaves the buffer
    for (int h = 0; h < 2; ++h) {
        SpeciesBufs &B = c->P.buf[sp][h];
        B.cell = (int32_t *)c->dalloc(slots * 4); B.off = (float *)c->dalloc(slots * 4);
        B.vx = (float *)c->dalloc(slots * 4); B.vy = (float *)c->dalloc(slots * 4);
        B.vz = (float *)c->dalloc(slots * 4); B.id = (uint32_t *)c->dalloc(slots * 4);
        if (!B.cell || !B.off || !B.vx || !B.vy || !B.vz || !B.id) return fail(PIC_ENOMEM, "particle allocation failed");
        if (c->d.axial_length_m > 0) {                              // axial excursion for the renewal
            B.z = (float *)c->dalloc(slots * 4);
            if (!B.z) return fail(PIC_ENOMEM, "particle allocation failed");
            CU(cudaMemsetAsync(B.z, 0, slots * 4, c->stream));
        }
    }
    c->P.cap[sp] = (unsigned long long)cap;
    return PIC_OK;
}

pic_status initialise(pic_case *c)
{
    for (int s = 0; s < c->d.n_species; ++s) fill_species(c, s);
    for (int s = 0; s < c->d.n_species; ++s)
        CU(cudaMemsetAsync(c->P.R[s], 0, sizeof(unsigned long long) * kDepositCopies * c->P.r_stride, c->stream));
    Timed t(c, KC_INIT, c->d.n_species * (c->d.rewind ? 2 : 1));
    for (int s = 0; s < c->d.n_species; ++s) {
        k_deposit_species<<<c->num_sms * 4, 256, 12 * (size_t)c->d.n_cells, c->stream>>>(c->P, s);
        CU(cudaGetLastError());
    }
    CU(launch_field(c, 0));
    if (c->d.rewind) {
        k_rewind<0><<<c->num_sms * 4, 256, 0, c->stream>>>(c->P);
        if (c->d.n_species > 1) k_rewind<1><<<c->num_sms * 4, 256, 0, c->stream>>>(c->P);
        CU(cudaGetLastError());
    }
    c->need_init = false;
    return PIC_OK;
}

__global__ void k_reset_counters(Ctrl *ctrl)
{
    ctrl->absorbed[0][0] = ctrl->absorbed[0][1] = ctrl->absorbed[1][0] = ctrl->absorbed[1][1] = 0;
    ctrl->see = ctrl->iz = 0;
    ctrl->renewed[0] = ctrl->renewed[1] = 0;
    ctrl->cand[0] = ctrl->cand[1] = 0;
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < kMaxProc; ++k) ctrl->coll[s][k] = 0;
    ctrl->fe_n = 0;
    ctrl->n_steps_acc = ctrl->n_diag_acc = 0;
}

// SI positions and velocities -> the internal layout.  xi = x / dx in FP64;
// cell = floor(xi), offset = xi - cell rounded to FP32 (an offset that rounds
// up to 1 moves to the next cell's 0, or stays below 1 in the last cell).  A
// position outside [0, L) or not finite is stored as cell n_cells, which the
// validation at the first step reports (PIC_EINVAL).
__global__ void k_load_si(SpeciesBufs B, long long n, int N, double inv_dx, double len, const double *__restrict__ x,
                          const double *__restrict__ v, const uint32_t *__restrict__ id)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double xm = x[k];
        int c = N;
        float o = 0.0f;
        if (xm >= 0.0 && xm < len) {
            const double xi = xm * inv_dx;
            const double fl = floor(xi);
            c = (int)fl;
            o = (float)(xi - fl);
            if (o >= 1.0f) { o = 0.0f; c += 1; }
            if (c >= N) { c = N - 1; o = 0.99999994f; }
        }
        B.cell[k] = c;
        B.off[k] = o;
        B.vx[k] = (float)v[3 * k];
        B.vy[k] = (float)v[3 * k + 1];
        B.vz[k] = (float)v[3 * k + 2];
        B.id[k] = id ? id[k] : (uint32_t)k;
    }
}

// Plain cell indices: a load restarts every species, and their collision
// clocks are drawn afresh at the first step.
__global__ void k_strip_clock(int32_t *cell, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int w = cell[i];
        if (w >= 0) cell[i] = w & kCellMask;
    }
}

// Ids 0..n-1 of a load that gives none.
__global__ void k_iota_u32(uint32_t *id, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        id[i] = (uint32_t)i;
}

pic_status reset_moments(pic_case *c)
{
    const size_t nn = (size_t)c->n_nodes;
    CU(cudaMemsetAsync(c->P.Rsum, 0, sizeof(unsigned long long) * 2 * nn, c->stream));
    CU(cudaMemsetAsync(c->P.Rdiag, 0, sizeof(unsigned long long) * 2 * nn, c->stream));
    CU(cudaMemsetAsync(c->P.en_sum, 0, sizeof(double) * 2 * nn, c->stream));
    CU(cudaMemsetAsync(c->P.phi_sum, 0, sizeof(double) * nn, c->stream));
    CU(cudaMemsetAsync(c->P.ke_sum, 0, sizeof(double) * 2, c->stream));
    CU(cudaMemsetAsync(c->P.pw_sum, 0, sizeof(double) * 2, c->stream));
    CU(cudaMemsetAsync(c->P.eepf, 0, sizeof(unsigned long long) * kEepfBins, c->stream));
    CU(cudaMemsetAsync(c->P.ifedf, 0, sizeof(unsigned long long) * 2 * kIfedfBins, c->stream));
    k_reset_counters<<<1, 1, 0, c->stream>>>(c->P.ctrl);
    CU(cudaGetLastError());
    return PIC_OK;
}

} // namespace

namespace {

void drop_graph(pic_case *c)
{
    for (auto &g : c->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// The kernels of one step (both species, field solve), launched on the case stream.
cudaError_t launch_one_step(pic_case *c)
{
    cudaError_t e = launch_step_sp<0>(c);
    if (e == cudaSuccess && c->d.n_species > 1) e = launch_step_sp<1>(c);
    if (e == cudaSuccess) e = launch_field(c, 1);
    return e;
}


// ---------------------------------------------------------------------------
// Autotuner, per species, of the sort interval K and of the step kernel's
// launch shape.
//  1. Sort interval: the tuner times one sort and the kTuneSteps steps after
//     it per species (default shape); choose_sort_interval (sort_interval.h)
//     picks K in [4, 1024] from them.
//  2. Launch shape: CTA size (256, 512 or 1024 threads) and particle tiles
//     in flight through shared memory (0 = each thread loads its own chunk;
//     1 or 2 = bulk-copy pipeline).  Fewer, larger CTAs flush fewer copies
//     of the shared deposit histogram, which matters once the particles have
//     lost their cell order.  Continuing from the state step 1 left
//     (the particle order of the middle of a sort period), the candidates
//     take turns, one step each, for kShapeRounds rounds; each species keeps
//     the candidate whose fastest round is the fastest (a candidate's first
//     launch can carry the loading of its kernel, or another one-off delay,
//     which a mean over the rounds would count against it).
// Particle results do not depend on any of these choices (the deposit is
// exact integer arithmetic); only FP32/FP64 moment sums may change in their
// last bits with the launch shape.  Results are kept per case shape for the
// process, and in the file named by PIC1D3V_TUNE_CACHE if that variable is set.
// ---------------------------------------------------------------------------
constexpr int kTuneSteps = 32;
constexpr int kShapeRounds = 3;
constexpr int kShapes = 6;
constexpr int kShapeThreads[kShapes] = {1024, 512, 256, 1024, 512, 512};
constexpr int kShapeStages[kShapes] = {0, 0, 0, 1, 1, 2};
constexpr int kTuneTotalSteps = kTuneSteps + kShapeRounds * kShapes;
constexpr int kMaxSortInterval = 1024;

struct TuneResult {
    int K[2], threads[2], stages[2];
};

std::mutex g_tune_mutex;
std::map<std::string, TuneResult> g_tune_cache;
bool g_tune_file_read = false;

std::string tune_key(const pic_case *c)
{
    char buf[160];
    int lg[2] = {0, 0};
    for (int s = 0; s < c->d.n_species; ++s)
        while ((1ull << (lg[s] + 1)) <= c->P.cap[s]) ++lg[s];
    std::snprintf(buf, sizeof buf, "p%d_c%d_n2^%d_2^%d_m%d%d", c->d.periodic, c->d.n_cells, lg[0], lg[1],
                  c->P.sp[0].mcc, c->d.n_species > 1 ? c->P.sp[1].mcc : 0);
    return buf;
}

bool tune_lookup(const std::string &key, TuneResult *out)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const char *path = std::getenv("PIC1D3V_TUNE_CACHE");
    if (path && !g_tune_file_read) {
        g_tune_file_read = true;
        if (FILE *f = std::fopen(path, "r")) {
            char line[256], k[160];
            TuneResult r;
            while (std::fgets(line, sizeof line, f))
                if (std::sscanf(line, "%159s %d %d %d %d %d %d", k, &r.K[0], &r.K[1], &r.threads[0], &r.stages[0],
                                &r.threads[1], &r.stages[1]) == 7) {
                    bool ok = true;
                    for (int s = 0; s < 2; ++s)
                        ok = ok && r.K[s] >= 1 && r.K[s] <= kMaxSortInterval &&
                             (r.threads[s] == 256 || r.threads[s] == 512 || r.threads[s] == 1024) &&
                             r.stages[s] >= 0 && r.stages[s] <= kMaxStages;
                    if (ok) g_tune_cache[k] = r;                     // malformed lines are ignored
                }
            std::fclose(f);
        }
    }
    auto it = g_tune_cache.find(key);
    if (it == g_tune_cache.end()) return false;
    *out = it->second;
    return true;
}

void tune_store(const std::string &key, const TuneResult &r)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = r;
    if (const char *path = std::getenv("PIC1D3V_TUNE_CACHE"))
        if (FILE *f = std::fopen(path, "a")) {
            std::fprintf(f, "%s %d %d %d %d %d %d\n", key.c_str(), r.K[0], r.K[1], r.threads[0], r.stages[0],
                         r.threads[1], r.stages[1]);
            std::fclose(f);
        }
}

void apply_tuning(pic_case *c, const TuneResult &r)
{
    for (int s = 0; s < 2; ++s) {
        c->sort_k[s] = r.K[s];
        c->step_threads[s] = r.threads[s];
        c->step_stages[s] = r.stages[s];
    }
    c->tuned = true;
    drop_graph(c);                                   // captured launches carry the old shape
}

// One step with events around each species' step kernel (ev[2 * s], ev[2 * s + 1]).
cudaError_t launch_one_step_timed(pic_case *c, const cudaEvent_t *ev)
{
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < c->d.n_species && e == cudaSuccess; ++s) {
        e = cudaEventRecord(ev[2 * s], c->stream);
        if (e == cudaSuccess) e = s == 0 ? launch_step_sp<0>(c) : launch_step_sp<1>(c);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * s + 1], c->stream);
    }
    if (e == cudaSuccess) e = launch_field(c, 1);
    return e;
}

pic_status autotune(pic_case *c, int64_t *left)
{
    const std::string key = tune_key(c);
    TuneResult r{};
    if (tune_lookup(key, &r)) {
        apply_tuning(c, r);
        return PIC_OK;
    }
    const int ns = c->d.n_species;
    drop_graph(c);
    struct Events {                                  // destroyed on every return path
        std::vector<cudaEvent_t> v;
        ~Events() { for (auto e : v) cudaEventDestroy(e); }
    } ev;
    ev.v.resize(4 + 4 * kTuneSteps + 4 * kShapeRounds * kShapes, nullptr);
    for (auto &e : ev.v) CU(cudaEventCreate(&e));
    cudaEvent_t *sev = ev.v.data();                  // sorts
    cudaEvent_t *tev = sev + 4;                      // steps after the sort
    cudaEvent_t *shev = tev + 4 * kTuneSteps;        // shape rounds
    // 1. sort interval with the default shape
    for (int s = 0; s < 2; ++s) { c->step_threads[s] = kShapeThreads[0]; c->step_stages[s] = kShapeStages[0]; }
    for (int s = 0; s < ns; ++s) {
        CU(cudaEventRecord(sev[2 * s], c->stream));
        CU(launch_sort(c, s));
        CU(cudaEventRecord(sev[2 * s + 1], c->stream));
    }
    int64_t alive0[2] = {0, 0}, alive1[2] = {0, 0};   // live particles around the timed steps
    {
        Ctrl h;
        CU(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        for (int s = 0; s < ns; ++s) alive0[s] = (int64_t)(h.n_total[s] - h.n_dead[s]);
    }
    for (int k = 0; k < kTuneSteps; ++k) CU(launch_one_step_timed(c, &tev[4 * k]));
    {
        Ctrl h;
        CU(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        for (int s = 0; s < ns; ++s) alive1[s] = (int64_t)(h.n_total[s] - h.n_dead[s]);
    }
    // 2. launch shapes, interleaved
    for (int rnd = 0; rnd < kShapeRounds; ++rnd)
        for (int k = 0; k < kShapes; ++k) {
            for (int s = 0; s < 2; ++s) { c->step_threads[s] = kShapeThreads[k]; c->step_stages[s] = kShapeStages[k]; }
            CU(launch_one_step_timed(c, &shev[4 * (rnd * kShapes + k)]));
        }
    CU(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < 2; ++s) {
        r.K[s] = kMaxSortInterval;
        r.threads[s] = kShapeThreads[0];
        r.stages[s] = kShapeStages[0];
        for (int k = 0; k < kShapes; ++k) c->tune_shape_ms[s][k] = 0.f;
        if (s >= ns) continue;
        float ts = 0.f;
        CU(cudaEventElapsedTime(&ts, sev[2 * s], sev[2 * s + 1]));
        double ty[kTuneSteps];                        // step k + 1 after the sort
        for (int k = 0; k < kTuneSteps; ++k) {
            float t = 0.f;
            CU(cudaEventElapsedTime(&t, tev[4 * k + 2 * s], tev[4 * k + 2 * s + 1]));
            ty[k] = t;
        }
        normalise_to_count(ty, kTuneSteps, (double)alive0[s], (double)alive1[s]);
        const SortIntervalFit fit = choose_sort_interval(ty, kTuneSteps, ts, 4, kMaxSortInterval);
        r.K[s] = fit.K;
        r.K[s] = std::max(4, std::min(kMaxSortInterval, r.K[s]));
        c->tune_sort_ms[s] = ts;
        c->tune_slope_ms[s] = (float)fit.slope;
        float shape_ms[kShapes];
        for (int k = 0; k < kShapes; ++k) shape_ms[k] = 3.0e38f;
        for (int rnd = 0; rnd < kShapeRounds; ++rnd)
            for (int k = 0; k < kShapes; ++k) {
                float t = 0.f;
                CU(cudaEventElapsedTime(&t, shev[4 * (rnd * kShapes + k) + 2 * s], shev[4 * (rnd * kShapes + k) + 2 * s + 1]));
                shape_ms[k] = std::min(shape_ms[k], t);
            }
        int best = 0;
        for (int k = 1; k < kShapes; ++k)
            if (shape_ms[k] < shape_ms[best]) best = k;
        r.threads[s] = kShapeThreads[best];
        r.stages[s] = kShapeStages[best];
        for (int k = 0; k < kShapes; ++k) c->tune_shape_ms[s][k] = shape_ms[k];
    }
    apply_tuning(c, r);
    c->host_step += kTuneTotalSteps;
    c->since_sort[0] = c->since_sort[1] = kTuneTotalSteps;
    *left -= kTuneTotalSteps;
    tune_store(key, r);
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of 1..kGraphSteps steps.  Kernel arguments are captured by
// value, so the graphs are dropped whenever they change (load, tables, launch
// shape) and rebuilt together at the next replay, so that their set-up falls
// in one call rather than in the middle of a caller's timed run.
// ---------------------------------------------------------------------------
pic_status build_graph(pic_case *c, int steps)
{
    if (std::memcmp(&c->graph_P, &c->P, sizeof(StepConst)) != 0) drop_graph(c);
    if (c->graph[steps]) return PIC_OK;
    c->graph_P = c->P;
    long long saved[pic_case::kClasses];
    for (int k = 0; k < pic_case::kClasses; ++k) saved[k] = c->launches[k];
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < steps && e == cudaSuccess; ++i) e = launch_one_step(c);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    for (int k = 0; k < pic_case::kClasses; ++k) c->launches[k] = saved[k];
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(PIC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&c->graph[steps], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph[steps] = nullptr;
        return fail(PIC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return PIC_OK;
}

// Every graph length a run of steps can need (at most the shortest sort interval).
pic_status build_graphs(pic_case *c)
{
    int G = kGraphSteps;
    for (int s = 0; s < c->d.n_species; ++s) G = std::min(G, c->sort_k[s]);
    for (int k = 1; k <= G; ++k) {
        pic_status st = build_graph(c, k);
        if (st != PIC_OK) return st;
    }
    return PIC_OK;
}

// Common start of a load: buffers allocated, other species moved to half 0.
pic_status load_begin(pic_case *c, int sp, int64_t n, Ctrl *h)
{
    CU(cudaStreamSynchronize(c->stream));
    pic_status st = alloc_species(c, sp, n);
    if (st != PIC_OK) return st;
    for (int s = 0; s < c->d.n_species; ++s)
        if (!c->P.buf[s][0].cell) {
            st = alloc_species(c, s, 0);
            if (st != PIC_OK) return st;
        }
    CU(cudaMemcpy(h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    // a load restarts the case: particles of the other species move back to
    // half 0 and lose their collision clocks (drawn afresh at the first step)
    for (int s = 0; s < c->d.n_species; ++s) {
        if (s == sp || !c->loaded[s] || h->n_total[s] == 0) continue;
        if (h->cur[s] == 0) {
            k_strip_clock<<<c->num_sms * 4, 256, 0, c->stream>>>(c->P.buf[s][0].cell, (long long)h->n_total[s]);
            CU(cudaGetLastError());
            continue;
        }
        const SpeciesBufs &A = c->P.buf[s][1], &D = c->P.buf[s][0];
        const size_t b = (size_t)h->n_total[s] * 4;
        CU(cudaMemcpyAsync(D.cell, A.cell, b, cudaMemcpyDeviceToDevice, c->stream));
        CU(cudaMemcpyAsync(D.off, A.off, b, cudaMemcpyDeviceToDevice, c->stream));
        CU(cudaMemcpyAsync(D.vx, A.vx, b, cudaMemcpyDeviceToDevice, c->stream));
        CU(cudaMemcpyAsync(D.vy, A.vy, b, cudaMemcpyDeviceToDevice, c->stream));
        CU(cudaMemcpyAsync(D.vz, A.vz, b, cudaMemcpyDeviceToDevice, c->stream));
        CU(cudaMemcpyAsync(D.id, A.id, b, cudaMemcpyDeviceToDevice, c->stream));
        if (A.z) CU(cudaMemcpyAsync(D.z, A.z, b, cudaMemcpyDeviceToDevice, c->stream));
        k_strip_clock<<<c->num_sms * 4, 256, 0, c->stream>>>(D.cell, (long long)h->n_total[s]);
        CU(cudaGetLastError());
    }
    return PIC_OK;
}

// Common end of a load: counts, drive phases, moments reset, state restarts at step 0.
pic_status load_finish(pic_case *c, int sp, int64_t n, const Ctrl &h)
{
    Ctrl z;
    std::memset(&z, 0, sizeof(z));
    for (int k = 0; k < c->d.n_harm; ++k) {                 // phases at the first step's field solve (t = dt)
        const double ph = 2.0 * M_PI * c->d.harm_freq_hz[k] * c->d.dt_s + c->d.harm_phase_rad[k];
        z.drive_c[k] = std::cos(ph);
        z.drive_s[k] = std::sin(ph);
    }
    for (int s = 0; s < 2; ++s) {
        const unsigned long long cnt = s == sp ? (unsigned long long)n : (c->loaded[s] ? h.n_total[s] : 0ull);
        z.n_total[s] = z.n_active[s] = cnt;
    }
    CU(cudaMemcpyAsync(c->P.ctrl, &z, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream));
    if (c->P.buf[sp][0].z && n > 0)                                   // loaded particles start at z = 0
        CU(cudaMemsetAsync(c->P.buf[sp][0].z, 0, sizeof(float) * (size_t)n, c->stream));
    pic_status st = reset_moments(c);
    if (st != PIC_OK) return st;
    CU(cudaStreamSynchronize(c->stream));
    c->loaded[sp] = true;
    c->need_init = true;
    c->host_step = 0;
    c->since_sort[0] = c->since_sort[1] = 0;
    return PIC_OK;                                   // graphs are dropped at replay if the load moved a buffer
}

} // namespace

// Message for pic_last_error() from the other translation units of the library.
namespace pic {
void set_last_error(const std::string &msg) { g_err = msg; }
}

// ===========================================================================
extern "C" {

const char *pic_status_str(pic_status s)
{
    switch (s) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument";
    case PIC_ENOMEM: return "out of device memory";
    case PIC_ECUDA: return "CUDA error";
    case PIC_ECAPACITY: return "particle capacity exceeded";
    case PIC_ENUMERIC: return "non-finite field";
    case PIC_ETIMEOUT: return "device wait timed out";
    case PIC_ESTATE: return "invalid state";
    }
    return "unknown status";
}

const char *pic_last_error(void) { return g_err.c_str(); }

pic_status pic_create_case(const pic_case_desc *desc, pic_case **out)
{
    if (!desc || !out) return fail(PIC_EINVAL, "null descriptor or output");
    *out = nullptr;
    if (desc->struct_size != sizeof(pic_case_desc) || desc->version != PIC_DESC_VERSION)
        return fail(PIC_EINVAL, "descriptor size/version mismatch");
    if (desc->n_cells < 2 || desc->n_cells > 4096) return fail(PIC_EINVAL, "n_cells must be in [2, 4096]");
    if (desc->n_species < 1 || desc->n_species > 2) return fail(PIC_EINVAL, "n_species must be 1 or 2");
    if (!(desc->dt_s > 0) || !(desc->length_m > 0)) return fail(PIC_EINVAL, "dt and length must be positive");
    if (desc->n_harm < 0 || desc->n_harm > 4) return fail(PIC_EINVAL, "n_harm must be in [0, 4]");
    if (desc->circuit < 0 || desc->circuit > 2) return fail(PIC_EINVAL, "circuit must be 0, 1 or 2");
    if (desc->circuit >= 1 && desc->periodic) return fail(PIC_EINVAL, "an electrode circuit needs electrodes");
    if (desc->circuit == 1 && (!(desc->blocking_cap_F_per_m2 >= 0) || !std::isfinite(desc->blocking_cap_F_per_m2)))
        return fail(PIC_EINVAL, "a series capacitor needs a finite capacitance >= 0");
    if (!(desc->ifedf_emax_ev >= 0)) return fail(PIC_EINVAL, "ifedf_emax_ev must be >= 0");
    if (!(desc->axial_length_m >= 0) || !std::isfinite(desc->axial_length_m))
        return fail(PIC_EINVAL, "axial_length_m must be finite and >= 0");
    for (int s = 0; s < desc->n_species; ++s)
        if (!(desc->renew_temp_ev[s] >= 0)) return fail(PIC_EINVAL, "renew_temp_ev must be >= 0");
    for (int s = 0; s < desc->n_species; ++s)
        if (!(desc->mass_kg[s] > 0)) return fail(PIC_EINVAL, "species mass must be positive");
    {   // every floating-point quantity of the descriptor must be finite
        std::vector<double> v = {desc->length_m, desc->dt_s, desc->gas_density_m3, desc->gas_temp_k, desc->gas_mass_kg,
                                 desc->see_gamma, desc->see_temp_ev, desc->background_charge_C_per_m3,
                                 desc->const_nu_e_per_s, desc->blocking_cap_F_per_m2, desc->ifedf_emax_ev,
                                 desc->axial_length_m};
        for (int k = 0; k < 3; ++k) { v.push_back(desc->B_T[k]); v.push_back(desc->E_ext_V_per_m[k]); }
        for (int h = 0; h < 4; ++h) {
            v.push_back(desc->harm_freq_hz[h]); v.push_back(desc->harm_amp_v[h]); v.push_back(desc->harm_phase_rad[h]);
        }
        for (int s = 0; s < 2; ++s) {
            v.push_back(desc->charge_C[s]); v.push_back(desc->mass_kg[s]); v.push_back(desc->weight_per_m2[s]);
            v.push_back(desc->renew_temp_ev[s]);
            for (int k = 0; k < 3; ++k) v.push_back(desc->renew_drift_m_per_s[s][k]);
        }
        for (double x : v)
            if (!std::isfinite(x)) return fail(PIC_EINVAL, "a descriptor quantity is not finite");
    }
    pic_case *c = new pic_case();
    c->d = *desc;
    c->autotune = c->d.sort_interval <= 0;
    c->sort_k[0] = c->sort_k[1] = c->autotune ? 16 : c->d.sort_interval;
    if (c->d.field_history <= 0) c->d.field_history = 65536;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) { delete c; return fail(PIC_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e)); }
    if (desc->stream) c->stream = (cudaStream_t)desc->stream;
    else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c; return fail(PIC_ECUDA, "stream creation failed");
        }
        c->own_stream = true;
    }
    const int N = desc->n_cells;
    c->n_nodes = desc->periodic ? N : N + 1;
    StepConst &P = c->P;
    P.n_cells = N; P.n_nodes = c->n_nodes; P.periodic = desc->periodic; P.n_species = desc->n_species;
    const double dx = desc->length_m / N;
    P.dx = dx; P.dt = desc->dt_s; P.eps0 = kEps0;
    P.dtdx = (float)(desc->dt_s / dx);
    P.push.ex_ext = (float)desc->E_ext_V_per_m[0];
    P.push.key0 = (uint32_t)desc->seed; P.push.key1 = (uint32_t)(desc->seed >> 32);
    P.see_gamma = (float)desc->see_gamma;
    P.see_vth = (float)std::sqrt(desc->see_temp_ev * kElem / desc->mass_kg[0]);
    P.see_dtdx = (float)(desc->dt_s / dx);
    P.eepf_lo = (float)(0.45 * N); P.eepf_hi = (float)(0.55 * N);
    P.inv_dlog = (float)(1.0 / (std::log(kEmax / kEmin) / (kNGrid - 1)));
    P.diag_interval = desc->diag_interval;
    P.wait_polls = kDefaultWaitPolls;
    P.vol_interior = dx; P.vol_wall = desc->periodic ? dx : 0.5 * dx;
    P.bg_charge = desc->background_charge_C_per_m3;
    P.bg_r = P.bg_charge * dx * dx / kEps0;
    P.inv_dx = 1.0 / dx;
    P.inv_2dx = 0.5 / dx;
    P.half_dx_eps0 = 0.5 * dx / kEps0;
    P.fe_c = 0.5 * kEps0 * dx;
    P.inv_n = 1.0 / N;
    P.v_init = 0.0;
    for (int h = 0; h < desc->n_harm; ++h) {
        P.v_init += desc->harm_amp_v[h] * std::cos(desc->harm_phase_rad[h]);
        P.rot_c[h] = std::cos(2.0 * M_PI * desc->harm_freq_hz[h] * desc->dt_s);
        P.rot_s[h] = std::sin(2.0 * M_PI * desc->harm_freq_hz[h] * desc->dt_s);
    }
    if (desc->circuit == 2) P.v_init = 0.0;                  // current drive: electrode at 0 V at load
    for (int s = 0; s < 2; ++s) {
        const double qw = s < desc->n_species ? desc->charge_C[s] * desc->weight_per_m2[s] / 4294967296.0 : 0.0;
        P.cq[s] = qw * dx / kEps0;
        P.rho_wall[s] = qw / (0.5 * dx);
    }
    P.circuit = desc->circuit;
    P.c_blk = desc->circuit == 1 ? desc->blocking_cap_F_per_m2 : 0.0;
    P.no_field = desc->no_field ? 1 : 0;
    P.axial_len = (float)desc->axial_length_m;
    P.dt_f = (float)desc->dt_s;
    P.eps0_L = kEps0 / desc->length_m;
    P.inv_cap_eps0_L = 1.0 / (P.c_blk + P.eps0_L);
    for (int s = 0; s < 2; ++s) {
        P.qw[s] = s < desc->n_species ? desc->charge_C[s] * desc->weight_per_m2[s] : 0.0;
        P.r0c[s] = P.qw[s] / 4294967296.0;
    }
    P.bg_half = P.bg_charge * 0.5 * dx;
    P.ifedf_scale = desc->ifedf_emax_ev > 0 ? (float)(kIfedfBins / desc->ifedf_emax_ev) : 0.0f;
    P.n_harm = desc->n_harm;
    for (int h = 0; h < 4; ++h) { P.harm_f[h] = desc->harm_freq_hz[h]; P.harm_a[h] = desc->harm_amp_v[h]; P.harm_p[h] = desc->harm_phase_rad[h]; }
    const size_t nn = (size_t)c->n_nodes;
    P.E32p = (float2 *)c->dalloc(sizeof(float2) * ((N + 1) / 2 * 2));
    P.E = (double *)c->dalloc(sizeof(double) * nn);
    P.phi = (double *)c->dalloc(sizeof(double) * nn);
    P.r_stride = (N + 1 + 15) / 16 * 16;
    for (int s = 0; s < 2; ++s)
        P.R[s] = (unsigned long long *)c->dalloc(sizeof(unsigned long long) * kDepositCopies * P.r_stride);
    c->R_last = (unsigned long long *)c->dalloc(sizeof(unsigned long long) * 2 * nn);
    P.R_last = c->R_last;
    P.ctrl = (Ctrl *)c->dalloc(sizeof(Ctrl));
    P.Rsum = (unsigned long long *)c->dalloc(sizeof(unsigned long long) * 2 * nn);
    P.Rdiag = (unsigned long long *)c->dalloc(sizeof(unsigned long long) * 2 * nn);
    P.en_sum = (double *)c->dalloc(sizeof(double) * 2 * nn);
    P.phi_sum = (double *)c->dalloc(sizeof(double) * nn);
    P.ke_sum = (double *)c->dalloc(sizeof(double) * 2);
    P.pw_sum = (double *)c->dalloc(sizeof(double) * 2);
    P.eepf = (unsigned long long *)c->dalloc(sizeof(unsigned long long) * kEepfBins);
    P.fe_cap = c->d.field_history;
    P.fe_hist = (double *)c->dalloc(sizeof(double) * (size_t)P.fe_cap * kFieldCluster);
    P.sort_count = (unsigned *)c->dalloc(sizeof(unsigned) * N);
    P.sort_cursor = (unsigned long long *)c->dalloc(sizeof(unsigned long long) * (N + 1));
    P.ifedf = (unsigned long long *)c->dalloc(sizeof(unsigned long long) * 2 * kIfedfBins);
    if (!P.ifedf || !P.E32p || !P.E || !P.phi || !P.R[0] || !P.R[1] || !c->R_last || !P.ctrl || !P.Rsum || !P.Rdiag ||
        !P.en_sum || !P.phi_sum || !P.ke_sum || !P.pw_sum || !P.eepf || !P.fe_hist || !P.sort_count || !P.sort_cursor) {
        pic_destroy(c);
        return fail(PIC_ENOMEM, "device allocation failed");
    }
    cudaMemsetAsync(P.E32p, 0, sizeof(float2) * ((N + 1) / 2 * 2), c->stream);
    cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), c->stream);
    cudaMemsetAsync(P.sort_count, 0, sizeof(unsigned) * N, c->stream);
    cudaMemsetAsync(c->R_last, 0, sizeof(unsigned long long) * 2 * nn, c->stream);
    c->field_smem = (unsigned)((kFieldThreads + 1) * sizeof(double));
    if (cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->field_smem) != cudaSuccess) {
        pic_destroy(c);
        return fail(PIC_ECUDA, "field kernel shared memory attribute");
    }
    pic_status st = reset_moments(c);
    if (st != PIC_OK) { pic_destroy(c); return st; }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) { pic_destroy(c); return fail(PIC_ECUDA, "create sync"); }
    *out = c;
    return PIC_OK;
}

pic_status pic_load_xsec_table(pic_case *c, int species, int kind, double thr, const double *e, const double *s, int n)
{
    if (!c || species < 0 || species >= c->d.n_species || !e || !s || n < 1) return fail(PIC_EINVAL, "bad table arguments");
    if (kind < PIC_ELASTIC || kind > PIC_CX) return fail(PIC_EINVAL, "unknown process kind");
    if ((int)c->proc[species].size() >= kMaxProc) return fail(PIC_EINVAL, "too many processes for this species");
    if (species == 0 && c->d.const_nu_e_per_s > 0) return fail(PIC_EINVAL, "tables and the constant-frequency model are exclusive");
    for (int i = 1; i < n; ++i)
        if (!(e[i] >= e[i - 1])) return fail(PIC_EINVAL, "table energies must ascend");
    Proc p;
    p.kind = kind;
    p.thr = thr;
    p.nu.resize(kNGrid);
    const double mu = reduced_mass(c, species);
    for (int i = 0; i < kNGrid; ++i) {
        const double eps = grid_energy(i);
        const double sig = eps < thr ? 0.0 : sample_table(e, s, n, eps);
        p.nu[i] = c->d.gas_density_m3 * sig * std::sqrt(2.0 * eps * kElem / mu);
    }
    c->proc[species].push_back(std::move(p));
    drop_graph(c);
    fill_species(c, species);
    return upload_tables(c, species);
}

pic_status pic_load_particles(pic_case *c, int sp, int64_t n, const int32_t *cell, const float *off, const float *vx,
                              const float *vy, const float *vz, const uint32_t *id, int on_device)
{
    if (!c || sp < 0 || sp >= c->d.n_species || n < 0) return fail(PIC_EINVAL, "bad load arguments");
    if (n > 0 && (!cell || !off || !vx || !vy || !vz)) return fail(PIC_EINVAL, "null particle array");
    Ctrl h;
    pic_status st = load_begin(c, sp, n, &h);
    if (st != PIC_OK) return st;
    const SpeciesBufs &B = c->P.buf[sp][0];
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n > 0) {
        CU(cudaMemcpyAsync(B.cell, cell, n * 4, k, c->stream));
        CU(cudaMemcpyAsync(B.off, off, n * 4, k, c->stream));
        CU(cudaMemcpyAsync(B.vx, vx, n * 4, k, c->stream));
        CU(cudaMemcpyAsync(B.vy, vy, n * 4, k, c->stream));
        CU(cudaMemcpyAsync(B.vz, vz, n * 4, k, c->stream));
        if (id) CU(cudaMemcpyAsync(B.id, id, n * 4, k, c->stream));
    }
    if (n > 0 && !id) {
        const long long blocks = std::min<long long>((n + 255) / 256, 4LL * c->num_sms);
        k_iota_u32<<<(unsigned)blocks, 256, 0, c->stream>>>(B.id, n);
        CU(cudaGetLastError());
    }
    return load_finish(c, sp, n, h);
}

pic_status pic_load_particles_si(pic_case *c, int sp, int64_t n, const double *x_m, const double *v_m_per_s,
                                 const uint32_t *id, int on_device)
{
    if (!c || sp < 0 || sp >= c->d.n_species || n < 0) return fail(PIC_EINVAL, "bad load arguments");
    if (n > 0 && (!x_m || !v_m_per_s)) return fail(PIC_EINVAL, "null particle array");
    Ctrl h;
    pic_status st = load_begin(c, sp, n, &h);
    if (st != PIC_OK) return st;
    if (n > 0) {
        const double *dx_ = x_m, *dv = v_m_per_s;
        const uint32_t *did = id;
        void *tmp = nullptr;
        if (!on_device) {                                 // staged through one device buffer
            const size_t bytes = (size_t)n * (4 * sizeof(double)) + (id ? (size_t)n * 4 : 0);
            CU(cudaMallocAsync(&tmp, bytes, c->stream));
            double *tx = (double *)tmp, *tv = tx + n;
            CU(cudaMemcpyAsync(tx, x_m, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            CU(cudaMemcpyAsync(tv, v_m_per_s, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            dx_ = tx;
            dv = tv;
            if (id) {
                uint32_t *ti = (uint32_t *)(tv + 3 * n);
                CU(cudaMemcpyAsync(ti, id, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
                did = ti;
            }
        }
        const int grid = (int)std::min<long long>((n + 255) / 256, (long long)c->num_sms * 16);
        k_load_si<<<grid, 256, 0, c->stream>>>(c->P.buf[sp][0], n, c->d.n_cells, 1.0 / c->P.dx, c->d.length_m, dx_, dv,
                                               did);
        CU(cudaGetLastError());
        if (tmp) CU(cudaFreeAsync(tmp, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return load_finish(c, sp, n, h);
}

pic_status pic_load_profile(pic_case *c, int sp, int64_t n, const double *density, const double *temp_ev,
                            const double drift[3], uint32_t id_base)
{
    if (!c || sp < 0 || sp >= c->d.n_species || n < 0 || !density || !temp_ev) return fail(PIC_EINVAL, "bad profile load");
    const int N = c->d.n_cells, nn = c->n_nodes;
    // cumulative CIC mass per cell of the linear density between nodes (node N = node 0 when periodic)
    std::vector<double> cdf(N + 1, 0.0);
    std::vector<float> dn(N + 1), tn(N + 1);
    for (int j = 0; j <= N; ++j) {
        const int jj = (c->d.periodic && j == N) ? 0 : j;
        if (!(density[jj] >= 0.0) || !(temp_ev[jj] >= 0.0)) return fail(PIC_EINVAL, "negative or NaN profile value");
        dn[j] = (float)density[jj];
        tn[j] = (float)temp_ev[jj];
    }
    for (int j = 0; j < N; ++j) cdf[j + 1] = cdf[j] + 0.5 * (density[j] + density[(c->d.periodic && j + 1 == N) ? 0 : j + 1]);
    const double total = cdf[N];
    if (n > 0 && !(total > 0.0)) return fail(PIC_EINVAL, "profile density integrates to zero");
    for (int j = 1; j < N; ++j) cdf[j] /= total;
    cdf[N] = 1.0;
    (void)nn;
    Ctrl h;
    pic_status st = load_begin(c, sp, n, &h);
    if (st != PIC_OK) return st;
    if (n > 0) {
        const size_t bytes = (N + 1) * (sizeof(double) + 2 * sizeof(float));
        void *tmp = nullptr;
        CU(cudaMallocAsync(&tmp, bytes, c->stream));
        double *d_cdf = (double *)tmp;
        float *d_dn = (float *)(d_cdf + (N + 1)), *d_tn = d_dn + (N + 1);
        CU(cudaMemcpyAsync(d_cdf, cdf.data(), (N + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CU(cudaMemcpyAsync(d_dn, dn.data(), (N + 1) * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CU(cudaMemcpyAsync(d_tn, tn.data(), (N + 1) * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        const float vt = (float)std::sqrt(kElem / c->d.mass_kg[sp]);
        const double z3[3] = {0, 0, 0};
        const double *dr = drift ? drift : z3;
        const int grid = (int)std::min<long long>((n + 255) / 256, (long long)c->num_sms * 16);
        k_load_profile<<<grid, 256, 0, c->stream>>>(c->P.buf[sp][0], n, N, d_cdf, d_dn, d_tn, vt, (float)dr[0],
                                                    (float)dr[1], (float)dr[2], id_base, sp, c->P.push.key0, c->P.push.key1);
        CU(cudaGetLastError());
        CU(cudaFreeAsync(tmp, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return load_finish(c, sp, n, h);
}

pic_status pic_warmstart_load(pic_case *c, pic_mlp *m, const double *params, int n_params, int n_points,
                              double ion_temp_ev, uint32_t id_base, int64_t max_per_species)
{
    if (!c || !m || !params || n_params < 1 || n_points < 2 || !(ion_temp_ev >= 0) || max_per_species < 0)
        return fail(PIC_EINVAL, "bad warm-start arguments");
    std::vector<float> x((size_t)n_params), y((size_t)3 * n_points);
    for (int k = 0; k < n_params; ++k) x[(size_t)k] = (float)params[k];
    pic_status st = pic_mlp_predict(m, x.data(), 1, y.data());
    if (st != PIC_OK) return st;
    const int N = c->d.n_cells, nn = c->n_nodes;
    std::vector<double> ne(nn), ni(nn), te(nn), ti(nn, ion_temp_ev);
    for (int i = 0; i < nn; ++i) {                      // the predicted points span [0, L] uniformly
        const double s = (double)i / N * (n_points - 1);
        const int k = std::min((int)s, n_points - 2);
        const double t = s - k;
        auto lerp = [&](int base) { return (1 - t) * y[(size_t)(base + k)] + t * y[(size_t)(base + k + 1)]; };
        ne[i] = std::pow(10.0, lerp(0));
        ni[i] = std::pow(10.0, lerp(n_points));
        te[i] = std::max(0.0, lerp(2 * n_points));
    }
    const double dx = c->P.dx;
    int64_t n_s[2] = {0, 0};
    for (int s = 0; s < c->d.n_species && s < 2; ++s) {
        const std::vector<double> &d = s == 0 ? ne : ni;
        double integral = 0;                             // particles per area, trapezoid over the cells
        for (int j = 0; j < N; ++j) integral += 0.5 * (d[j] + d[(c->d.periodic && j + 1 == N) ? 0 : j + 1]) * dx;
        n_s[s] = (int64_t)std::llround(integral / c->d.weight_per_m2[s]);
        if (max_per_species > 0) n_s[s] = std::min(n_s[s], max_per_species);
    }
    st = pic_load_profile(c, 0, n_s[0], ne.data(), te.data(), nullptr, id_base);
    if (st != PIC_OK || c->d.n_species < 2) return st;
    return pic_load_profile(c, 1, n_s[1], ni.data(), ti.data(), nullptr, id_base);
}

pic_status pic_step(pic_case *c, int64_t n_steps)
{
    if (!c || n_steps < 0) return fail(PIC_EINVAL, "bad step arguments");
    for (int s = 0; s < c->d.n_species; ++s)
        if (!c->loaded[s] && !(s == 1 && c->loaded[0])) return fail(PIC_ESTATE, "particles not loaded");
    if (c->need_init) {
        pic_status st = initialise(c);
        if (st != PIC_OK) return st;
    }
    int64_t left = n_steps;
    auto sort_due = [&]() -> pic_status {
        for (int s = 0; s < c->d.n_species; ++s)
            if (c->since_sort[s] >= c->sort_k[s]) {
                CU(launch_sort(c, s));
                c->since_sort[s] = 0;
            }
        return PIC_OK;
    };
    while (left > 0) {
        if (c->autotune && !c->tuned && c->host_step > 0 && left >= kTuneTotalSteps) {
            pic_status st = autotune(c, &left);
            if (st != PIC_OK) return st;
            continue;
        }
        pic_status st = sort_due();
        if (st != PIC_OK) return st;
        // steps before the next sort of any species (at least one)
        long long room = kGraphSteps;
        for (int s = 0; s < c->d.n_species; ++s) room = std::min(room, c->sort_k[s] - c->since_sort[s]);
        // replay a graph of that many steps (steps run directly while
        // profiling, and for the first step after a load)
        if (!c->prof && c->host_step > 0) {
            const int seg = (int)std::min<long long>(left, room);
            if (std::memcmp(&c->graph_P, &c->P, sizeof(StepConst)) != 0) drop_graph(c);
            if (!c->graph[seg]) {
                st = build_graphs(c);
                if (st != PIC_OK) return st;
                st = build_graph(c, seg);
                if (st != PIC_OK) return st;
            }
            CU(cudaGraphLaunch(c->graph[seg], c->stream));
            c->launches[KC_STEP] += (long long)seg * c->d.n_species;
            c->launches[KC_FIELD] += seg;
            c->host_step += seg;
            for (int s = 0; s < 2; ++s) c->since_sort[s] += seg;
            left -= seg;
        } else {
            CU(launch_one_step(c));
            c->host_step++;
            for (int s = 0; s < 2; ++s) c->since_sort[s]++;
            left--;
        }
    }
    return sort_due();
}

pic_status pic_sync(pic_case *c)
{
    if (!c) return fail(PIC_EINVAL, "null case");
    CU(cudaStreamSynchronize(c->stream));
    return device_error(c);
}

pic_status pic_clear_error(pic_case *c)
{
    if (!c) return fail(PIC_EINVAL, "null case");
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaMemsetAsync(&c->P.ctrl->err, 0, sizeof(unsigned), c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_set_wait_limit(pic_case *c, uint32_t polls)
{
    if (!c) return fail(PIC_EINVAL, "null case");
    c->P.wait_polls = polls;
    drop_graph(c);                                   // captured launches carry the old limit
    return PIC_OK;
}

pic_status pic_count(pic_case *c, int64_t n_alive[2])
{
    if (!c || !n_alive) return fail(PIC_EINVAL, "null argument");
    Ctrl h;
    CU(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < 2; ++s)
        n_alive[s] = s < c->d.n_species ? (int64_t)(h.n_total[s] - h.n_dead[s]) : 0;
    return device_error(c);
}

pic_status pic_read_particles(pic_case *c, int sp, int64_t max_n, int64_t *n_out, int32_t *cell, float *off, float *vx,
                              float *vy, float *vz, uint32_t *id)
{
    if (!c || sp < 0 || sp >= c->d.n_species || max_n < 0) return fail(PIC_EINVAL, "bad read arguments");
    Ctrl h;
    CU(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    const size_t n = (size_t)h.n_total[sp];
    const SpeciesBufs &B = c->P.buf[sp][h.cur[sp]];
    std::vector<int32_t> hc(n);
    std::vector<float> ho(n), hx(n), hy(n), hz(n);
    std::vector<uint32_t> hi(n);
    if (n) {
        CU(cudaMemcpy(hc.data(), B.cell, n * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(ho.data(), B.off, n * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(hx.data(), B.vx, n * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(hy.data(), B.vy, n * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(hz.data(), B.vz, n * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(hi.data(), B.id, n * 4, cudaMemcpyDeviceToHost));
    }
    int64_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        if (hc[i] < 0) continue;
        if (k < max_n) {
            if (cell) cell[k] = hc[i] & kCellMask;
            if (off) off[k] = ho[i];
            if (vx) vx[k] = hx[i];
            if (vy) vy[k] = hy[i];
            if (vz) vz[k] = hz[i];
            if (id) id[k] = hi[i];
        }
        ++k;
    }
    if (n_out) *n_out = k;
    if (k > max_n) return fail(PIC_ECAPACITY, "output buffers smaller than the live count");
    return device_error(c);
}

pic_status pic_read_clock(pic_case *c, int sp, int64_t max_n, int64_t *n_out, uint32_t *clock)
{
    if (!c || sp < 0 || sp >= c->d.n_species || max_n < 0) return fail(PIC_EINVAL, "bad read arguments");
    Ctrl h;
    CU(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    const size_t n = (size_t)h.n_total[sp];
    std::vector<int32_t> hc(n);
    if (n) CU(cudaMemcpy(hc.data(), c->P.buf[sp][h.cur[sp]].cell, n * 4, cudaMemcpyDeviceToHost));
    int64_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        if (hc[i] < 0) continue;
        if (k < max_n && clock) clock[k] = (uint32_t)hc[i] >> kCellBits;
        ++k;
    }
    if (n_out) *n_out = k;
    if (k > max_n) return fail(PIC_ECAPACITY, "output buffer smaller than the live count");
    return device_error(c);
}

pic_status pic_read_axial(pic_case *c, int sp, int64_t max_n, int64_t *n_out, float *z)
{
    if (!c || sp < 0 || sp >= c->d.n_species || max_n < 0) return fail(PIC_EINVAL, "bad read arguments");
    if (!c->P.buf[sp][0].z) return fail(PIC_ESTATE, "the case has no axial renewal");
    Ctrl h;
    CU(cudaMemcpyAsync(&h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    const size_t n = (size_t)h.n_total[sp];
    const SpeciesBufs &B = c->P.buf[sp][h.cur[sp]];
    std::vector<int32_t> hc(n);
    std::vector<float> hz(n);
    if (n) {
        CU(cudaMemcpy(hc.data(), B.cell, n * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(hz.data(), B.z, n * 4, cudaMemcpyDeviceToHost));
    }
    int64_t k = 0;
    for (size_t i = 0; i < n; ++i) {                 // live slots, in pic_read_particles' order
        if (hc[i] < 0) continue;
        if (k < max_n && z) z[k] = hz[i];
        ++k;
    }
    if (n_out) *n_out = k;
    if (k > max_n) return fail(PIC_ECAPACITY, "output buffer smaller than the live count");
    return device_error(c);
}

pic_status pic_read_field(pic_case *c, double *phi, double *E, int64_t *rho_raw)
{
    if (!c) return fail(PIC_EINVAL, "null case");
    const size_t nn = (size_t)c->n_nodes;
    if (phi) CU(cudaMemcpyAsync(phi, c->P.phi, nn * 8, cudaMemcpyDeviceToHost, c->stream));
    if (E) CU(cudaMemcpyAsync(E, c->P.E, nn * 8, cudaMemcpyDeviceToHost, c->stream));
    if (rho_raw) CU(cudaMemcpyAsync(rho_raw, c->R_last, (size_t)c->d.n_species * nn * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return device_error(c);
}

pic_status pic_set_step_shape(pic_case *c, int species, int threads, int stages)
{
    if (!c) return fail(PIC_EINVAL, "null case");
    if (species < 0 || species >= c->d.n_species) return fail(PIC_EINVAL, "bad species");
    if (threads != 256 && threads != 512 && threads != 1024) return fail(PIC_EINVAL, "threads must be 256, 512 or 1024");
    if (stages < 0 || stages > kMaxStages) return fail(PIC_EINVAL, "stages must be in [0, 4]");
    c->step_threads[species] = threads;
    c->step_stages[species] = stages;
    drop_graph(c);
    return PIC_OK;
}

pic_status pic_read_tuning(pic_case *c, pic_tuning *t)
{
    if (!c || !t) return fail(PIC_EINVAL, "null argument");
    if (t->struct_size != sizeof(pic_tuning)) return fail(PIC_EINVAL, "pic_tuning size mismatch");
    t->tuned = c->tuned ? 1 : 0;
    for (int s = 0; s < 2; ++s) {
        t->sort_interval[s] = c->sort_k[s];
        t->threads[s] = c->step_threads[s];
        t->stages[s] = c->step_grid_stages[s] >= 0 ? c->step_grid_stages[s] : c->step_stages[s];
        t->grid[s] = c->step_grid[s];
        for (int k = 0; k < 6; ++k) t->shape_ms[s][k] = c->tune_shape_ms[s][k];
        t->sort_ms[s] = c->tune_sort_ms[s];
        t->slope_ms[s] = c->tune_slope_ms[s];
    }
    return PIC_OK;
}

pic_status pic_read_moments(pic_case *c, pic_moments *m)
{
    if (!c || !m || m->struct_size != sizeof(pic_moments)) return fail(PIC_EINVAL, "bad moments struct");
    const size_t nn = (size_t)c->n_nodes;
    const size_t ns = (size_t)c->d.n_species;
    // every piece is copied into one pinned host buffer (asynchronous copies,
    // one synchronisation), then out of it on the host
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t o_ke = al(sizeof(Ctrl)), o_pw = o_ke + 16, o_rs = o_pw + 16, o_rd = o_rs + al(2 * nn * 8),
                 o_phi = o_rd + al(2 * nn * 8), o_en = o_phi + al(nn * 8), o_ee = o_en + al(ns * nn * 8),
                 o_ifd = o_ee + al(kEepfBins * 8), need = o_ifd + al(2 * kIfedfBins * 8);
    if (c->h_stage_bytes < need) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        CU(cudaMallocHost(&c->h_stage, need));
        c->h_stage_bytes = need;
    }
    char *hb = static_cast<char *>(c->h_stage);
    CU(cudaMemcpyAsync(hb, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hb + o_ke, c->P.ke_sum, 16, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hb + o_pw, c->P.pw_sum, 16, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hb + o_rs, c->P.Rsum, 2 * nn * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hb + o_rd, c->P.Rdiag, 2 * nn * 8, cudaMemcpyDeviceToHost, c->stream));
    if (m->phi_sum) CU(cudaMemcpyAsync(hb + o_phi, c->P.phi_sum, nn * 8, cudaMemcpyDeviceToHost, c->stream));
    if (m->en_sum) CU(cudaMemcpyAsync(hb + o_en, c->P.en_sum, ns * nn * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hb + o_ee, c->P.eepf, kEepfBins * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hb + o_ifd, c->P.ifedf, 2 * kIfedfBins * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    Ctrl h;
    std::memcpy(&h, hb, sizeof(Ctrl));
    const double *ke = reinterpret_cast<const double *>(hb + o_ke), *pw = reinterpret_cast<const double *>(hb + o_pw);
    const unsigned long long *rs = reinterpret_cast<const unsigned long long *>(hb + o_rs);
    const unsigned long long *rd = reinterpret_cast<const unsigned long long *>(hb + o_rd);
    const unsigned long long *ee = reinterpret_cast<const unsigned long long *>(hb + o_ee);
    const unsigned long long *ifd = reinterpret_cast<const unsigned long long *>(hb + o_ifd);
    if (m->phi_sum) std::memcpy(m->phi_sum, hb + o_phi, nn * 8);
    if (m->en_sum) std::memcpy(m->en_sum, hb + o_en, ns * nn * 8);
    m->n_nodes = (int32_t)nn;
    m->step = h.step;
    m->n_steps = (int64_t)h.n_steps_acc;
    m->n_diag = (int64_t)h.n_diag_acc;
    for (int s = 0; s < 2; ++s) {
        m->n_alive[s] = s < (int)ns ? (int64_t)(h.n_total[s] - h.n_dead[s]) : 0;
        m->absorbed[s][0] = (int64_t)h.absorbed[s][0];
        m->absorbed[s][1] = (int64_t)h.absorbed[s][1];
        m->candidates[s] = (int64_t)h.cand[s];
        for (int k = 0; k < PIC_MAX_PROC; ++k) m->collisions[s][k] = (int64_t)h.coll[s][k];
        m->ke_sum[s] = s < (int)ns ? ke[s] : 0.0;
        m->pw_sum[s] = s < (int)ns ? pw[s] : 0.0;
    }
    // densities from the exact integer deposit sums: w R 2^-32 / node volume
    for (size_t s = 0; s < ns; ++s)
        for (size_t i = 0; i < nn; ++i) {
            const double vol = (!c->d.periodic && (i == 0 || i == nn - 1)) ? c->P.vol_wall : c->P.vol_interior;
            const double f = c->d.weight_per_m2[s] / 4294967296.0 / vol;
            if (m->dens_sum) m->dens_sum[s * nn + i] = f * (double)rs[s * nn + i];
            if (m->dens_diag_sum) m->dens_diag_sum[s * nn + i] = f * (double)rd[s * nn + i];
        }
    m->sort_interval = c->d.n_species > 1 ? std::min(c->sort_k[0], c->sort_k[1]) : c->sort_k[0];
    m->see_emitted = (int64_t)h.see;
    m->ionizations = (int64_t)h.iz;
    if (m->eepf) for (int b = 0; b < kEepfBins; ++b) m->eepf[b] = (double)ee[b];
    if (m->ifedf) for (int b = 0; b < 2 * kIfedfBins; ++b) m->ifedf[b] = (double)ifd[b];
    m->electrode_charge = h.q_el;
    m->renewed[0] = (int64_t)h.renewed[0];
    m->renewed[1] = (int64_t)h.renewed[1];
    // the oldest `want` entries of the ring that are still held: at most two
    // contiguous pieces of it, copied only when asked for
    const long long cap = c->P.fe_cap;
    const long long have = std::min<long long>((long long)h.fe_n, cap);
    long long want = m->field_energy ? std::min<long long>(have, m->field_energy_cap) : 0;
    if (want > 0) {
        std::vector<double> fe((size_t)want * kFieldCluster);
        const long long p0 = ((long long)h.fe_n - have) % cap;
        const long long n1 = std::min(want, cap - p0);
        CU(cudaMemcpyAsync(fe.data(), c->P.fe_hist + (size_t)p0 * kFieldCluster, (size_t)n1 * kFieldCluster * 8,
                           cudaMemcpyDeviceToHost, c->stream));
        if (want > n1)
            CU(cudaMemcpyAsync(fe.data() + (size_t)n1 * kFieldCluster, c->P.fe_hist,
                               (size_t)(want - n1) * kFieldCluster * 8, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        for (long long i = 0; i < want; ++i) {
            double v = 0.0;
            for (int r = 0; r < kFieldCluster; ++r) v += fe[(size_t)i * kFieldCluster + r];   // rank order
            m->field_energy[i] = v;
        }
    }
    m->field_energy_n = want;
    pic_status st = device_error(c);
    if (m->reset) {
        pic_status r = reset_moments(c);
        if (r != PIC_OK) return r;
        CU(cudaStreamSynchronize(c->stream));
    }
    return st;
}

pic_status pic_profile(pic_case *c, int enable)
{
    if (!c) return fail(PIC_EINVAL, "null case");
    CU(cudaStreamSynchronize(c->stream));
    c->prof = enable != 0;
    if (enable) {
        c->ev_used.clear();
        for (int k = 0; k < pic_case::kClasses; ++k) c->launches[k] = 0;
    }
    return PIC_OK;
}

pic_status pic_profile_read(pic_case *c, pic_kernel_stat *out, int max_entries, int *n_out)
{
    if (!c || (max_entries > 0 && !out)) return fail(PIC_EINVAL, "bad profile arguments");
    CU(cudaStreamSynchronize(c->stream));
    double ms[pic_case::kClasses] = {0, 0, 0, 0};
    long long timed[pic_case::kClasses] = {0, 0, 0, 0};
    for (auto &u : c->ev_used) {
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, c->ev_pool[u.second].first, c->ev_pool[u.second].second));
        ms[u.first] += t;
        timed[u.first] += 1;
    }
    const int n = std::min(max_entries, pic_case::kClasses);
    for (int k = 0; k < n; ++k) {
        std::memset(out[k].name, 0, sizeof(out[k].name));
        std::strncpy(out[k].name, kClassName[k], sizeof(out[k].name) - 1);
        out[k].launches = c->launches[k];
        out[k].timed = timed[k];
        out[k].total_ms = ms[k];
    }
    if (n_out) *n_out = n;
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint: header, control block, particles of the current halves, then
// fixed-size device arrays, in this order.
// ---------------------------------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'P', 'I', 'C', '1', 'D', '3', 'V', 'C'};
constexpr uint32_t kCkptVersion = 3;

struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t n_cells, n_species, n_nodes, r_stride, deposit_copies, need_init;
    int64_t fe_cap, host_step, since_sort[2];
    int32_t sort_k[2], threads[2], stages[2], tuned, autotune, has_z, pad_;
    double dt, length, q[2], m[2], w[2];
    uint64_t seed;
    uint64_t n_slots[2];           // particle slots saved per species
};

// The device arrays after the particles: (pointer, bytes) in save order.
std::vector<std::pair<void *, size_t>> ckpt_arrays(const pic_case *c)
{
    const StepConst &P = c->P;
    const size_t nn = (size_t)c->n_nodes, N = (size_t)c->d.n_cells;
    return {
        {P.E32p, sizeof(float2) * ((N + 1) / 2 * 2)}, {P.E, 8 * nn}, {P.phi, 8 * nn},
        {P.R[0], 8 * (size_t)kDepositCopies * P.r_stride}, {P.R[1], 8 * (size_t)kDepositCopies * P.r_stride},
        {c->R_last, 8 * 2 * nn}, {P.Rsum, 8 * 2 * nn}, {P.Rdiag, 8 * 2 * nn}, {P.en_sum, 8 * 2 * nn},
        {P.phi_sum, 8 * nn}, {P.ke_sum, 16}, {P.pw_sum, 16}, {P.eepf, 8 * (size_t)kEepfBins},
        {P.ifedf, 8 * 2 * (size_t)kIfedfBins}, {P.fe_hist, 8 * (size_t)P.fe_cap * kFieldCluster},
    };
}

pic_status ckpt_layout(pic_case *c, Ctrl *h, uint64_t *total)
{
    CU(cudaMemcpyAsync(h, c->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    uint64_t b = sizeof(CkptHeader) + sizeof(Ctrl);
    const uint64_t per = c->P.buf[0][0].z ? 28ull : 24ull;        // + axial excursion
    for (int s = 0; s < c->d.n_species; ++s)
        if (c->loaded[s] || (s == 1 && c->loaded[0])) b += per * h->n_total[s];
    for (auto &a : ckpt_arrays(c)) b += a.second;
    *total = b;
    return PIC_OK;
}

} // namespace

extern "C" {

pic_status pic_checkpoint_size(pic_case *c, uint64_t *bytes)
{
    if (!c || !bytes) return fail(PIC_EINVAL, "null argument");
    Ctrl h;
    return ckpt_layout(c, &h, bytes);
}

pic_status pic_checkpoint_save(pic_case *c, void *host, uint64_t bytes)
{
    if (!c || !host) return fail(PIC_EINVAL, "null argument");
    Ctrl h;
    uint64_t need = 0;
    pic_status st = ckpt_layout(c, &h, &need);
    if (st != PIC_OK) return st;
    if (bytes < need) return fail(PIC_EINVAL, "checkpoint buffer too small");
    st = device_error(c);
    if (st != PIC_OK) return st;
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.version = kCkptVersion;
    hd.header_bytes = sizeof(CkptHeader);
    hd.n_cells = c->d.n_cells; hd.n_species = c->d.n_species; hd.n_nodes = c->n_nodes;
    hd.r_stride = c->P.r_stride; hd.deposit_copies = kDepositCopies; hd.need_init = c->need_init ? 1 : 0;
    hd.fe_cap = c->P.fe_cap; hd.host_step = c->host_step;
    hd.tuned = c->tuned ? 1 : 0; hd.autotune = c->autotune ? 1 : 0;
    hd.has_z = c->P.buf[0][0].z ? 1 : 0;
    for (int s = 0; s < 2; ++s) {
        hd.since_sort[s] = c->since_sort[s]; hd.sort_k[s] = c->sort_k[s];
        hd.threads[s] = c->step_threads[s]; hd.stages[s] = c->step_stages[s];
        hd.q[s] = c->d.charge_C[s]; hd.m[s] = c->d.mass_kg[s]; hd.w[s] = c->d.weight_per_m2[s];
        hd.n_slots[s] = (s < c->d.n_species && (c->loaded[s] || (s == 1 && c->loaded[0]))) ? h.n_total[s] : 0;
    }
    hd.dt = c->d.dt_s; hd.length = c->d.length_m; hd.seed = c->d.seed;
    char *p = static_cast<char *>(host);
    std::memcpy(p, &hd, sizeof hd); p += sizeof hd;
    std::memcpy(p, &h, sizeof h); p += sizeof h;
    for (int s = 0; s < 2; ++s) {
        const size_t n = hd.n_slots[s];
        if (!n) continue;
        const SpeciesBufs &B = c->P.buf[s][h.cur[s]];
        const void *src[7] = {B.cell, B.off, B.vx, B.vy, B.vz, B.id, B.z};
        for (int a = 0; a < (hd.has_z ? 7 : 6); ++a) {
            CU(cudaMemcpyAsync(p, src[a], 4 * n, cudaMemcpyDeviceToHost, c->stream));
            p += 4 * n;
        }
    }
    for (auto &a : ckpt_arrays(c)) {
        CU(cudaMemcpyAsync(p, a.first, a.second, cudaMemcpyDeviceToHost, c->stream));
        p += a.second;
    }
    CU(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_checkpoint_load(pic_case *c, const void *host, uint64_t bytes)
{
    if (!c || !host) return fail(PIC_EINVAL, "null argument");
    if (bytes < sizeof(CkptHeader) + sizeof(Ctrl)) return fail(PIC_EINVAL, "checkpoint buffer too small");
    CkptHeader hd;
    const char *p = static_cast<const char *>(host);
    std::memcpy(&hd, p, sizeof hd);
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion || hd.header_bytes != sizeof hd)
        return fail(PIC_EINVAL, "not a checkpoint of this library version");
    bool same = hd.n_cells == c->d.n_cells && hd.n_species == c->d.n_species && hd.n_nodes == c->n_nodes &&
                hd.r_stride == c->P.r_stride && hd.deposit_copies == kDepositCopies && hd.fe_cap == c->P.fe_cap &&
                hd.dt == c->d.dt_s && hd.length == c->d.length_m && hd.seed == c->d.seed;
    for (int s = 0; s < c->d.n_species; ++s)
        same = same && hd.q[s] == c->d.charge_C[s] && hd.m[s] == c->d.mass_kg[s] && hd.w[s] == c->d.weight_per_m2[s];
    same = same && hd.has_z == (c->d.axial_length_m > 0 ? 1 : 0);
    if (!same) return fail(PIC_EINVAL, "checkpoint of a different case descriptor");
    uint64_t need = sizeof hd + sizeof(Ctrl) + (hd.has_z ? 28ull : 24ull) * (hd.n_slots[0] + hd.n_slots[1]);
    for (auto &a : ckpt_arrays(c)) need += a.second;
    if (bytes < need) return fail(PIC_EINVAL, "checkpoint buffer too small");
    CU(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < c->d.n_species; ++s) {
        pic_status st = alloc_species(c, s, (long long)hd.n_slots[s]);
        if (st != PIC_OK) return st;
    }
    Ctrl h;
    std::memcpy(&h, p + sizeof hd, sizeof h);
    p += sizeof hd + sizeof h;
    for (int s = 0; s < 2; ++s) {
        const size_t n = hd.n_slots[s];
        h.cur[s] = 0;                                  // particles go to half 0
        if (!n) continue;
        const SpeciesBufs &B = c->P.buf[s][0];
        void *dst[7] = {B.cell, B.off, B.vx, B.vy, B.vz, B.id, B.z};
        for (int a = 0; a < (hd.has_z ? 7 : 6); ++a) {
            CU(cudaMemcpyAsync(dst[a], p, 4 * n, cudaMemcpyHostToDevice, c->stream));
            p += 4 * n;
        }
    }
    CU(cudaMemcpyAsync(c->P.ctrl, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
    for (auto &a : ckpt_arrays(c)) {
        CU(cudaMemcpyAsync(a.first, p, a.second, cudaMemcpyHostToDevice, c->stream));
        p += a.second;
    }
    CU(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < c->d.n_species; ++s) {
        fill_species(c, s);                            // tables and constants of the descriptor
        c->loaded[s] = hd.n_slots[s] > 0 || s == 0;
    }
    c->need_init = hd.need_init != 0;
    c->host_step = hd.host_step;
    c->tuned = hd.tuned != 0;
    for (int s = 0; s < 2; ++s) {
        c->since_sort[s] = hd.since_sort[s];
        c->sort_k[s] = hd.sort_k[s];
        c->step_threads[s] = hd.threads[s];
        c->step_stages[s] = hd.stages[s];
    }
    drop_graph(c);
    return PIC_OK;
}

} // extern "C"

pic_status pic_destroy(pic_case *c)
{
    if (!c) return PIC_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &e : c->ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    drop_graph(c);
    while (!c->allocs.empty()) c->dfree(c->allocs.back().first);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return PIC_OK;
}

pic_status pic_philox(uint64_t seed, int64_t n, const uint32_t *ctr, uint32_t *out, void *stream)
{
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(PIC_EINVAL, "bad philox arguments");
    if (((uintptr_t)ctr | (uintptr_t)out) & 15) return fail(PIC_EINVAL, "philox buffers must be 16-byte aligned");
    if (n == 0) return PIC_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 65535);
    k_philox<<<grid, 256, 0, (cudaStream_t)stream>>>((uint32_t)seed, (uint32_t)(seed >> 32), n,
                                                      (const uint4 *)ctr, (uint4 *)out);
    CU(cudaGetLastError());
    return PIC_OK;
}

pic_status pic_deposit(int32_t n_cells, int32_t periodic, int64_t n, const int32_t *cell, const float *off, int64_t *R,
                       void *stream)
{
    if (n_cells < 2 || n < 0 || (n > 0 && (!cell || !off || !R))) return fail(PIC_EINVAL, "bad deposit arguments");
    if (n == 0) return PIC_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 65535);
    k_deposit_plain<<<grid, 256, 0, (cudaStream_t)stream>>>(n_cells, periodic, n, cell, off, (unsigned long long *)R);
    CU(cudaGetLastError());
    return PIC_OK;
}

pic_status pic_sort_by_cell(int32_t n_cells, int64_t n, const int32_t *cell, const float *off, const float *vx,
                            const float *vy, const float *vz, const uint32_t *id, int32_t *cell_out, float *off_out,
                            float *vx_out, float *vy_out, float *vz_out, uint32_t *id_out, int64_t *n_live, void *stream)
{
    if (n_cells < 1 || n_cells > 4096 || n < 0) return fail(PIC_EINVAL, "bad sort sizes");
    if (n > 0 && (!cell || !off || !vx || !vy || !vz || !id || !cell_out || !off_out || !vx_out || !vy_out ||
                  !vz_out || !id_out))
        return fail(PIC_EINVAL, "null sort array");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = n_cells;
    // scratch: per-cell counts and cursors, from the stream-ordered pool
    const size_t cnt_bytes = ((size_t)N * sizeof(unsigned) + 15) / 16 * 16;
    const size_t bytes = cnt_bytes + (size_t)(N + 1) * sizeof(unsigned long long);
    void *scratch = nullptr;
    CU(cudaMallocAsync(&scratch, bytes, st));
    unsigned *counts = (unsigned *)scratch;
    unsigned long long *cursor = (unsigned long long *)((char *)scratch + cnt_bytes);
    CU(cudaMemsetAsync(counts, 0, (size_t)N * sizeof(unsigned), st));
    CU(cudaMemsetAsync(cursor + N, 0, sizeof(unsigned long long), st));
    SortHalves H{{SpeciesBufs{const_cast<int32_t *>(cell), const_cast<float *>(off), const_cast<float *>(vx),
                              const_cast<float *>(vy), const_cast<float *>(vz), const_cast<uint32_t *>(id)},
                  SpeciesBufs{cell_out, off_out, vx_out, vy_out, vz_out, id_out}}};
    if (n > 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int gc = (int)std::min<long long>(sms * 4, std::max<long long>(1, n / 1024));
        k_cells_count<false><<<gc, 512, N * sizeof(unsigned), st>>>(H, nullptr, nullptr, n, N, counts);
        k_cells_scan<<<1, 1024, N * sizeof(double), st>>>(counts, N, cursor);
        const int gs = (int)std::min<long long>(sms, std::max<long long>(1, (n + 2047) / 2048));
        CU(allow_cells_scatter<false>());
        k_cells_scatter<false><<<gs, kScatterThreads, scatter_smem(N), st>>>(H, nullptr, nullptr, n, N, cursor);
        CU(cudaGetLastError());
    }
    if (n_live) CU(cudaMemcpyAsync(n_live, cursor + N, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    CU(cudaFreeAsync(scratch, st));
    return PIC_OK;
}

} // extern "C"

// ===========================================================================
// Batched sweep: many independent cases stepped together.
// ===========================================================================
struct pic_batch {
    std::vector<pic_case *> cases;
    std::vector<char> frozen;        // per case: left out of the steps (pic_batch_freeze)
    std::vector<pic_case *> run;     // the cases the current plan steps, in case order
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    StepConst *d_cases = nullptr;
    BatchItem *d_items = nullptr;
    SortItem *d_sort_items[2] = {nullptr, nullptr};   // batched sort blocks per species
    int n_sort_items[2] = {0, 0};
    unsigned *d_next = nullptr;
    std::vector<GridTable> grid_tab;  // shape 4: one parameter table per launch of k_batch_grid
    std::vector<int> grid_case0, grid_n, grid_sp;
    bool grid_ok = false;           // every item fits the grid kernel's table
    int *d_field_cases = nullptr;   // run-case indices grouped by field cluster size (1, 2, 4, 8)
    int n_field[4] = {}, field_off[4] = {}, field_threads[4] = {};
    int n_items = 0;
    bool planned = false;
    int periodic = 0, mcc0 = 0, mcc1 = 0;
    int stages = 0;                 // particle tiles in flight per CTA requested (0 = direct loads;
                                    // on the 256-case sweep, direct loads measured 2.23 ms/step
                                    // and two tile buffers 2.39 ms/step)
    int run_stages = 0;             // in use (fewer if shared memory is short)
    // cases with at least own_threshold particles run their own step kernels
    // (single-case kernels, 1024-thread CTAs) inside the batch's graph; the
    // rest share the persistent kernel; all field solves share one launch
    long long own_threshold = 0;
    std::vector<int> own;
    int max_cells = 0, max_nproc = 0;   // largest grid and table of the cases (shared memory layout)
    unsigned smem_of[kBatchShapes] = {};
    int grid_of[kBatchShapes] = {};   // persistent grid per launch shape (0 = not computed)
    int shape = 0;                    // launch shape of the batch kernel (BatchShape)
    int sort_k = 64;
    bool autotune = false, tuned = false;   // sort interval and shape chosen by batch_autotune
    float tune_shape_ms[kBatchShapes] = {}, tune_sort_ms = 0.f, tune_slope_ms = 0.f;
    float tune_step_ms[32] = {};      // the autotuner's timed steps after its sort (kBatchTuneSteps)
    long long host_step = 0, steps_since_sort = 0;
    cudaGraphExec_t graph[kGraphSteps + 1] = {};   // graph[k]: k batch steps
    long long launches = 0;
};

namespace {

constexpr long long kItemParticles = 262144;      // largest work item
constexpr long long kMinItemParticles = 16384;    // smallest work item when splitting for balance

// Shared memory of a batch launch shape: the largest case's tables, the draw
// queues of the shape's warps, an append buffer and the electrons'
// ionization queues (every case's layout fits in it: a case without appends
// lays out no buffer, the ions no ionization queue).
template <int M0, int M1, bool STAGED, int SHAPE>
unsigned batch_smem(const pic_batch *b)
{
    constexpr int ch = STAGED ? 4 : BatchShape<SHAPE>::chunk;
    constexpr int qcap = draw_queue_cap(M0, ch) > draw_queue_cap(M1, ch) ? draw_queue_cap(M0, ch)
                                                                            : draw_queue_cap(M1, ch);
    return StepSmem(b->max_cells, b->max_nproc, BatchShape<SHAPE>::threads, STAGED ? b->run_stages : 0, 5, qcap,
                    kAppendCap, child_queue_cap(0, M0))
        .total;
}

template <bool PER, int M0, int M1, bool STAGED, int SHAPE>
cudaError_t batch_step_k(pic_batch *b)
{
    auto k = k_batch_particle_step<PER, M0, M1, STAGED, SHAPE>;
    constexpr int T = BatchShape<SHAPE>::threads;
    const unsigned smem = batch_smem<M0, M1, STAGED, SHAPE>(b);
    int &grid = b->grid_of[SHAPE];
    if (grid == 0 || b->smem_of[SHAPE] != smem) {
        static std::once_flag once;
        static cudaError_t attr_err = cudaSuccess;
        cudaError_t e = allow_max_step_smem(k, once, attr_err, b->run[0]->device);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, T, smem);
        if (e != cudaSuccess) return e;
        grid = std::max(1, occ) * b->run[0]->num_sms;
        b->smem_of[SHAPE] = smem;
    }
    k<<<grid, T, smem, b->stream>>>(b->d_cases, b->d_items, b->n_items, b->d_next);
    return cudaGetLastError();
}

// Shape 4: the grid of work items, one launch per parameter table.
template <bool PER, int M0, int M1, int SHAPE>
cudaError_t batch_grid(pic_batch *b)
{
    auto k0 = k_batch_grid<0, PER, M0, SHAPE>;
    auto k1 = k_batch_grid<1, PER, M1, SHAPE>;
    static std::once_flag once0, once1;
    static cudaError_t err0 = cudaSuccess, err1 = cudaSuccess;
    cudaError_t e = allow_max_step_smem(k0, once0, err0, b->run[0]->device);
    if (e == cudaSuccess) e = allow_max_step_smem(k1, once1, err1, b->run[0]->device);
    if (e != cudaSuccess) return e;
    const unsigned smem = batch_smem<M0, M1, false, SHAPE>(b);
    for (size_t g = 0; g < b->grid_tab.size(); ++g) {
        const dim3 grid((unsigned)b->grid_n[g]), block(BatchShape<SHAPE>::threads);
        if (g == 0) {                               // after the previous step's field solve
            if (b->grid_sp[g] == 0) k0<<<grid, block, smem, b->stream>>>(b->grid_tab[g], b->d_cases, b->grid_case0[g]);
            else k1<<<grid, block, smem, b->stream>>>(b->grid_tab[g], b->d_cases, b->grid_case0[g]);
            e = cudaGetLastError();
        } else if (b->grid_sp[g] == 0) {
            e = launch_programmatic(k0, grid, block, smem, b->stream, b->grid_tab[g], b->d_cases, b->grid_case0[g]);
        } else {
            e = launch_programmatic(k1, grid, block, smem, b->stream, b->grid_tab[g], b->d_cases, b->grid_case0[g]);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Tile buffers (bulk-copy pipeline) exist for shape 0 only.
template <bool PER, int M0, int M1>
cudaError_t batch_step_t(pic_batch *b)
{
    if (b->run_stages > 0) return batch_step_k<PER, M0, M1, true, 0>(b);
    // a shape whose draw queues do not fit next to the largest case's tables
    // runs as shape 0 (the fewest warps, chunks of one)
    const unsigned lim = (unsigned)step_smem_limit(b->run[0]->device);
    if (b->shape == 4 && b->grid_ok && batch_smem<M0, M1, false, 2>(b) <= lim) return batch_grid<PER, M0, M1, 2>(b);
    if (b->shape == 5 && b->grid_ok && batch_smem<M0, M1, false, 3>(b) <= lim) return batch_grid<PER, M0, M1, 3>(b);
    if (b->shape == 1 && batch_smem<M0, M1, false, 1>(b) <= lim) return batch_step_k<PER, M0, M1, false, 1>(b);
    if (b->shape == 2 && batch_smem<M0, M1, false, 2>(b) <= lim) return batch_step_k<PER, M0, M1, false, 2>(b);
    if (b->shape == 3 && batch_smem<M0, M1, false, 3>(b) <= lim) return batch_step_k<PER, M0, M1, false, 3>(b);
    return batch_step_k<PER, M0, M1, false, 0>(b);
}

cudaError_t batch_particles(pic_batch *b)
{
    const int m = b->mcc0 * 3 + b->mcc1;
    if (b->periodic) {
        if (m == 0) return batch_step_t<true, 0, 0>(b);
        if (m == 4) return batch_step_t<true, 1, 1>(b);
        if (m == 6) return batch_step_t<true, 2, 0>(b);
    } else {
        if (m == 0) return batch_step_t<false, 0, 0>(b);
        if (m == 4) return batch_step_t<false, 1, 1>(b);
        if (m == 6) return batch_step_t<false, 2, 0>(b);
    }
    return cudaErrorInvalidValue;
}

int batch_launches_per_step(const pic_batch *b)
{
    int field = 0;
    for (int g = 0; g < 4; ++g) field += b->n_field[g] > 0 ? 1 : 0;
    const int particles = b->n_items == 0 ? 0 : (b->shape >= 4 && b->grid_ok) ? (int)b->grid_tab.size() : 1;
    return particles + field + (int)b->own.size() * b->run[0]->d.n_species;
}

cudaError_t batch_one_step(pic_batch *b)
{
    cudaError_t e = b->n_items > 0 ? batch_particles(b) : cudaSuccess;
    for (int i : b->own) {
        pic_case *c = b->run[(size_t)i];
        if (e == cudaSuccess) e = launch_step_sp<0>(c);
        if (e == cudaSuccess && c->d.n_species > 1) e = launch_step_sp<1>(c);
    }
    if (e != cudaSuccess) return e;
    // one launch per cluster size, each cluster as small as its case's grid allows
    const unsigned fsm = b->run[0]->field_smem;
    unsigned *reset = b->d_next;
    for (int g = 0; g < 4; ++g) {
        const int n = b->n_field[g];
        if (n == 0) continue;
        const int *cl_cases = b->d_field_cases + b->field_off[g];
        const unsigned T = (unsigned)b->field_threads[g];
        if (g == 0) k_batch_field<1><<<(unsigned)n, T, fsm, b->stream>>>(b->d_cases, cl_cases, 1, reset);
        if (g == 1) k_batch_field<2><<<(unsigned)(2 * n), T, fsm, b->stream>>>(b->d_cases, cl_cases, 1, reset);
        if (g == 2) k_batch_field<4><<<(unsigned)(4 * n), T, fsm, b->stream>>>(b->d_cases, cl_cases, 1, reset);
        if (g == 3) k_batch_field<8><<<(unsigned)(8 * n), T, fsm, b->stream>>>(b->d_cases, cl_cases, 1, reset);
        reset = nullptr;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The counting sort of every case, one launch per kernel and species (the
// cases' own count/cursor arrays; species one after the other, as they share
// them), over the sort items batch_plan made.
cudaError_t batch_sort(pic_batch *b)
{
    const unsigned nc = (unsigned)b->run.size();
    int maxN = 0;
    for (pic_case *c : b->run) maxN = std::max(maxN, c->d.n_cells);
    for (int sp = 0; sp < b->run[0]->d.n_species; ++sp) {
        const unsigned ni = (unsigned)b->n_sort_items[sp];
        k_batch_cells_count<<<ni, 512, maxN * sizeof(unsigned), b->stream>>>(b->d_cases, b->d_sort_items[sp], sp);
        k_batch_cells_scan<<<nc, 1024, maxN * sizeof(double), b->stream>>>(b->d_cases, sp);
        cudaError_t ea = allow_batch_scatter();
        if (ea != cudaSuccess) return ea;
        k_batch_cells_scatter<<<ni, kScatterThreads, scatter_smem(maxN), b->stream>>>(b->d_cases, b->d_sort_items[sp],
                                                                                       sp);
        k_batch_sort_finish<<<dim3(4, nc), 256, 0, b->stream>>>(b->d_cases, sp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void batch_drop_graph(pic_batch *b)
{
    for (auto &g : b->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

pic_status batch_plan(pic_batch *b)
{
    b->run.clear();                                 // the cases this plan steps
    for (size_t i = 0; i < b->cases.size(); ++i)
        if (!b->frozen[i]) b->run.push_back(b->cases[i]);
    batch_drop_graph(b);
    for (int &g : b->grid_of) g = 0;
    if (b->run.empty()) {
        b->planned = true;
        return PIC_OK;
    }
    const size_t nc = b->run.size();
    for (pic_case *c : b->run) {
        for (int s = 0; s < c->d.n_species; ++s)
            if (!c->loaded[s] && !(s == 1 && c->loaded[0])) return fail(PIC_ESTATE, "a batch case has no particles");
        if (c->need_init) {
            pic_status st = initialise(c);
            if (st != PIC_OK) return st;
        }
    }
    const pic_case *c0 = b->run[0];
    b->periodic = c0->d.periodic;
    b->mcc0 = c0->P.sp[0].mcc;
    b->mcc1 = c0->d.n_species > 1 ? c0->P.sp[1].mcc : 0;
    const int m = b->mcc0 * 3 + b->mcc1;
    if (m != 0 && m != 4 && m != 6)
        return fail(PIC_EINVAL, "batch supports: no collisions, tables for both species, or constant-frequency electrons");
    std::vector<BatchItem> items;
    std::vector<StepConst> consts(nc);
    // current particle counts, then slices small enough that every CTA of the
    // persistent grid gets several (at least kMinItemParticles each)
    std::vector<Ctrl> hs(nc);
    long long total = 0;
    for (size_t i = 0; i < nc; ++i) {
        CU(cudaMemcpyAsync(&hs[i], b->run[i]->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
    }
    CU(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < nc; ++i)
        for (int s = 0; s < b->run[i]->d.n_species; ++s) total += (long long)hs[i].n_active[s];
    b->own.clear();
    long long shared_total = 0;
    for (size_t i = 0; i < nc; ++i) {
        long long n = 0;
        for (int s = 0; s < b->run[i]->d.n_species; ++s) n += (long long)hs[i].n_active[s];
        if (b->own_threshold > 0 && n >= b->own_threshold) b->own.push_back((int)i);
        else shared_total += n;
    }
    (void)total;
    const long long target_items = 3LL * c0->num_sms;
    const long long item_particles =
        std::min(kItemParticles, std::max(kMinItemParticles, (shared_total + target_items - 1) / target_items));
    size_t next_own = 0;
    for (size_t i = 0; i < nc; ++i) {
        pic_case *c = b->run[i];
        if (c->d.periodic != b->periodic || c->P.sp[0].mcc != b->mcc0 ||
            (c->d.n_species > 1 ? c->P.sp[1].mcc : 0) != b->mcc1)
            return fail(PIC_EINVAL, "batch cases differ in boundary or collision model");
        if (c->P.axial_len > 0.0f) return fail(PIC_EINVAL, "axial renewal is for single cases, not batches");
        consts[i] = c->P;
        if (next_own < b->own.size() && b->own[next_own] == (int)i) {   // stepped by its own kernels
            ++next_own;
            continue;
        }
        const Ctrl &h = hs[i];
        for (int s = 0; s < c->d.n_species; ++s) {
            const long long n = (long long)h.n_active[s];
            const int nk = (int)std::max<long long>(1, (n + item_particles - 1) / item_particles);
            for (int k = 0; k < nk; ++k) items.push_back(BatchItem{(int)i, s, k, nk});
        }
    }
    // largest items first: CTAs take them in list order, so the small ones fill the tail
    std::stable_sort(items.begin(), items.end(), [&](const BatchItem &a, const BatchItem &b2) {
        const long long na = (long long)hs[(size_t)a.case_idx].n_active[a.species] / a.nk;
        const long long nb = (long long)hs[(size_t)b2.case_idx].n_active[b2.species] / b2.nk;
        return na > nb;
    });
    // shape 4: parameter tables of at most kGridCases cases and kGridItems
    // items each, items in the list's (largest first) order
    b->grid_tab.clear();
    b->grid_case0.clear();
    b->grid_n.clear();
    b->grid_sp.clear();
    b->grid_ok = true;
    for (int sp = 0; sp < c0->d.n_species && b->grid_ok; ++sp)
        for (size_t g0 = 0; g0 < nc && b->grid_ok; g0 += kGridCases) {
            GridTable t{};
            for (size_t i = 0; i < (size_t)kGridCases && g0 + i < nc; ++i) t.push[i] = consts[g0 + i].push;
            int ni = 0;
            auto flush = [&]() {
                b->grid_tab.push_back(t);
                b->grid_case0.push_back((int)g0);
                b->grid_n.push_back(ni);
                b->grid_sp.push_back(sp);
                ni = 0;
            };
            for (const BatchItem &it : items) {
                if (it.species != sp || (size_t)it.case_idx < g0 || (size_t)it.case_idx >= g0 + kGridCases) continue;
                if (it.nk >= 2048) { b->grid_ok = false; break; }
                t.item[ni++] = (uint32_t)((size_t)it.case_idx - g0) | ((uint32_t)it.k << 8) | ((uint32_t)it.nk << 19);
                if (ni == kGridItems) flush();
            }
            if (ni > 0) flush();
        }
    // tile buffers: as many as the largest case leaves room for (same for all cases)
    int stages = b->stages;
    for (size_t i = 0; i < nc; ++i) {
        const pic_case *c = b->run[i];
        for (int s = 0; s < c->d.n_species; ++s) {
            const int np = c->P.sp[s].mcc == 1 ? c->P.sp[s].nproc : 0;
            const int narr = step_arrays(s, b->periodic != 0, c->P.sp[s].mcc);
            stages = std::min(stages, fit_stages(c->d.n_cells, np, BatchShape<0>::threads, stages, narr,
                                                 draw_queue_cap(c->P.sp[s].mcc, 4), kAppendCap,
                                                 child_queue_cap(s, c->P.sp[s].mcc), step_smem_limit(c->device)));
        }
    }
    int max_cells = 0, max_nproc = 0;
    for (size_t i = 0; i < nc; ++i) {
        const pic_case *c = b->run[i];
        max_cells = std::max(max_cells, c->d.n_cells);
        for (int s = 0; s < c->d.n_species; ++s) {
            if (c->P.sp[s].mcc == 1) max_nproc = std::max(max_nproc, c->P.sp[s].nproc);
            consts[i].sp[s].stages = stages;
        }
    }
    // sort items: about one block per kSortItemParticles particles of a case
    // (counts as at this plan, doubled for growth before the next one), at
    // most one wave of the scatter kernel, in case order
    for (int sp = 0; sp < c0->d.n_species; ++sp) {
        std::vector<SortItem> si;
        for (size_t i = 0; i < nc; ++i) {
            const long long n = sp < b->run[i]->d.n_species ? 2 * (long long)hs[i].n_active[sp] : 0;
            const int nb = (int)std::max<long long>(1, std::min<long long>(2LL * c0->num_sms,
                                                                          (n + kSortItemParticles - 1) / kSortItemParticles));
            for (int k = 0; k < nb; ++k) si.push_back(SortItem{(int)i, k, nb});
        }
        if (b->d_sort_items[sp]) cudaFree(b->d_sort_items[sp]);
        b->d_sort_items[sp] = nullptr;
        CU(cudaMalloc(&b->d_sort_items[sp], si.size() * sizeof(SortItem)));
        CU(cudaMemcpyAsync(b->d_sort_items[sp], si.data(), si.size() * sizeof(SortItem), cudaMemcpyHostToDevice,
                           b->stream));
        b->n_sort_items[sp] = (int)si.size();
    }
    if (stages != b->run_stages)
        for (int &g : b->grid_of) g = 0;
    b->run_stages = stages;
    if (b->d_cases) cudaFree(b->d_cases);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_field_cases) cudaFree(b->d_field_cases);
    b->d_cases = nullptr;
    b->d_items = nullptr;
    b->d_field_cases = nullptr;
    // field solves grouped by cluster size
    std::vector<int> fcases;
    for (int g = 0; g < 4; ++g) {
        b->field_off[g] = (int)fcases.size();
        b->field_threads[g] = 64;
        for (size_t i = 0; i < nc; ++i)
            if (field_cluster_for(b->run[i]->d.n_cells) == (1 << g)) {
                fcases.push_back((int)i);
                b->field_threads[g] = std::max(b->field_threads[g], field_threads_for(b->run[i]->d.n_cells, 1 << g));
            }
        b->n_field[g] = (int)fcases.size() - b->field_off[g];
    }
    CU(cudaMalloc(&b->d_field_cases, fcases.size() * sizeof(int)));
    CU(cudaMemcpyAsync(b->d_field_cases, fcases.data(), fcases.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CU(cudaMalloc(&b->d_cases, nc * sizeof(StepConst)));
    CU(cudaMalloc(&b->d_items, std::max<size_t>(1, items.size()) * sizeof(BatchItem)));
    CU(cudaMemcpyAsync(b->d_cases, consts.data(), nc * sizeof(StepConst), cudaMemcpyHostToDevice, b->stream));
    if (!items.empty())
        CU(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, b->stream));
    CU(cudaMemsetAsync(b->d_next, 0, sizeof(unsigned), b->stream));
    CU(cudaStreamSynchronize(b->stream));
    b->n_items = (int)items.size();
    b->max_cells = max_cells;
    b->max_nproc = max_nproc;
    b->planned = true;
    batch_drop_graph(b);
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// Batch autotuner: the launch shape and the sort interval, chosen by
// measurement while the simulation continues (results do not depend on any
// choice):
//  1. each launch shape of the batch kernels runs kBatchShapeRounds steps in
//     turn, timed with events around the step; the least summed time wins;
//  2. one batched sort, then kBatchTuneSteps steps each timed with the chosen
//     shape and rescaled by the live particle count; choose_sort_interval
//     picks K from them, as for a single case.
// The tile pipeline (stages > 0) is left as the caller set it.
// ---------------------------------------------------------------------------
constexpr int kBatchShapeRounds = 2, kBatchTuneSteps = 32;
static_assert(kBatchTuneSteps <= 32, "pic_batch keeps 32 tuner step times");
constexpr int kBatchTuneTotal = kBatchShapeRounds * kBatchShapes + kBatchTuneSteps;

pic_status batch_autotune(pic_batch *b, int64_t *left)
{
    batch_drop_graph(b);
    struct Events {
        std::vector<cudaEvent_t> v;
        ~Events() { for (auto e : v) cudaEventDestroy(e); }
    } ev;
    const int n_shape_ev = 2 * kBatchShapeRounds * kBatchShapes;
    ev.v.resize(n_shape_ev + 2 + 2 * kBatchTuneSteps, nullptr);
    for (auto &e : ev.v) CU(cudaEventCreate(&e));
    const int shapes = b->run_stages > 0 ? 1 : kBatchShapes;       // tiles: shape 0 only
    for (int rnd = 0; rnd < kBatchShapeRounds; ++rnd)
        for (int k = 0; k < kBatchShapes; ++k) {
            b->shape = k < shapes ? k : 0;
            CU(cudaEventRecord(ev.v[2 * (rnd * kBatchShapes + k)], b->stream));
            CU(batch_one_step(b));
            CU(cudaEventRecord(ev.v[2 * (rnd * kBatchShapes + k) + 1], b->stream));
        }
    CU(cudaStreamSynchronize(b->stream));
    int best = 0;
    for (int k = 0; k < kBatchShapes; ++k) {               // the fastest round of each shape
        float best_t = 3.0e38f;
        for (int rnd = 0; rnd < kBatchShapeRounds; ++rnd) {
            float t = 0.f;
            CU(cudaEventElapsedTime(&t, ev.v[2 * (rnd * kBatchShapes + k)], ev.v[2 * (rnd * kBatchShapes + k) + 1]));
            best_t = std::min(best_t, t);
        }
        b->tune_shape_ms[k] = best_t;
        if (k < shapes && b->tune_shape_ms[k] < b->tune_shape_ms[best]) best = k;
    }
    b->shape = best;
    cudaEvent_t *sev = ev.v.data() + n_shape_ev, *tev = sev + 2;
    CU(cudaEventRecord(sev[0], b->stream));
    CU(batch_sort(b));
    CU(cudaEventRecord(sev[1], b->stream));
    std::vector<Ctrl> hs(b->run.size());
    auto alive = [&](double &a) -> pic_status {      // live particles of the stepped cases
        for (size_t i = 0; i < b->run.size(); ++i)
            CU(cudaMemcpyAsync(&hs[i], b->run[i]->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
        CU(cudaStreamSynchronize(b->stream));
        a = 0;
        for (size_t i = 0; i < b->run.size(); ++i)
            for (int s = 0; s < b->run[i]->d.n_species; ++s) a += (double)(hs[i].n_total[s] - hs[i].n_dead[s]);
        return PIC_OK;
    };
    double alive0 = 0, alive1 = 0;
    pic_status st = alive(alive0);
    if (st != PIC_OK) return st;
    for (int k = 0; k < kBatchTuneSteps; ++k) {
        CU(cudaEventRecord(tev[2 * k], b->stream));
        CU(batch_one_step(b));
        CU(cudaEventRecord(tev[2 * k + 1], b->stream));
    }
    st = alive(alive1);
    if (st != PIC_OK) return st;
    float ts = 0.f;
    CU(cudaEventElapsedTime(&ts, sev[0], sev[1]));
    double ty[kBatchTuneSteps];
    for (int k = 0; k < kBatchTuneSteps; ++k) {
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, tev[2 * k], tev[2 * k + 1]));
        ty[k] = t;
        b->tune_step_ms[k] = t;
    }
    normalise_to_count(ty, kBatchTuneSteps, alive0, alive1);
    const SortIntervalFit fit = choose_sort_interval(ty, kBatchTuneSteps, ts, 4, kMaxSortInterval);
    b->sort_k = std::max(4, std::min(kMaxSortInterval, fit.K));
    b->tune_sort_ms = ts;
    b->tune_slope_ms = (float)fit.slope;
    b->tuned = true;
    b->launches += (long long)batch_launches_per_step(b) * kBatchTuneTotal + 4LL * b->run[0]->d.n_species;
    b->host_step += kBatchTuneTotal;
    b->steps_since_sort = kBatchTuneSteps;
    *left -= kBatchTuneTotal;
    return PIC_OK;
}

pic_status batch_build_graph(pic_batch *b, int steps)
{
    if (b->graph[steps]) return PIC_OK;
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < steps && e == cudaSuccess; ++i) e = batch_one_step(b);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(PIC_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph[steps], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph[steps] = nullptr;
        return fail(PIC_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    }
    return PIC_OK;
}

} // namespace

extern "C" {

pic_status pic_batch_create(const pic_case_desc *descs, int n_cases, pic_batch **out)
{
    if (!descs || !out || n_cases < 1) return fail(PIC_EINVAL, "bad batch arguments");
    *out = nullptr;
    for (int i = 1; i < n_cases; ++i)
        if (descs[i].periodic != descs[0].periodic || descs[i].n_species != descs[0].n_species)
            return fail(PIC_EINVAL, "batch cases must share the boundary kind and the number of species");
    pic_batch *b = new pic_batch();
    if (descs[0].stream) b->stream = (cudaStream_t)descs[0].stream;
    else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return fail(PIC_ECUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    b->autotune = descs[0].sort_interval <= 0;
    b->sort_k = b->autotune ? 64 : descs[0].sort_interval;
    for (int i = 0; i < n_cases; ++i) {
        pic_case_desc d = descs[i];
        d.stream = b->stream;                       // every case on the batch stream
        pic_case *c = nullptr;
        pic_status st = pic_create_case(&d, &c);
        if (st != PIC_OK) {
            pic_batch_destroy(b);
            return st;
        }
        b->cases.push_back(c);
        b->frozen.push_back(0);
    }
    if (cudaMalloc(&b->d_next, sizeof(unsigned)) != cudaSuccess) {
        pic_batch_destroy(b);
        return fail(PIC_ENOMEM, "batch counter allocation failed");
    }
    *out = b;
    return PIC_OK;
}

pic_case *pic_batch_case(pic_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->cases.size()) return nullptr;
    b->planned = false;                              // the caller may load or change this case
    return b->cases[(size_t)i];
}

pic_status pic_batch_step(pic_batch *b, int64_t n_steps)
{
    if (!b || n_steps < 0) return fail(PIC_EINVAL, "bad batch step arguments");
    if (!b->planned) {
        pic_status st = batch_plan(b);
        if (st != PIC_OK) return st;
    }
    if (b->run.empty()) return PIC_OK;                // every case frozen
    int64_t left = n_steps;
    while (left > 0) {
        if (b->autotune && !b->tuned && b->host_step > 0 && left >= kBatchTuneTotal) {
            pic_status st = batch_autotune(b, &left);
            if (st != PIC_OK) return st;
            continue;
        }
        const int K = b->sort_k;
        if (b->steps_since_sort >= K) {
            CU(batch_sort(b));
            b->launches += 4LL * b->run[0]->d.n_species;
            b->steps_since_sort = 0;
        }
        // steps before the next sort, replayed as one graph (every length up
        // to the sort interval is built at the first replay)
        const int seg = (int)std::min<long long>(std::min<long long>(left, kGraphSteps), K - b->steps_since_sort);
        if (b->host_step > 0) {
            if (!b->graph[seg]) {
                for (int k = 1; k <= std::min(kGraphSteps, K); ++k) {
                    pic_status st = batch_build_graph(b, k);
                    if (st != PIC_OK) return st;
                }
            }
            CU(cudaGraphLaunch(b->graph[seg], b->stream));
            b->launches += (long long)batch_launches_per_step(b) * seg;
            b->host_step += seg;
            b->steps_since_sort += seg;
            left -= seg;
        } else {
            CU(batch_one_step(b));
            b->launches += batch_launches_per_step(b);
            b->host_step++;
            b->steps_since_sort++;
            left--;
        }
    }
    if (b->steps_since_sort >= b->sort_k) {
        CU(batch_sort(b));
        b->launches += 4LL * b->run[0]->d.n_species;
        b->steps_since_sort = 0;
    }
    return PIC_OK;
}

pic_status pic_batch_sync(pic_batch *b)
{
    if (!b) return fail(PIC_EINVAL, "null batch");
    CU(cudaStreamSynchronize(b->stream));
    for (pic_case *c : b->cases) {
        pic_status st = device_error(c);
        if (st != PIC_OK) return st;
    }
    return PIC_OK;
}

int64_t pic_batch_launches(const pic_batch *b) { return b ? b->launches : 0; }

pic_status pic_batch_set_own_threshold(pic_batch *b, int64_t particles)
{
    if (!b || particles < 0) return fail(PIC_EINVAL, "threshold must be >= 0");
    b->own_threshold = particles;
    b->planned = false;
    batch_drop_graph(b);
    return PIC_OK;
}

pic_status pic_batch_tuning(pic_batch *b, int *shape, int *sort_interval, int *tuned, float *shape_ms, float *sort_ms,
                            float *step_ms)
{
    if (!b) return fail(PIC_EINVAL, "null batch");
    if (step_ms)
        for (int k = 0; k < kBatchTuneSteps; ++k) step_ms[k] = b->tune_step_ms[k];
    if (shape) *shape = b->shape;
    if (sort_interval) *sort_interval = b->sort_k;
    if (tuned) *tuned = b->tuned ? 1 : 0;
    if (shape_ms)
        for (int k = 0; k < kBatchShapes; ++k) shape_ms[k] = b->tune_shape_ms[k];
    if (sort_ms) *sort_ms = b->tune_sort_ms;
    return PIC_OK;
}

pic_status pic_batch_freeze(pic_batch *b, int i, int frozen)
{
    if (!b || i < 0 || i >= (int)b->cases.size()) return fail(PIC_EINVAL, "case index out of range");
    CU(cudaStreamSynchronize(b->stream));
    b->frozen[(size_t)i] = frozen ? 1 : 0;
    b->planned = false;                              // re-planned at the next step
    return PIC_OK;
}

pic_status pic_batch_retune(pic_batch *b)
{
    if (!b) return fail(PIC_EINVAL, "null batch");
    b->autotune = true;
    b->tuned = false;
    return PIC_OK;
}

pic_status pic_batch_set_shape(pic_batch *b, int shape)
{
    if (!b || shape < 0 || shape >= kBatchShapes) return fail(PIC_EINVAL, "shape must be in [0, 5]");
    b->shape = shape;
    b->tuned = true;                                 // a fixed shape: the autotuner does not run
    batch_drop_graph(b);
    return PIC_OK;
}

pic_status pic_batch_set_stages(pic_batch *b, int stages)
{
    if (!b || stages < 0 || stages > kMaxStages) return fail(PIC_EINVAL, "stages must be in [0, 4]");
    b->stages = stages;
    b->planned = false;                              // re-planned (and the graph rebuilt) at the next step
    batch_drop_graph(b);
    return PIC_OK;
}

pic_status pic_batch_destroy(pic_batch *b)
{
    if (!b) return PIC_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    for (pic_case *c : b->cases) pic_destroy(c);
    if (b->d_cases) cudaFree(b->d_cases);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_field_cases) cudaFree(b->d_field_cases);
    for (SortItem *p : b->d_sort_items)
        if (p) cudaFree(p);
    if (b->d_next) cudaFree(b->d_next);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return PIC_OK;
}

} // extern "C"
